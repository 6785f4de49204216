// Per-run setup kernel (FP64): the tracer's geometry records, the source
// list with its energies and the cumulative source thresholds.
#include "launch.h"

namespace mcbte {

namespace {

// One thread per geometry: derive the tracer's geometry record and the
// source list with E_i (Eq. dev_tot / Eq. source_energy, Sec. 3.1):
//   isothermal wall  E = (A/4) sum C v |T_b - T_eq|           (Eq. iso_flux)
//   control gradient E = (V/2) |grad T| sum C v                (Eq. grad_flux over both signs)
//   initial Gaussian E = C_tot |dT| (2 pi)^{3/2} sigma^3 / 2  (Eq. Nbin; half inside the box)
// (x t_max for transient wall sources), then the cumulative source
// thresholds used with one 32-bit word (Sec. 3.2).
__global__ void k_setup(SetupArgs a, int G, MatView M, int transient, double t_max_s, int ta, GeoRun* geos,
                        uint64_t* offs, unsigned long long* t0) {
  const int gi = threadIdx.x;
  if (gi == 0) {
    *t0 = globaltimer_ns();
    uint64_t acc = 0;
    for (int k = 0; k < G; ++k) {
      offs[k] = acc;
      acc += a.n[k];
    }
    offs[G] = acc;
  }
  if (gi >= G) return;
  const mcbte_geometry_desc& d = *a.desc[gi];
  GeoRun r;
  const double C_tot = M.sums[0];
  const double sum_Cv = M.sums[1];
  for (int k = 0; k < 3; ++k) {
    r.L[k] = d.L[k] * 1e9;
    r.Lf[k] = (float)r.L[k];
  }
  r.fbin = 0;
  for (int f = 0; f < 6; ++f) {
    r.type[f] = d.face_type[f];
    r.pthr[f] = spec_threshold(d.face_p[f]);
    r.face_sign[f] = (d.face_T[f] > d.T_eq) ? 1.0 : -1.0;
    if (d.face_p[f] < 0.0) r.fbin |= 1 << f;
  }
  // internal walls: oriented with the solid on their right (normal = (dy, -dx)
  // direction), so the shoelace sum over them is the holes' area
  r.n_inner = d.n_inner;
  r.sbin = 0;
  double hole_area = 0.0;
  for (int k = 0; k < d.n_inner; ++k) {
    double x1 = d.inner[k][0], y1 = d.inner[k][1], x2 = d.inner[k][2], y2 = d.inner[k][3];
    const double nx = d.inner_n[k][0], ny = d.inner_n[k][1];
    if ((y2 - y1) * nx - (x2 - x1) * ny < 0.0) {
      const double tx = x1, ty = y1;
      x1 = x2; y1 = y2; x2 = tx; y2 = ty;
    }
    hole_area += 0.5 * (x1 * y2 - x2 * y1);
    r.sx1[k] = x1 * 1e9; r.sy1[k] = y1 * 1e9; r.sx2[k] = x2 * 1e9; r.sy2[k] = y2 * 1e9;
    r.snx[k] = nx; r.sny[k] = ny;
    r.sx1f[k] = (float)r.sx1[k]; r.sy1f[k] = (float)r.sy1[k];
    r.sx2f[k] = (float)r.sx2[k]; r.sy2f[k] = (float)r.sy2[k];
    r.snxf[k] = (float)nx; r.snyf[k] = (float)ny;
    r.sthr[k] = spec_threshold(d.inner_p[k]);
    if (d.inner_p[k] < 0.0) r.sbin |= 1 << k;
  }
  r.pore = d.pore;
  // periodic axes a flight may cross without stopping (no pore and no walls
  // inside the box: crossing a periodic face changes nothing but the position)
  r.unfold = 0;
  if (!d.pore && d.n_inner == 0)
    for (int a = 0; a < 3; ++a)
      if (r.type[axis_min_face(a)] == MCBTE_FACE_PERIODIC) r.unfold |= 1 << a;
  r.cx = d.pore_c[0] * 1e9;
  r.cy = d.pore_c[1] * 1e9;
  const double rr = d.pore_r * 1e9;
  r.r2 = rr * rr;
  r.cxf = (float)r.cx;
  r.cyf = (float)r.cy;
  r.r2f = (float)r.r2;
  r.p_pore = d.pore_p;
  r.pthr_pore = spec_threshold(d.pore_p);
  double V = d.L[0] * d.L[1] * d.L[2];
  r.V_box = V;
  if (d.pore) V = V - (3.141592653589793 * (d.pore_r * d.pore_r)) * d.L[2];
  if (d.n_inner > 0) V = V - hole_area * d.L[2];
  r.V_solid = V;
  const double tf = transient ? t_max_s : 1.0;
  int ns = 0;
  double E[kMaxSources];
  for (int f = 0; f < 6; ++f) {
    if (d.face_type[f] != MCBTE_FACE_ISOTHERMAL) continue;
    const double dT = d.face_T[f] - d.T_eq;
    if (dT == 0.0) continue;
    const int ax = face_axis(f);
    const double A = d.L[(ax + 1) % 3] * d.L[(ax + 2) % 3];
    E[ns] = (((0.25 * A) * sum_Cv) * fabs(dT)) * tf;
    r.src_kind[ns] = 0;
    r.src_face[ns] = f;
    ++ns;
  }
  r.grad_axis = 0;
  r.grad_sign = 0.0;
  r.grad_general = 0;
  int nz = 0;
  for (int k = 0; k < 3; ++k)
    if (d.grad_T[k] != 0.0) {
      ++nz;
      r.grad_axis = k;
      r.grad_sign = d.grad_T[k] > 0.0 ? 1.0 : -1.0;
    }
  if (nz == 1) {
    E[ns] = ((0.5 * V) * fabs(d.grad_T[r.grad_axis])) * sum_Cv;
    r.src_kind[ns] = 1;
    r.src_face[ns] = -1;
    ++ns;
  } else if (nz > 1) {
    // gradient in any direction: |grad T| for the source, Lambertian about
    // +-grad T / |grad T| (Sec. 3.2.3)
    const double gmag = sqrt((d.grad_T[0] * d.grad_T[0] + d.grad_T[1] * d.grad_T[1]) + d.grad_T[2] * d.grad_T[2]);
    r.grad_general = 1;
    r.grad_sign = 1.0;
    double gv[3];
    for (int k = 0; k < 3; ++k) gv[k] = d.grad_T[k] / gmag;
    frame_about(gv, -1.0, r.gframe[0]);
    frame_about(gv, 1.0, r.gframe[1]);
    for (int k = 0; k < 9; ++k) {
      r.gframef[0][k] = (float)r.gframe[0][k];
      r.gframef[1][k] = (float)r.gframe[1][k];
    }
    E[ns] = ((0.5 * V) * gmag) * sum_Cv;
    r.src_kind[ns] = 1;
    r.src_face[ns] = -1;
    ++ns;
  }
  for (int k = 0; k < 3; ++k) r.gauss_c[k] = d.gauss_c[k] * 1e9;
  r.gauss_sigma = d.gauss_sigma * 1e9;
  r.gauss_sign = d.gauss_dT > 0.0 ? 1.0 : -1.0;
  if (d.gauss) {
    const double s = d.gauss_sigma;
    E[ns] = (((C_tot * fabs(d.gauss_dT)) * 15.749609945722419) * ((s * s) * s)) * 0.5;
    r.src_kind[ns] = 2;
    r.src_face[ns] = -1;
    ++ns;
  }
  r.n_src = ns;
  double Et = 0.0;
  for (int k = 0; k < ns; ++k) Et += E[k];
  r.E_tot = Et;
  double acc = 0.0;
  for (int k = 0; k < ns; ++k) {
    acc += E[k];
    r.src_thr[k] = (k + 1 == ns) ? (1ull << 32) : (uint64_t)((acc / Et) * 4294967296.0);
  }
  for (int k = ns; k < kMaxSources; ++k) {
    r.src_thr[k] = 1ull << 32;
    r.src_kind[k] = 0;
    r.src_face[k] = 0;
  }
  // dT/dx defining kappa along the tally axis
  double kg = d.grad_T[ta];
  if (kg == 0.0) {
    const int lo = axis_min_face(ta), hi = axis_max_face(ta);
    if (d.face_type[lo] == MCBTE_FACE_ISOTHERMAL && d.face_type[hi] == MCBTE_FACE_ISOTHERMAL)
      kg = (d.face_T[hi] - d.face_T[lo]) / d.L[ta];
    else
      kg = __longlong_as_double(0x7ff8000000000000ll);
  }
  r.kappa_grad = kg;
  r.n = a.n[gi];
  r.offset = 0;
  r.pid0 = a.pid0[gi];
  r.n_norm = a.n_norm[gi] ? a.n_norm[gi] : a.n[gi];
  geos[gi] = r;
}

}  // namespace

cudaError_t launch_setup(const SetupArgs& a, int n_geoms, const MatView& M, int transient, double t_max_s,
                         int tally_axis, GeoRun* geos, uint64_t* offs, unsigned long long* t0, cudaStream_t s) {
  k_setup<<<1, kMaxGeoms, 0, s>>>(a, n_geoms, M, transient, t_max_s, tally_axis, geos, offs, t0);
  return cudaGetLastError();
}

}  // namespace mcbte
