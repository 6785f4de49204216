// MCBTE oracle: plain, slow, FP64 scalar reference for the deviational
// energy-based Monte Carlo solution of the linearised phonon BTE.
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
// bench's CPU-baseline leg may load this library.  It shares no code,
// header or table generator with the CUDA library.
//
// What it follows (sections / equations of arXiv:2104.03573):
//   - per-bin heat capacity C_i = D_i dE/dT(omega_i) d_omega_i           Eq. BE_derivative, Eq. Nbin
//   - source energies E_i and E_eff = E_tot / N                           Eq. dev_tot, Eq. source_energy
//   - source choice from the cumulative source energy                     Sec. 3.2 (Initialization)
//   - emission: initial condition (bin ~ C|dT|, isotropic)                Eqs. Nbin, cumul_freq, angle_gen
//               isothermal wall (bin ~ C v, Lambertian)                   Eqs. iso_flux, wall_dir
//               control-gradient body source (bin ~ C v, Lambertian)      Eqs. grad_flux, grad_flux_sim
//   - straight flights, exponential relaxation clock x = -Lambda ln R    Eqs. advection_eq, time_to_scat
//   - remaining clock kept across boundary hits                           Sec. 3.3 case (iii)
//   - relaxation: bin redrawn ~ C/tau, isotropic, sign kept               Eq. n_scatt, Sec. 3.5.2
//   - adiabatic wall: specular with probability d, else Lambertian        Eq. specular, Sec. 3.5.3
//   - isothermal wall absorbs; periodic wall translates                   Secs. 3.5.4, 3.5.5 (Eq. periodic_lin_final)
//   - termination: absorbed, t > t_max, or N_scat_max relaxations         Sec. 3.5.6
//   - steady track-length tallies                                         Eqs. steady_estimate, temp_steady, flux_x_steady
//   - N_scat_max convergence curve: X_p of every smaller N_scat_max       Sec. 3.5.6 (the study of N_scat_max)
//   - transient snapshot tallies                                          Eq. sampling, Sec. 3.4
//   - likelihood-ratio scores for d/d(log tau_i) and d/dp (no counterpart in the paper; derived
//     from the exponential law of Eq. time_to_scat and the discrete draws of Eq. n_scatt / Eq. specular)
//   - measure-valued d/dp of the pore specularity (the weak derivative of the specular / diffuse
//     draw of Eq. specular: one pore hit per particle, chosen uniformly, traced again with the
//     other branch)
//
// The random numbers are Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11,
// "Parallel random numbers: as easy as 1, 2, 3"), implemented here from
// that published definition.  Counter = (particle id, batch index, event
// index, sub-block); key = (seed low, seed high).  Which word feeds which
// draw is a fixed contract (listed at each use below); an emission uses
// sub-blocks 0 and 1 exactly as a relaxation does for the bin, direction
// and flight draws.
//
// Internal units: length nm, time ps, velocity nm/ps.
//
// Compile with -O2 -ffp-contract=off (no fused multiply-add), so every
// floating-point operation is the one written.

#include <algorithm>
#include <cmath>
#include <limits>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

const double kHbar = 1.054571817e-34;   // J s
const double kBoltz = 1.380649e-23;     // J / K
const double k2m32 = 2.3283064365386963e-10;   // 2^-32
const double k2m53 = 1.1102230246251565e-16;   // 2^-53

// ---------------------------------------------------------------- Philox4x32-10
void philox4x32_10(const uint32_t ctr[4], uint32_t k0, uint32_t k1, uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Real-valued maps of random words.
inline double oc32(uint32_t w) { return ((double)w + 1.0) * k2m32; }    // (0, 1]
inline double co32(uint32_t w) { return (double)w * k2m32; }            // [0, 1)
inline double mid32(uint32_t w) { return ((double)w + 0.5) * k2m32; }   // (0, 1)
inline double oc53(uint32_t lo, uint32_t hi) {                          // (0, 1], 53 bits
  uint64_t m = ((uint64_t)hi << 21) ^ (uint64_t)(lo >> 11);
  return ((double)m + 1.0) * k2m53;
}

// ---------------------------------------------------------------- elementary functions
// The transcendental functions of the tracer are evaluated by fixed
// published series with a fixed operation order, so that any IEEE-754
// double implementation without fused multiply-add produces the same bits
// (a library log / sin / cos may differ by an ulp between platforms, and
// diffuse reflection off a convex pore amplifies such differences).
//
// ln x (x > 0, normal): x = m 2^e with m in [sqrt(2)/2, sqrt(2)];
// ln x = e ln 2 + 2 atanh(z), z = (m - 1)/(m + 1), |z| < 0.172, atanh by its
// Taylor series z + z^3/3 + ... + z^25/25 (Abramowitz & Stegun 4.1.27 /
// 4.6.22), nested from the highest term.
double series_log(double x) {
  uint64_t b;
  std::memcpy(&b, &x, sizeof(b));
  int e = (int)((b >> 52) & 0x7ffu) - 1023;
  uint64_t mb = (b & 0x000fffffffffffffull) | 0x3ff0000000000000ull;
  double m;
  std::memcpy(&m, &mb, sizeof(m));
  if (m > 1.4142135623730951) {
    m = m * 0.5;
    e = e + 1;
  }
  const double z = (m - 1.0) / (m + 1.0);
  const double z2 = z * z;
  const double p = 0.3333333333333333 + z2 * (0.2 + z2 * (0.14285714285714285 + z2 * (0.1111111111111111 +
                   z2 * (0.09090909090909091 + z2 * (0.07692307692307693 + z2 * (0.06666666666666667 +
                   z2 * (0.058823529411764705 + z2 * (0.05263157894736842 + z2 * (0.047619047619047616 +
                   z2 * (0.043478260869565216 + z2 * 0.04))))))))));
  const double lm = 2.0 * (z + z * (z2 * p));
  return (double)e * 0.6931471805599453 + lm;
}

// cos(2 pi r), sin(2 pi r) for r in [0, 1): octant k = floor(8 r), the
// remainder mapped to theta in [0, pi/4] (reflected on odd octants), Taylor
// series of sin and cos at theta (terms to theta^15 / theta^16), then the
// octant symmetries of the unit circle.
void series_sincos2pi(double r, double* sn, double* cs) {
  const double t = r * 8.0;
  const int k = (int)t;
  double f = t - (double)k;
  if (k & 1) f = 1.0 - f;
  const double th = f * 0.7853981633974483;
  const double t2 = th * th;
  const double S = th * (1.0 + t2 * (-0.16666666666666666 + t2 * (0.008333333333333333 + t2 * (-0.0001984126984126984 +
                   t2 * (2.7557319223985893e-06 + t2 * (-2.505210838544172e-08 + t2 * (1.6059043836821613e-10 +
                   t2 * -7.647163731819816e-13)))))));
  const double Cc = 1.0 + t2 * (-0.5 + t2 * (0.041666666666666664 + t2 * (-0.001388888888888889 +
                    t2 * (2.48015873015873e-05 + t2 * (-2.755731922398589e-07 + t2 * (2.08767569878681e-09 +
                    t2 * (-1.1470745597729725e-11 + t2 * 4.779477332387385e-14)))))));
  switch (k & 7) {
    case 0: *cs = Cc; *sn = S; break;
    case 1: *cs = S; *sn = Cc; break;
    case 2: *cs = -S; *sn = Cc; break;
    case 3: *cs = -Cc; *sn = S; break;
    case 4: *cs = -Cc; *sn = -S; break;
    case 5: *cs = -S; *sn = -Cc; break;
    case 6: *cs = S; *sn = -Cc; break;
    default: *cs = Cc; *sn = -S; break;
  }
}

// The tracer's ln and sincos(2 pi r): the series above by default; the C
// library's std::log, std::sin, std::cos after or_set_libm(1).  The libm mode
// exists to show what the choice changes (a particle whose trajectory turns
// on a last-bit difference: a near-tie between two distances); results are
// compared with the CUDA path in the series mode.
static int g_use_libm = 0;

double ln_(double x) { return g_use_libm ? std::log(x) : series_log(x); }

void sincos2pi_(double r, double* sn, double* cs) {
  if (g_use_libm) {
    const double a = 6.283185307179586 * r;
    *sn = std::sin(a);
    *cs = std::cos(a);
  } else {
    series_sincos2pi(r, sn, cs);
  }
}

// ---------------------------------------------------------------- tables
struct Alias {
  std::vector<double> prob;
  std::vector<uint64_t> thr;
  std::vector<int32_t> alias;
};

// Walker's alias method, built with Vose's two work lists (stacks filled in
// increasing bin order, popped from the back).  The sampled law is the pmf
// w_i / sum(w).
Alias build_alias(const std::vector<double>& w) {
  const int n = (int)w.size();
  double W = 0.0;
  for (int i = 0; i < n; ++i) W += w[i];
  std::vector<double> p(n);
  for (int i = 0; i < n; ++i) p[i] = (w[i] * (double)n) / W;
  std::vector<int> small, large;
  for (int i = 0; i < n; ++i) {
    if (p[i] < 1.0) small.push_back(i); else large.push_back(i);
  }
  Alias a;
  a.prob.assign(n, 1.0);
  a.alias.assign(n, 0);
  for (int i = 0; i < n; ++i) a.alias[i] = i;
  while (!small.empty() && !large.empty()) {
    int l = small.back(); small.pop_back();
    int g = large.back(); large.pop_back();
    a.prob[l] = p[l];
    a.alias[l] = g;
    p[g] = (p[g] + p[l]) - 1.0;
    if (p[g] < 1.0) small.push_back(g); else large.push_back(g);
  }
  // leftovers keep prob 1 and alias = self
  a.thr.resize(n);
  for (int i = 0; i < n; ++i) {
    double q = a.prob[i];
    a.thr[i] = (q >= 1.0) ? UINT64_MAX : (uint64_t)(q * 18446744073709551616.0);
  }
  return a;
}

// Draw a bin: column from one word (exact integer multiply-high), then keep
// the column iff the 64-bit threshold word is below its threshold.
inline int alias_draw(const Alias& a, int n, uint32_t wcol, uint32_t thr_lo, uint32_t thr_hi) {
  int col = (int)(((uint64_t)wcol * (uint64_t)n) >> 32);
  uint64_t r = ((uint64_t)thr_hi << 32) | (uint64_t)thr_lo;
  return (r < a.thr[col]) ? col : a.alias[col];
}

// dE/dT of the Bose-Einstein mode energy hbar*omega*f_eq at temperature T:
// k_B (x/2)^2 / sinh^2(x/2), x = hbar omega / (k_B T)   (Eq. BE_derivative, read as
// the derivative of hbar*omega/(exp(x)-1)).
double dEdT(double omega, double T) {
  double x = (kHbar * omega) / (kBoltz * T);
  double h = 0.5 * x;
  double s = std::sinh(h);
  return kBoltz * (h * h) / (s * s);
}

}  // namespace

extern "C" {

typedef struct {
  // material (SI)
  int n_bins;
  const double* omega;
  const double* v;
  const double* tau;
  const double* C;        // format 2, or NULL
  const double* D;        // format 1, or NULL
  const double* domega;   // format 1
  double T_lin;
  const double* tau_imp;  // optional two-phonon (impurity) relaxation times, or NULL (Sec. 3.3, Sec. 4.1)
  const double* spec_bin; // optional per-bin specularity d(omega) in [0, 1] (Sec. 3.5.3), or NULL
  // geometry (SI)
  double L[3];
  int face_type[6];       // 0 isothermal, 1 adiabatic, 2 periodic
  double face_T[6];
  double face_p[6];
  double T_eq;
  double grad_T[3];
  int pore;
  double pore_c[2];
  double pore_r;
  double pore_p;
  int gauss;
  double gauss_c[3];
  double gauss_sigma;
  double gauss_dT;
  // internal boundaries (Sec. 4.2): segments in the x-y plane through the
  // thickness, normal pointing into the solid, specularity (< 0: per bin)
  int n_inner;
  double inner[16][4];    // x1, y1, x2, y2 (m)
  double inner_n[16][2];
  double inner_p[16];
  // run
  uint64_t seed;
  uint32_t batch_index;
  int transient;
  uint64_t n_particles;   // N that defines E_eff
  uint64_t pid_begin;
  uint64_t pid_end;
  int n_scat_max;         // 0 = unlimited
  uint64_t max_events;
  int n_cells;
  int cell_axis;
  int tally_axis;
  double t_max;           // s
  int n_times;
  const double* t_meas;   // s
  int grid[3];
  // detector regions (Sec. 4.5, Measure_region): axis-aligned cuboids, each
  // split into nx x ny x nz detectors; none: the whole box with `grid`
  int n_regions;
  const double* regions;      // [n_regions][6] xmin, xmax, ymin, ymax, zmin, zmax (m)
  const int* region_grid;     // [n_regions][3]
  int time_average;           // 0: snapshots at t_m (Eq. sampling); 1: averages over [t_{m-1}, t_m)
  int det_per_bin;            // steady regions: one T, q per detector and frequency bin (Sec. 4.5)
  int nscat_curve;            // 1: X sums for every N_scat_max' = 1..n_scat_max (steady)
  int want_grad;
  int dp_mvd;                 // 1: d kappa / d p_pore by the measure-valued estimator
  int n_dirs;
  const double* dirs;     // [n_dirs][n_bins]
  int n_threads;
} or_params;

enum {
  OR_SUMX = 0, OR_SUMX2, OR_EVENTS, OR_TRUNC, OR_ABSORBED, OR_SIGNED_ABS, OR_SIGNED_EMIT,
  OR_RSUM, OR_GP, OR_GP2, OR_ETOT, OR_CTOT, OR_VSOLID, OR_MAXEV, OR_NSCAL = 16
};

typedef struct {
  double* T_sum;        // [n_cells]            sum s * l_c / v           (ps)
  double* Q_sum;        // [n_cells][3]         sum s * l_c * u_b         (nm)
  double* qbin_sum;     // [n_bins]             sum s * l * u_tally       (nm)
  double* snap;         // [n_times][cells][4]  sum s, sum s v u_{x,y,z}  (-, nm/ps)
  uint32_t* events_pp;  // [pid_end - pid_begin]
  double* X_pp;         // [pid_end - pid_begin]  per-particle sum s l u_tally (nm)
  double* G;            // [n_bins]  sum over particles of the sparse LR part
  double* dir_sum;      // [n_dirs]
  double* dir_sum2;     // [n_dirs]
  double* curve;        // [n_scat_max][2]  sum X_p(k), sum X_p(k)^2 for N_scat_max = k (nscat_curve)
  double scal[16];
} or_out;

}  // extern "C"

namespace {

uint64_t spec_threshold(double p) {
  if (p <= 0.0) return 0;
  if (p >= 1.0) return (uint64_t)1 << 32;
  return (uint64_t)(p * 4294967296.0);
}

struct Tables {
  int n = 0;
  std::vector<double> C, v_nm, lam_nm, inv_v, pi_relax;
  bool imp = false;              // a two-phonon clock is present
  std::vector<double> lam2_nm;   // v tau_imp (nm); +inf for bins without impurity scattering
  std::vector<uint64_t> spec_thr_bin;  // per-bin specular thresholds (empty without d(omega))
  double C_tot = 0, sum_Cv = 0, sum_Ct = 0;
  Alias emit, init, relax;
};

int build_tables(const or_params* P, Tables& t) {
  const int n = P->n_bins;
  if (n < 1) return 1;
  t.n = n;
  t.C.resize(n);
  for (int i = 0; i < n; ++i) {
    if (P->C) t.C[i] = P->C[i];
    else t.C[i] = (P->D[i] * dEdT(P->omega[i], P->T_lin)) * P->domega[i];
  }
  std::vector<double> w_emit(n), w_init(n), w_relax(n);
  for (int i = 0; i < n; ++i) {
    w_emit[i] = t.C[i] * P->v[i];
    w_init[i] = t.C[i];
    w_relax[i] = t.C[i] / P->tau[i];
  }
  t.C_tot = 0; t.sum_Cv = 0; t.sum_Ct = 0;
  for (int i = 0; i < n; ++i) {
    t.C_tot += t.C[i];
    t.sum_Cv += w_emit[i];
    t.sum_Ct += w_relax[i];
  }
  t.emit = build_alias(w_emit);
  t.init = build_alias(w_init);
  t.relax = build_alias(w_relax);
  t.v_nm.resize(n); t.lam_nm.resize(n); t.inv_v.resize(n); t.pi_relax.resize(n);
  for (int i = 0; i < n; ++i) {
    t.v_nm[i] = P->v[i] * 1e-3;
    double tau_ps = P->tau[i] * 1e12;
    t.lam_nm[i] = t.v_nm[i] * tau_ps;
    t.inv_v[i] = 1.0 / t.v_nm[i];
    t.pi_relax[i] = w_relax[i] / t.sum_Ct;
  }
  if (P->spec_bin) {
    t.spec_thr_bin.resize(n);
    for (int i = 0; i < n; ++i) t.spec_thr_bin[i] = spec_threshold(P->spec_bin[i]);
  }
  t.imp = P->tau_imp != nullptr;
  t.lam2_nm.assign(n, std::numeric_limits<double>::infinity());
  if (t.imp)
    for (int i = 0; i < n; ++i)
      if (std::isfinite(P->tau_imp[i])) t.lam2_nm[i] = t.v_nm[i] * (P->tau_imp[i] * 1e12);
  return 0;
}

const int kFaceAxis[6] = {1, 0, 1, 0, 2, 2};
const int kFaceIsMax[6] = {0, 1, 1, 0, 0, 1};
const int kAxisMinFace[3] = {3, 0, 4};
const int kAxisMaxFace[3] = {1, 2, 5};

struct Geo {
  double L[3];
  int type[6];
  double Tb[6];
  uint64_t pthr[6];
  bool pore;
  double cx, cy, r, r2, p_pore;
  uint64_t pthr_pore;
  bool fbin[6];             // outer face uses the per-bin specularity
  int n_inner;
  double sx1[16], sy1[16], sx2[16], sy2[16], snx[16], sny[16];   // nm
  uint64_t sthr[16];
  bool sbin[16];
  double V_solid_m3;
};

// Inside a hole bounded by the internal segments: even-odd count of the
// segments crossed by the ray from (x, y) towards +x.
inline bool in_hole(const Geo& g, double x, double y) {
  bool c = false;
  for (int k = 0; k < g.n_inner; ++k) {
    const double y1 = g.sy1[k], y2 = g.sy2[k];
    if ((y1 > y) != (y2 > y)) {
      const double xc = g.sx1[k] + ((y - y1) * (g.sx2[k] - g.sx1[k])) / (y2 - y1);
      if (x < xc) c = !c;
    }
  }
  return c;
}


struct Source {
  int kind;   // 0 face, 1 body, 2 gauss
  int face;
  double E;
};

struct Setup {
  Geo g;
  std::vector<Source> src;
  std::vector<uint64_t> src_thr;
  double E_tot = 0;
  int grad_axis = -1;
  double grad_sign = 0;
  bool grad_general = false;   // more than one gradient component: Lambertian about gvec
  double gvec[3] = {0, 0, 0};  // grad T / |grad T|
  double t_max_ps = 0;
  std::vector<double> t_meas_ps;
  double gauss_c[3], gauss_sigma;
  double dpi_dirs[64];
  struct Region {
    double lo[3], hi[3];   // nm
    int n[3];
    size_t off;            // first detector of the region
    bool whole;            // the whole box (every position inside, clamped to the grid)
    bool hi_closed[3];     // the upper face lies on (or beyond) the box's upper face
  };
  std::vector<Region> regs;
  size_t n_det = 0;
};

int setup(const or_params* P, const Tables& t, Setup& S) {
  Geo& g = S.g;
  for (int a = 0; a < 3; ++a) g.L[a] = P->L[a] * 1e9;
  for (int f = 0; f < 6; ++f) {
    g.type[f] = P->face_type[f];
    g.Tb[f] = P->face_T[f];
    g.fbin[f] = P->face_p[f] < 0.0;
    g.pthr[f] = spec_threshold(P->face_p[f]);
  }
  g.n_inner = P->n_inner;
  double hole_area = 0.0;   // m^2: segments oriented with the solid on their right
  for (int k = 0; k < g.n_inner; ++k) {
    double x1 = P->inner[k][0], y1 = P->inner[k][1], x2 = P->inner[k][2], y2 = P->inner[k][3];
    const double nx = P->inner_n[k][0], ny = P->inner_n[k][1];
    if ((y2 - y1) * nx - (x2 - x1) * ny < 0.0) {
      std::swap(x1, x2);
      std::swap(y1, y2);
    }
    hole_area += 0.5 * (x1 * y2 - x2 * y1);
    g.sx1[k] = x1 * 1e9; g.sy1[k] = y1 * 1e9; g.sx2[k] = x2 * 1e9; g.sy2[k] = y2 * 1e9;
    g.snx[k] = nx; g.sny[k] = ny;
    g.sbin[k] = P->inner_p[k] < 0.0;
    g.sthr[k] = spec_threshold(P->inner_p[k]);
  }
  if (P->spec_bin == nullptr) {   // a per-bin specularity needs the material's d(omega)
    for (int f = 0; f < 6; ++f) if (g.fbin[f] && g.type[f] == 1) return 5;
    for (int k = 0; k < g.n_inner; ++k) if (g.sbin[k]) return 5;
  }
  g.pore = P->pore != 0;
  g.cx = P->pore_c[0] * 1e9;
  g.cy = P->pore_c[1] * 1e9;
  g.r = P->pore_r * 1e9;
  g.r2 = g.r * g.r;
  g.p_pore = P->pore_p;
  g.pthr_pore = spec_threshold(P->pore_p);
  double V = P->L[0] * P->L[1] * P->L[2];
  if (g.pore) V = V - (3.141592653589793 * (P->pore_r * P->pore_r)) * P->L[2];
  if (g.n_inner > 0) V = V - hole_area * P->L[2];
  g.V_solid_m3 = V;
  // sources, in order: isothermal faces by ID, body, initial condition
  const double time_factor = P->transient ? P->t_max : 1.0;
  for (int f = 0; f < 6; ++f) {
    if (g.type[f] != 0) continue;
    double dT = P->face_T[f] - P->T_eq;
    if (dT == 0.0) continue;
    int a = kFaceAxis[f];
    double A = P->L[(a + 1) % 3] * P->L[(a + 2) % 3];
    double E = ((0.25 * A) * t.sum_Cv) * std::fabs(dT);
    S.src.push_back({0, f, E * time_factor});
  }
  int nz = 0;
  for (int a = 0; a < 3; ++a) if (P->grad_T[a] != 0.0) { nz++; S.grad_axis = a; }
  if (nz == 1) {
    if (P->transient) return 2;
    double gmag = std::fabs(P->grad_T[S.grad_axis]);
    S.grad_sign = P->grad_T[S.grad_axis] > 0 ? 1.0 : -1.0;
    double E = ((0.5 * V) * gmag) * t.sum_Cv;
    S.src.push_back({1, -1, E});
  } else if (nz > 1) {
    // a control gradient in any direction: the same body source with |grad T|,
    // particles Lambertian about -/+ grad T / |grad T| (Sec. 3.2.3)
    if (P->transient) return 2;
    double gmag = std::sqrt((P->grad_T[0] * P->grad_T[0] + P->grad_T[1] * P->grad_T[1]) + P->grad_T[2] * P->grad_T[2]);
    S.grad_general = true;
    S.grad_sign = 1.0;
    for (int a = 0; a < 3; ++a) S.gvec[a] = P->grad_T[a] / gmag;
    double E = ((0.5 * V) * gmag) * t.sum_Cv;
    S.src.push_back({1, -1, E});
  }
  if (P->gauss) {
    double s = P->gauss_sigma;
    double E = (((t.C_tot * std::fabs(P->gauss_dT)) * 15.749609945722419) * ((s * s) * s)) * 0.5;
    S.src.push_back({2, -1, E});
    for (int a = 0; a < 3; ++a) S.gauss_c[a] = P->gauss_c[a] * 1e9;
    S.gauss_sigma = s * 1e9;
  }
  if (S.src.empty()) return 3;
  double run = 0;
  for (auto& s : S.src) run += s.E;
  S.E_tot = run;
  double acc = 0;
  for (size_t k = 0; k < S.src.size(); ++k) {
    acc += S.src[k].E;
    if (k + 1 == S.src.size()) S.src_thr.push_back((uint64_t)1 << 32);
    else S.src_thr.push_back((uint64_t)((acc / S.E_tot) * 4294967296.0));
  }
  S.t_max_ps = P->t_max * 1e12;
  for (int m = 0; m < P->n_times; ++m) S.t_meas_ps.push_back(P->t_meas[m] * 1e12);
  if (P->transient || P->n_regions > 0) {
    if (P->n_regions == 0) {
      Setup::Region r;
      for (int a = 0; a < 3; ++a) { r.lo[a] = 0.0; r.hi[a] = g.L[a]; r.n[a] = P->grid[a]; r.hi_closed[a] = true; }
      r.off = 0;
      r.whole = true;
      S.regs.push_back(r);
      S.n_det = (size_t)P->grid[0] * P->grid[1] * P->grid[2];
    } else {
      size_t off = 0;
      for (int k = 0; k < P->n_regions; ++k) {
        Setup::Region r;
        for (int a = 0; a < 3; ++a) {
          r.lo[a] = P->regions[6 * k + 2 * a] * 1e9;
          r.hi[a] = P->regions[6 * k + 2 * a + 1] * 1e9;
          r.n[a] = P->region_grid[3 * k + a];
          r.hi_closed[a] = r.hi[a] >= g.L[a];
          if (!(r.hi[a] > r.lo[a]) || r.n[a] < 1) return 6;
        }
        r.off = off;
        r.whole = false;
        off += (size_t)r.n[0] * r.n[1] * r.n[2];
        S.regs.push_back(r);
      }
      S.n_det = off;
    }
  }
  if (P->want_grad) {
    if (P->n_dirs > 64) return 4;
    for (int k = 0; k < P->n_dirs; ++k) {
      double acc2 = 0;
      for (int i = 0; i < t.n; ++i) acc2 += P->dirs[(size_t)k * t.n + i] * t.pi_relax[i];
      S.dpi_dirs[k] = acc2;
    }
  }
  return 0;
}

// First boundary along the ray: the faces met in the direction of travel and
// the pore cylinder.  Ties go to the lowest paper boundary ID (faces 1..6,
// pore 7).  Returns the distance (nm) and the face index (0..5, or 6).
inline void first_hit(const Geo& g, const double x[3], const double u[3], double* dist, int* face) {
  double best = INFINITY;
  int bf = -1;
  for (int a = 0; a < 3; ++a) {
    double d;
    int f;
    if (u[a] > 0.0) { d = (g.L[a] - x[a]) / u[a]; f = kAxisMaxFace[a]; }
    else if (u[a] < 0.0) { d = (0.0 - x[a]) / u[a]; f = kAxisMinFace[a]; }
    else continue;
    if (d < 0.0) d = 0.0;
    if (d < best || (d == best && f < bf)) { best = d; bf = f; }
  }
  if (g.pore) {
    double dx = x[0] - g.cx, dy = x[1] - g.cy;
    double a = u[0] * u[0] + u[1] * u[1];
    double b = dx * u[0] + dy * u[1];
    if (a > 0.0 && b < 0.0) {
      double c = (dx * dx + dy * dy) - g.r2;
      double disc = b * b - a * c;
      if (disc >= 0.0) {
        double d = c / (std::sqrt(disc) - b);
        if (d < 0.0) d = 0.0;
        if (d < best) { best = d; bf = 6; }
      }
    }
  }
  // internal walls (IDs 8, 9, ...): only approached from the solid side
  for (int k = 0; k < g.n_inner; ++k) {
    const double un = u[0] * g.snx[k] + u[1] * g.sny[k];
    if (!(un < 0.0)) continue;
    // behind the wall's line (beyond the hole): not this wall; on it within
    // rounding (after a hit the particle is projected onto the line): d = 0
    const double dn = (x[0] - g.sx1[k]) * g.snx[k] + (x[1] - g.sy1[k]) * g.sny[k];
    if (dn < -1e-9) continue;
    double d = dn / (-un);
    if (d < 0.0) d = 0.0;
    const double tx = g.sx2[k] - g.sx1[k], ty = g.sy2[k] - g.sy1[k];
    const double hs = ((x[0] + d * u[0]) - g.sx1[k]) * tx + ((x[1] + d * u[1]) - g.sy1[k]) * ty;
    if (hs < 0.0 || hs > tx * tx + ty * ty) continue;
    if (d < best) { best = d; bf = 7 + k; }
  }
  *dist = best;
  *face = bf;
}

// Direction with polar cosine mu about +/- axis a; the other two axes, in
// cyclic order a+1, a+2, take s cos(phi), s sin(phi).
inline void dir_about_axis(double u[3], int a, double sgn, double mu, uint32_t wphi) {
  double s = std::sqrt(std::max(0.0, 1.0 - mu * mu));
  double sn, cs;
  sincos2pi_(co32(wphi), &sn, &cs);
  u[a] = sgn * mu;
  u[(a + 1) % 3] = s * cs;
  u[(a + 2) % 3] = s * sn;
}

// Direction with polar cosine mu about sgn * gv (a unit vector): the
// orthonormal frame {b1, b2, n} of n = sgn gv by the branchless construction
// of Duff et al., "Building an Orthonormal Basis, Revisited" (JCGT 6(1),
// 2017); u = mu n + s cos(phi) b1 + s sin(phi) b2, phi = 2 pi co(wphi).
inline void dir_about_vector(double u[3], const double gv[3], double sgn, double mu, uint32_t wphi) {
  const double n[3] = {sgn * gv[0], sgn * gv[1], sgn * gv[2]};
  const double sg = n[2] >= 0.0 ? 1.0 : -1.0;
  const double a = -1.0 / (sg + n[2]);
  const double b = (n[0] * n[1]) * a;
  const double b1[3] = {1.0 + ((sg * n[0]) * n[0]) * a, sg * b, -sg * n[0]};
  const double b2[3] = {b, sg + (n[1] * n[1]) * a, -n[1]};
  double s = std::sqrt(std::max(0.0, 1.0 - mu * mu));
  double sn, cs;
  sincos2pi_(co32(wphi), &sn, &cs);
  for (int k = 0; k < 3; ++k) u[k] = (mu * n[k] + (s * cs) * b1[k]) + (s * sn) * b2[k];
}

// Time the straight path x(tau) = x0 + w (tau - t0) spends in each detector
// of region r between times ta < tb (w in nm/ps): clip [ta, tb) to the
// region's box, then walk the detector grid from cell to cell in time order
// (cell-crossing times from the grid planes; ties advance every axis that
// crosses).  add(detector index within the region, duration).
template <class Add>
void region_track(const Setup::Region& r, const double x0[3], const double w[3], double t0, double ta, double tb,
                  Add add) {
  double t_in = ta, t_out = tb;
  for (int a = 0; a < 3; ++a) {
    const double p = x0[a] + w[a] * (ta - t0);
    if (w[a] == 0.0) {
      if (!(p >= r.lo[a] && (p < r.hi[a] || (r.hi_closed[a] && p <= r.hi[a])))) return;
      continue;
    }
    double c0 = t0 + (r.lo[a] - x0[a]) / w[a];
    double c1 = t0 + (r.hi[a] - x0[a]) / w[a];
    if (c0 > c1) std::swap(c0, c1);
    t_in = std::max(t_in, c0);
    t_out = std::min(t_out, c1);
  }
  if (!(t_in < t_out)) return;
  int i3[3];
  double h[3];
  for (int a = 0; a < 3; ++a) {
    h[a] = (r.hi[a] - r.lo[a]) / (double)r.n[a];
    const double p = x0[a] + w[a] * (t_in - t0);
    int ia = (int)std::floor((p - r.lo[a]) / h[a]);
    if (w[a] < 0.0 && ia * h[a] + r.lo[a] == p) ia = ia - 1;   // on a plane, moving down: the cell below
    i3[a] = std::min(std::max(ia, 0), r.n[a] - 1);
  }
  double tau = t_in;
  const int max_steps = r.n[0] + r.n[1] + r.n[2] + 3;
  for (int step = 0; step < max_steps && tau < t_out; ++step) {
    double tn = t_out;
    double tc[3];
    for (int a = 0; a < 3; ++a) {
      tc[a] = INFINITY;
      if (w[a] > 0.0) tc[a] = t0 + ((r.lo[a] + (i3[a] + 1) * h[a]) - x0[a]) / w[a];
      else if (w[a] < 0.0) tc[a] = t0 + ((r.lo[a] + i3[a] * h[a]) - x0[a]) / w[a];
      if (tc[a] < tn) tn = tc[a];
    }
    if (tn < tau) tn = tau;
    add(((size_t)i3[2] * r.n[1] + i3[1]) * r.n[0] + i3[0], tn - tau);
    tau = tn;
    if (!(tau < t_out)) break;
    bool out_of = false;
    for (int a = 0; a < 3; ++a)
      if (tc[a] <= tn) {
        i3[a] += w[a] > 0.0 ? 1 : -1;
        if (i3[a] < 0 || i3[a] >= r.n[a]) out_of = true;
      }
    if (out_of) break;
  }
}

struct Partial {
  std::vector<double> T, Q, qbin, snap, G, dsum, dsum2, curve;
  double scal[OR_NSCAL] = {0};
};

struct Period { int bin; double A, B; };

// The pore hit a particle's phantom trace flips: `sel` of its K pore hits,
// and whether the nominal trajectory reflected specularly there.
struct MvdPick { uint32_t K = 0, sel = 0; bool spec = false; };

void trace_range(const or_params* P, const Tables& t, const Setup& S, uint64_t p0, uint64_t p1,
                 Partial& res, or_out* O) {
  const Geo& g = S.g;
  const int n = t.n;
  const uint32_t k0 = (uint32_t)P->seed, k1 = (uint32_t)(P->seed >> 32);
  const int ta = P->tally_axis;
  const bool cells = P->n_cells > 0 && !P->transient;
  const double h_cell = cells ? g.L[P->cell_axis] / (double)P->n_cells : 0.0;
  std::vector<Period> periods;
  std::vector<double> x_relax;   // X at each relaxation event (N_scat_max curve)
  // tallies of phantom traces (discarded)
  Partial scratch;
  if (P->dp_mvd) scratch = res;
  // One trajectory of particle pid.  flip = 0: the nominal trace, with all
  // tallies; `pick` receives the reservoir choice of a pore hit.  flip = j > 0:
  // the phantom trace of the measure-valued derivative: the same random words,
  // but the j-th pore hit takes the other branch; only its X is used.
  auto trace_one = [&](uint64_t pid, uint32_t flip, MvdPick* pick) -> double {
    Partial& out = flip ? scratch : res;
    uint32_t n_pore = 0;
    uint32_t ctr[4] = {(uint32_t)pid, P->batch_index, 0u, 0u};
    uint32_t w[4], w1[4], w2[4], w3[4];
    // ---- emission (event 0): sub-blocks 0 and 1 carry the bin, direction
    // and flight words exactly as a relaxation event does; sub 1 word 3
    // picks the source; sub 2 carries the position and the sign / emission time.
    ctr[3] = 0; philox4x32_10(ctr, k0, k1, w);
    ctr[3] = 1; philox4x32_10(ctr, k0, k1, w1);
    ctr[3] = 2; philox4x32_10(ctr, k0, k1, w2);
    int k = 0;
    while ((uint64_t)w1[3] >= S.src_thr[k]) ++k;
    const Source& src = S.src[k];
    double x[3], u[3];
    int bin;
    double s;
    double t_now = 0.0;
    if (src.kind == 0) {
      int f = src.face, a = kFaceAxis[f];
      bin = alias_draw(t.emit, n, w[0], w[1], w1[0]);
      s = (g.Tb[f] > P->T_eq) ? 1.0 : -1.0;
      double mu = std::sqrt(oc32(w[2]));
      dir_about_axis(u, a, kFaceIsMax[f] ? -1.0 : 1.0, mu, w[3]);
      if (P->transient) t_now = co32(w2[3]) * S.t_max_ps;
      x[a] = kFaceIsMax[f] ? g.L[a] : 0.0;
      x[(a + 1) % 3] = mid32(w2[0]) * g.L[(a + 1) % 3];
      x[(a + 2) % 3] = mid32(w2[1]) * g.L[(a + 2) % 3];
    } else if (src.kind == 1) {
      bin = alias_draw(t.emit, n, w[0], w[1], w1[0]);
      s = (w2[3] < 0x80000000u) ? 1.0 : -1.0;
      // positive particles travel down the control gradient, negative ones up it
      double dsgn = (s > 0.0) ? -S.grad_sign : S.grad_sign;
      double mu = std::sqrt(oc32(w[2]));
      if (S.grad_general) dir_about_vector(u, S.gvec, dsgn, mu, w[3]);
      else dir_about_axis(u, S.grad_axis, dsgn, mu, w[3]);
      // uniform position in the solid: attempt 0 uses sub 2, attempt j sub 2 + j
      for (int j = 0;; ++j) {
        if (j > 0) {
          ctr[3] = 2u + (uint32_t)j; philox4x32_10(ctr, k0, k1, w3);
        } else {
          for (int q = 0; q < 4; ++q) w3[q] = w2[q];
        }
        x[0] = mid32(w3[0]) * g.L[0];
        x[1] = mid32(w3[1]) * g.L[1];
        x[2] = mid32(w3[2]) * g.L[2];
        bool inside = false;
        if (g.pore) {
          double dx = x[0] - g.cx, dy = x[1] - g.cy;
          inside = dx * dx + dy * dy < g.r2;
        }
        if (!inside && g.n_inner > 0) inside = in_hole(g, x[0], x[1]);
        if (!inside) break;
        if (j + 1 >= 64) break;   // unreachable for porosities the API accepts
      }
    } else {
      bin = alias_draw(t.init, n, w[0], w[1], w1[0]);
      s = (P->gauss_dT > 0.0) ? 1.0 : -1.0;
      double mu = 1.0 - 2.0 * oc32(w[2]);
      dir_about_axis(u, 2, 1.0, mu, w[3]);
      ctr[3] = 3; philox4x32_10(ctr, k0, k1, w3);
      double m1 = std::sqrt(-2.0 * ln_(oc32(w3[0])));
      double m2 = std::sqrt(-2.0 * ln_(oc32(w3[2])));
      double s1, c1, s2, c2;
      sincos2pi_(co32(w3[1]), &s1, &c1);
      sincos2pi_(co32(w3[3]), &s2, &c2);
      double nrm[3] = {m1 * c1, m1 * s1, m2 * c2};
      for (int a = 0; a < 3; ++a) {
        double c = S.gauss_c[a] + S.gauss_sigma * nrm[a];
        if (c < 0.0) c = -c;
        if (c > g.L[a]) c = 2.0 * g.L[a] - c;
        if (c < 0.0) c = 0.0;
        if (c > g.L[a]) c = g.L[a];
        x[a] = c;
      }
    }
    double d_rel = t.lam_nm[bin] * (-ln_(oc53(w1[1], w1[2])));
    // two-phonon clock (Sec. 3.3): its own exponential distance, drawn from
    // sub-block 256 of the event that (re)starts it
    auto draw_d2 = [&](uint32_t ev) -> double {
      if (!t.imp || !std::isfinite(t.lam2_nm[bin])) return std::numeric_limits<double>::infinity();
      uint32_t c4[4] = {(uint32_t)pid, P->batch_index, ev, 256u};
      uint32_t w4[4];
      philox4x32_10(c4, k0, k1, w4);
      return t.lam2_nm[bin] * (-ln_(oc53(w4[0], w4[1])));
    };
    double d2 = draw_d2(0);
    out.scal[OR_SIGNED_EMIT] += s;
    uint32_t e = 0;
    int n_relax = 0;
    double X = 0.0;
    bool truncated = false;
    // adjoint bookkeeping
    periods.clear();
    if (P->want_grad) periods.push_back({bin, 0.0, 0.0});
    int n_res = 0;
    double sum_x_res = 0.0;
    double PA = 0.0, PB = 0.0;
    x_relax.clear();
    size_t mi = 0;
    if (P->transient) {
      if (P->time_average) { while (mi < S.t_meas_ps.size() && S.t_meas_ps[mi] <= t_now) ++mi; }
      else { while (mi < S.t_meas_ps.size() && S.t_meas_ps[mi] < t_now) ++mi; }
    }
    for (;;) {
      if ((uint64_t)e + 1 >= P->max_events) { truncated = true; break; }
      double db;
      int face;
      first_hit(g, x, u, &db, &face);
      const double v = t.v_nm[bin];
      bool final_seg = false;
      bool relax;           // three-phonon relaxation ends the flight
      bool relax2 = false;  // two-phonon (impurity) scattering ends the flight
      double seg;
      // the flight ends at the nearest of: t_max (transient), the three-phonon
      // clock, the two-phonon clock, the boundary; the boundary wins ties, and
      // the three-phonon clock wins a tie with the two-phonon one
      if (P->transient && (S.t_max_ps - t_now) * v <= d_rel && (S.t_max_ps - t_now) * v <= db &&
          (S.t_max_ps - t_now) * v <= d2) {
        final_seg = true; seg = (S.t_max_ps - t_now) * v; relax = false;
      } else if (d_rel < db && d_rel <= d2) {
        seg = d_rel; relax = true;
      } else if (d2 < db) {
        seg = d2; relax = false; relax2 = true;
      } else {
        seg = db; relax = false;
      }
      // ---- tallies of this flight
      if (P->transient) {
        // the flight ended by t_max ends at t_max exactly (its length was
        // derived from t_max; dividing it by v again could land an ulp short)
        double t_end = final_seg ? S.t_max_ps : t_now + seg / v;
        if (P->time_average) {
          // time-bin averages: the flight's time in each detector during each
          // bin [t_{m-1}, t_m) it overlaps, over the bin's length
          const double w3[3] = {v * u[0], v * u[1], v * u[2]};
          while (mi < S.t_meas_ps.size()) {
            const double b0 = mi == 0 ? 0.0 : S.t_meas_ps[mi - 1];
            const double b1 = S.t_meas_ps[mi];
            if (!(b0 < t_end)) break;
            const double ta = std::max(t_now, b0), tb = std::min(t_end, b1);
            if (ta < tb) {
              const double wb = 1.0 / (b1 - b0);
              for (const Setup::Region& r : S.regs)
                region_track(r, x, w3, t_now, ta, tb, [&](size_t det, double dur) {
                  const size_t c = ((size_t)mi * S.n_det + r.off + det) * 4;
                  const double f = (s * dur) * wb;
                  out.snap[c + 0] += f;
                  out.snap[c + 1] += (f * v) * u[0];
                  out.snap[c + 2] += (f * v) * u[1];
                  out.snap[c + 3] += (f * v) * u[2];
                });
            }
            if (b1 <= t_end) ++mi;
            else break;
          }
          t_now = t_end;
        } else
        while (mi < S.t_meas_ps.size() &&
               (S.t_meas_ps[mi] < t_end || (final_seg && S.t_meas_ps[mi] <= t_end))) {
          double dist = v * (S.t_meas_ps[mi] - t_now);
          double pm[3];
          for (int a = 0; a < 3; ++a) pm[a] = x[a] + dist * u[a];
          // every detector region containing the position: half-open cuboids
          // [lo, hi), closed on the box's upper faces, so that regions tiling
          // the box partition it
          for (const Setup::Region& r : S.regs) {
            if (!r.whole) {
              bool in = true;
              for (int a = 0; a < 3; ++a)
                in = in && pm[a] >= r.lo[a] && (pm[a] < r.hi[a] || (pm[a] == r.hi[a] && pm[a] >= g.L[a]));
              if (!in) continue;
            }
            int i3[3];
            for (int a = 0; a < 3; ++a) {
              int ia = (int)std::floor((pm[a] - r.lo[a]) / ((r.hi[a] - r.lo[a]) / (double)r.n[a]));
              i3[a] = std::min(std::max(ia, 0), r.n[a] - 1);
            }
            size_t c = ((size_t)mi * S.n_det + r.off + ((size_t)i3[2] * r.n[1] + i3[1]) * r.n[0] + i3[0]) * 4;
            out.snap[c + 0] += s;
            out.snap[c + 1] += (s * v) * u[0];
            out.snap[c + 2] += (s * v) * u[1];
            out.snap[c + 3] += (s * v) * u[2];
          }
          ++mi;
        }
        t_now = t_end;
      } else {
        double contrib = (s * seg) * u[ta];
        double Xb = X;
        X += contrib;
        if (P->n_bins > 0 && O->qbin_sum) out.qbin[bin] += contrib;
        if (cells) {
          int ca = P->cell_axis;
          double z0 = x[ca];
          double z1 = z0 + seg * u[ca];
          double inv_v = t.inv_v[bin];
          if (u[ca] == 0.0) {
            int c = (int)std::floor(z0 / h_cell);
            c = std::min(std::max(c, 0), P->n_cells - 1);
            out.T[c] += (s * seg) * inv_v;
            for (int b = 0; b < 3; ++b) out.Q[(size_t)c * 3 + b] += (s * seg) * u[b];
          } else {
            double zlo = std::min(z0, z1), zhi = std::max(z0, z1);
            int clo = std::min(std::max((int)std::floor(zlo / h_cell), 0), P->n_cells - 1);
            int chi = std::min(std::max((int)std::floor(zhi / h_cell), 0), P->n_cells - 1);
            double au = std::fabs(u[ca]);
            for (int c = clo; c <= chi; ++c) {
              double lo = std::max(zlo, c * h_cell);
              double hi = std::min(zhi, (c + 1) * h_cell);
              if (c == P->n_cells - 1) hi = zhi;
              if (c == 0) lo = zlo;
              double ov = hi - lo;
              if (ov <= 0.0) continue;
              double l = ov / au;
              out.T[c] += (s * l) * inv_v;
              for (int b = 0; b < 3; ++b) out.Q[(size_t)c * 3 + b] += (s * l) * u[b];
            }
          }
        }
        if (P->n_regions > 0) {
          // steady detector regions (Sec. 4.5): track length in each detector,
          // s dt for T (ps) and s v dt u for q (nm), dt the time spent there
          const double w3[3] = {v * u[0], v * u[1], v * u[2]};
          const double dt = seg / v;
          for (const Setup::Region& r : S.regs)
            region_track(r, x, w3, 0.0, 0.0, dt, [&](size_t det, double dur) {
              // per detector, or per detector and the particle's bin
              const size_t c = P->det_per_bin ? ((r.off + det) * (size_t)n + (size_t)bin) * 4 : (r.off + det) * 4;
              out.snap[c + 0] += s * dur;
              out.snap[c + 1] += ((s * v) * dur) * u[0];
              out.snap[c + 2] += ((s * v) * dur) * u[1];
              out.snap[c + 3] += ((s * v) * dur) * u[2];
            });
        }
        if (P->want_grad) {
          double score = seg / t.lam_nm[bin];
          if (relax) score = score - 1.0;
          Period& pr = periods.back();
          pr.A += score;
          pr.B += score * Xb;
        }
      }
      // ---- move
      for (int a = 0; a < 3; ++a) x[a] = x[a] + seg * u[a];
      if (final_seg) break;
      ++e;
      if (relax) {
        ++n_relax;
        if (P->nscat_curve) x_relax.push_back(X);
        if (P->n_scat_max > 0 && n_relax >= P->n_scat_max) break;
        ctr[2] = e;
        ctr[3] = 0; philox4x32_10(ctr, k0, k1, w);
        ctr[3] = 1; philox4x32_10(ctr, k0, k1, w1);
        bin = alias_draw(t.relax, n, w[0], w[1], w1[0]);
        dir_about_axis(u, 2, 1.0, 1.0 - 2.0 * oc32(w[2]), w[3]);
        d_rel = t.lam_nm[bin] * (-ln_(oc53(w1[1], w1[2])));
        d2 = draw_d2(e);
        if (P->want_grad) {
          periods.push_back({bin, -1.0, -X});
          ++n_res;
          sum_x_res += X;
        }
        continue;
      }
      d_rel = d_rel - seg;
      if (relax2) {
        // same mode, new isotropic direction (Sec. 3.5.1), new two-phonon clock
        ctr[2] = e;
        ctr[3] = 0; philox4x32_10(ctr, k0, k1, w);
        dir_about_axis(u, 2, 1.0, 1.0 - 2.0 * oc32(w[2]), w[3]);
        d2 = draw_d2(e);
        continue;
      }
      d2 = d2 - seg;
      if (face < 6) {
        int a = kFaceAxis[face];
        x[a] = kFaceIsMax[face] ? g.L[a] : 0.0;
        int ty = g.type[face];
        if (ty == 0) {
          out.scal[OR_ABSORBED] += 1.0;
          out.scal[OR_SIGNED_ABS] += s;
          break;
        } else if (ty == 2) {
          x[a] = kFaceIsMax[face] ? 0.0 : g.L[a];
        } else {
          ctr[2] = e;
          ctr[3] = 0; philox4x32_10(ctr, k0, k1, w);
          if ((uint64_t)w[0] < (g.fbin[face] ? t.spec_thr_bin[bin] : g.pthr[face])) {
            u[a] = -u[a];
          } else {
            dir_about_axis(u, a, kFaceIsMax[face] ? -1.0 : 1.0, std::sqrt(oc32(w[2])), w[3]);
          }
        }
      } else if (face >= 7) {
        // internal wall: onto its line, then specular or Lambertian about its normal
        const int k = face - 7;
        const double nx0 = g.snx[k], ny0 = g.sny[k];
        const double dn = (x[0] - g.sx1[k]) * nx0 + (x[1] - g.sy1[k]) * ny0;
        x[0] = x[0] - dn * nx0;
        x[1] = x[1] - dn * ny0;
        ctr[2] = e;
        ctr[3] = 0; philox4x32_10(ctr, k0, k1, w);
        if ((uint64_t)w[0] < (g.sbin[k] ? t.spec_thr_bin[bin] : g.sthr[k])) {
          double un = u[0] * nx0 + u[1] * ny0;
          u[0] = u[0] - (2.0 * un) * nx0;
          u[1] = u[1] - (2.0 * un) * ny0;
        } else {
          double mu = std::sqrt(oc32(w[2]));
          double sn = std::sqrt(std::max(0.0, 1.0 - mu * mu));
          double sphi, cphi;
          sincos2pi_(co32(w[3]), &sphi, &cphi);
          double sc = sn * cphi;
          u[0] = mu * nx0 - sc * ny0;
          u[1] = mu * ny0 + sc * nx0;
          u[2] = sn * sphi;
        }
      } else {
        // pore wall: outward normal of the cylinder points into the solid
        double nx0 = x[0] - g.cx, ny0 = x[1] - g.cy;
        double len = std::sqrt(nx0 * nx0 + ny0 * ny0);
        nx0 = nx0 / len;
        ny0 = ny0 / len;
        ctr[2] = e;
        ctr[3] = 0; philox4x32_10(ctr, k0, k1, w);
        bool spec = (uint64_t)w[0] < g.pthr_pore;
        ++n_pore;
        if (flip) {
          if (n_pore == flip) spec = !spec;
        } else if (P->want_grad && P->dp_mvd) {
          // reservoir choice, uniform over the trajectory's pore hits: hit j
          // takes the choice with probability 1/j, decided by the 64-bit word
          // r of sub-block 257 of its event (r <= floor((2^64 - 1) / j) holds
          // for exactly ceil(2^64 / j) of the 2^64 words)
          uint32_t c5[4] = {(uint32_t)pid, P->batch_index, e, 257u};
          uint32_t w5[4];
          philox4x32_10(c5, k0, k1, w5);
          const uint64_t r = (uint64_t)w5[0] | ((uint64_t)w5[1] << 32);
          if (r <= UINT64_MAX / (uint64_t)n_pore) {
            pick->sel = n_pore;
            pick->spec = spec;
          }
          pick->K = n_pore;
        } else if (P->want_grad) {
          double sc = spec ? 1.0 / g.p_pore : -1.0 / (1.0 - g.p_pore);
          PA += sc;
          PB += sc * X;
        }
        if (spec) {
          double un = u[0] * nx0 + u[1] * ny0;
          u[0] = u[0] - (2.0 * un) * nx0;
          u[1] = u[1] - (2.0 * un) * ny0;
        } else {
          double mu = std::sqrt(oc32(w[2]));
          double sn = std::sqrt(std::max(0.0, 1.0 - mu * mu));
          double sphi, cphi;
          sincos2pi_(co32(w[3]), &sphi, &cphi);
          double sc = sn * cphi;
          u[0] = mu * nx0 - sc * ny0;
          u[1] = mu * ny0 + sc * nx0;
          u[2] = sn * sphi;
        }
      }
    }
    const uint64_t nev = (uint64_t)e + 1;
    out.scal[OR_EVENTS] += (double)nev;
    if ((double)nev > out.scal[OR_MAXEV]) out.scal[OR_MAXEV] = (double)nev;
    if (truncated) out.scal[OR_TRUNC] += 1.0;
    out.scal[OR_SUMX] += X;
    out.scal[OR_SUMX2] += X * X;
    if (flip) return X;
    if (P->nscat_curve) {
      // a run with N_scat_max = k ends this trajectory at its k-th
      // relaxation (Sec. 3.5.6) with the tally it had there; a trajectory
      // that ended earlier is the same in that run
      for (int k = 1; k <= P->n_scat_max; ++k) {
        const double Xk = (size_t)k <= x_relax.size() ? x_relax[(size_t)k - 1] : X;
        out.curve[2 * (size_t)(k - 1) + 0] += Xk;
        out.curve[2 * (size_t)(k - 1) + 1] += Xk * Xk;
      }
    }
    if (O->events_pp) O->events_pp[pid - P->pid_begin] = (uint32_t)std::min<uint64_t>(nev, 0xFFFFFFFFu);
    if (O->X_pp) O->X_pp[pid - P->pid_begin] = X;
    if (P->want_grad) {
      for (const Period& pr : periods) out.G[pr.bin] += pr.A * X - pr.B;
      double R = (double)n_res * X - sum_x_res;
      out.scal[OR_RSUM] += R;
      if (!P->dp_mvd) {
        double gp = PA * X - PB;
        out.scal[OR_GP] += gp;
        out.scal[OR_GP2] += gp * gp;
      }
      for (int kd = 0; kd < P->n_dirs; ++kd) {
        const double* d = P->dirs + (size_t)kd * n;
        double val = 0.0;
        for (const Period& pr : periods) val += (pr.A * X - pr.B) * d[pr.bin];
        val += R * S.dpi_dirs[kd];
        out.dsum[kd] += val;
        out.dsum2[kd] += val * val;
      }
    }
    return X;
  };
  for (uint64_t pid = p0; pid < p1; ++pid) {
    MvdPick pick;
    const double X = trace_one(pid, 0, &pick);
    if (P->want_grad && P->dp_mvd) {
      // measure-valued derivative of the specular / diffuse draw at the chosen
      // hit: K (X with a specular reflection there - X with a diffuse one),
      // whose mean over the uniform choice is the sum over all K hits
      double D = 0.0;
      if (pick.K > 0) {
        const double Xph = trace_one(pid, pick.sel, nullptr);
        D = (double)pick.K * (pick.spec ? X - Xph : Xph - X);
      }
      res.scal[OR_GP] += D;
      res.scal[OR_GP2] += D * D;
    }
  }
}

}  // namespace

extern "C" {

void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  philox4x32_10(ctr, key[0], key[1], out);
}

double or_dEdT(double omega, double T) { return dEdT(omega, T); }

double or_log(double x) { return series_log(x); }

void or_set_libm(int on) { g_use_libm = on ? 1 : 0; }

void or_sincos2pi(double r, double* s, double* c) { series_sincos2pi(r, s, c); }

// Alias table of arbitrary weights (for the table tests).
void or_alias(int n, const double* w, double* prob, uint64_t* thr, int32_t* alias) {
  std::vector<double> ww(w, w + n);
  Alias a = build_alias(ww);
  for (int i = 0; i < n; ++i) { prob[i] = a.prob[i]; thr[i] = a.thr[i]; alias[i] = a.alias[i]; }
}

int or_alias_draw(int n, const uint64_t* thr, const int32_t* alias, uint32_t wcol, uint32_t lo, uint32_t hi) {
  Alias a;
  a.thr.assign(thr, thr + n);
  a.alias.assign(alias, alias + n);
  return alias_draw(a, n, wcol, lo, hi);
}

// Material tables: C[n]; for table k in (emit ~ C v, init ~ C, relax ~ C/tau):
// prob[k*n+i], thr[k*n+i], alias[k*n+i]; sums = (C_tot, sum C v, sum C/tau).
int or_tables(const or_params* P, double* C, double* prob, uint64_t* thr, int32_t* alias, double* sums) {
  Tables t;
  if (build_tables(P, t)) return 1;
  const int n = t.n;
  const Alias* al[3] = {&t.emit, &t.init, &t.relax};
  for (int i = 0; i < n; ++i) C[i] = t.C[i];
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < n; ++i) {
      prob[k * n + i] = al[k]->prob[i];
      thr[k * n + i] = al[k]->thr[i];
      alias[k * n + i] = al[k]->alias[i];
    }
  sums[0] = t.C_tot; sums[1] = t.sum_Cv; sums[2] = t.sum_Ct;
  return 0;
}

// Geometry probe for the unit tests: x, u in nm.
int or_first_hit(const or_params* P, const double x[3], const double u[3], double* dist, int* face) {
  Tables t;
  Setup S;
  Geo& g = S.g;
  for (int a = 0; a < 3; ++a) g.L[a] = P->L[a] * 1e9;
  g.pore = P->pore != 0;
  g.cx = P->pore_c[0] * 1e9; g.cy = P->pore_c[1] * 1e9; g.r = P->pore_r * 1e9; g.r2 = g.r * g.r;
  g.n_inner = P->n_inner;
  for (int k = 0; k < g.n_inner; ++k) {
    g.sx1[k] = P->inner[k][0] * 1e9; g.sy1[k] = P->inner[k][1] * 1e9;
    g.sx2[k] = P->inner[k][2] * 1e9; g.sy2[k] = P->inner[k][3] * 1e9;
    g.snx[k] = P->inner_n[k][0]; g.sny[k] = P->inner_n[k][1];
  }
  first_hit(g, x, u, dist, face);
  return 0;
}

// The direction of a body particle about sgn * gv (pins of the frame).
int or_dir_about_vector(const double gv[3], double sgn, double mu, uint32_t wphi, double u[3]) {
  dir_about_vector(u, gv, sgn, mu, wphi);
  return 0;
}

// 1 if (x, y) (nm) lies inside a hole bounded by the internal segments.
int or_in_hole(const or_params* P, double x, double y) {
  Geo g;
  g.n_inner = P->n_inner;
  for (int k = 0; k < g.n_inner; ++k) {
    g.sx1[k] = P->inner[k][0] * 1e9; g.sy1[k] = P->inner[k][1] * 1e9;
    g.sx2[k] = P->inner[k][2] * 1e9; g.sy2[k] = P->inner[k][3] * 1e9;
  }
  return in_hole(g, x, y) ? 1 : 0;
}

// Source energies: out[0] = E_tot, out[1] = V_solid, out[2..] = E per source.
int or_sources(const or_params* P, double* out, int* n_src) {
  Tables t;
  if (build_tables(P, t)) return 1;
  Setup S;
  int rc = setup(P, t, S);
  if (rc) return 10 + rc;
  out[0] = S.E_tot;
  out[1] = S.g.V_solid_m3;
  for (size_t k = 0; k < S.src.size(); ++k) out[2 + k] = S.src[k].E;
  *n_src = (int)S.src.size();
  return 0;
}

int or_run(const or_params* P, or_out* O) {
  Tables t;
  if (build_tables(P, t)) return 1;
  Setup S;
  int rc = setup(P, t, S);
  if (rc) return 10 + rc;
  if (P->transient && (P->grid[0] < 1 || P->grid[1] < 1 || P->grid[2] < 1)) return 20;
  if (P->want_grad && P->transient) return 21;
  if (P->nscat_curve && (P->transient || P->n_scat_max < 1 || !O->curve)) return 22;
  const uint64_t total = P->pid_end - P->pid_begin;
  int nt = P->n_threads > 0 ? P->n_threads : (int)std::thread::hardware_concurrency();
  if (nt < 1) nt = 1;
  if ((uint64_t)nt > total) nt = (int)std::max<uint64_t>(1, total);
  const size_t ncell_t = S.n_det;
  std::vector<Partial> parts(nt);
  for (auto& p : parts) {
    if (!P->transient && P->n_cells > 0) { p.T.assign(P->n_cells, 0.0); p.Q.assign((size_t)P->n_cells * 3, 0.0); }
    if (O->qbin_sum) p.qbin.assign(P->n_bins, 0.0);
    if (P->transient) p.snap.assign((size_t)P->n_times * ncell_t * 4, 0.0);
    else if (P->n_regions > 0)                                      // steady detector regions
      p.snap.assign(ncell_t * 4 * (P->det_per_bin ? (size_t)P->n_bins : 1), 0.0);
    if (P->want_grad) { p.G.assign(P->n_bins, 0.0); p.dsum.assign(P->n_dirs, 0.0); p.dsum2.assign(P->n_dirs, 0.0); }
    if (P->nscat_curve) p.curve.assign(2 * (size_t)P->n_scat_max, 0.0);
  }
  std::vector<std::thread> th;
  for (int i = 0; i < nt; ++i) {
    uint64_t a = P->pid_begin + total * (uint64_t)i / (uint64_t)nt;
    uint64_t b = P->pid_begin + total * (uint64_t)(i + 1) / (uint64_t)nt;
    th.emplace_back([&, a, b, i]() { trace_range(P, t, S, a, b, parts[i], O); });
  }
  for (auto& x : th) x.join();
  for (int k = 0; k < OR_NSCAL; ++k) O->scal[k] = 0.0;
  for (int i = 0; i < nt; ++i) {
    const Partial& p = parts[i];
    for (int k = 0; k < OR_NSCAL; ++k) {
      if (k == OR_MAXEV) O->scal[k] = std::max(O->scal[k], p.scal[k]);
      else O->scal[k] += p.scal[k];
    }
    if (O->T_sum) for (size_t c = 0; c < p.T.size(); ++c) O->T_sum[c] += p.T[c];
    if (O->Q_sum) for (size_t c = 0; c < p.Q.size(); ++c) O->Q_sum[c] += p.Q[c];
    if (O->qbin_sum) for (size_t c = 0; c < p.qbin.size(); ++c) O->qbin_sum[c] += p.qbin[c];
    if (O->snap) for (size_t c = 0; c < p.snap.size(); ++c) O->snap[c] += p.snap[c];
    if (O->G) for (size_t c = 0; c < p.G.size(); ++c) O->G[c] += p.G[c];
    if (O->dir_sum) for (size_t c = 0; c < p.dsum.size(); ++c) { O->dir_sum[c] += p.dsum[c]; O->dir_sum2[c] += p.dsum2[c]; }
    if (O->curve) for (size_t c = 0; c < p.curve.size(); ++c) O->curve[c] += p.curve[c];
  }
  O->scal[OR_ETOT] = S.E_tot;
  O->scal[OR_CTOT] = t.C_tot;
  O->scal[OR_VSOLID] = S.g.V_solid_m3;
  (void)nt;
  return 0;
}

}  // extern "C"
