// Steady-state tracing (Sec. 3.6, Eq. steady_estimate): the FP64 plain
// kernel (one thread per particle, FP64 throughout) and the persistent FP32
// kernel (FP32 flights, FP64 tallies, per-lane refill from a warp-aggregated
// work counter, shared-memory alias tables and privatised tallies), plus the
// per-run setup and finalisation kernels.
#include "launch.h"

#ifndef MCBTE_F64
#define MCBTE_F64 0
#endif
#ifndef MCBTE_F32
#define MCBTE_F32 0
#endif

namespace mcbte {

namespace {

__device__ __forceinline__ uint64_t spec_threshold(double p) {
  if (p <= 0.0) return 0ull;
  if (p >= 1.0) return 1ull << 32;
  return (uint64_t)(p * 4294967296.0);
}

#if MCBTE_F64
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
  for (int f = 0; f < 6; ++f) {
    r.type[f] = d.face_type[f];
    r.pthr[f] = spec_threshold(d.face_p[f]);
    r.face_sign[f] = (d.face_T[f] > d.T_eq) ? 1.0 : -1.0;
  }
  r.pore = d.pore;
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
  for (int k = 0; k < 3; ++k)
    if (d.grad_T[k] != 0.0) {
      r.grad_axis = k;
      r.grad_sign = d.grad_T[k] > 0.0 ? 1.0 : -1.0;
    }
  if (r.grad_sign != 0.0) {
    E[ns] = ((0.5 * V) * fabs(d.grad_T[r.grad_axis])) * sum_Cv;
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
  geos[gi] = r;
}
#endif  // MCBTE_F64

__device__ __forceinline__ int find_geom(const uint64_t* offs, int G, uint64_t idx) {
  int lo = 0, hi = G;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (offs[mid] <= idx) lo = mid; else hi = mid;
  }
  return lo;
}

// Book-keeping of a finished particle (idx = flattened index).
template <typename R, bool GRAD>
__device__ __forceinline__ void finish_particle(const Particle<R>& p, int outcome, uint64_t idx, const RunCfg& C,
                                                const Acc& A, double* qb, const GradState* gs, const MatView& M) {
  const int g = p.g;
  const unsigned long long nev = (unsigned long long)p.e + 1ull;
  atomicAdd(&A.cnt[g * 4 + 0], nev);
  if (outcome == STEP_TRUNCATED) atomicAdd(&A.cnt[g * 4 + 1], 1ull);
  atomicMax(&A.cnt[g * 4 + 2], nev);
  atomicAdd(&A.cnt[g * 4 + 3], 1ull);
  atomicAdd(&A.dsc[g * 8 + 0], p.X);
  atomicAdd(&A.dsc[g * 8 + 1], p.X * p.X);
  atomicAdd(&A.dsc[g * 8 + 2], (double)p.s);
  if (outcome == STEP_ABSORBED) {
    atomicAdd(&A.dsc[g * 8 + 3], (double)p.s);
    atomicAdd(&A.dsc[g * 8 + 7], 1.0);
  }
  if (qb) atomicAdd(&qb[p.bin], p.X - p.Xper);
  if (A.events_pp) A.events_pp[idx] = (uint32_t)nev;
  if (A.X_pp) A.X_pp[idx] = p.X;
  if (GRAD) {
    const double X = p.X;
    for (int k = 0; k < gs->np; ++k) atomicAdd(&A.G[gs->bin[k]], gs->A[k] * X - gs->B[k]);
    const double Rv = (double)gs->n_res * X - gs->sum_x_res;
    atomicAdd(&A.dsc[g * 8 + 4], Rv);
    const double gp = gs->PA * X - gs->PB;
    atomicAdd(&A.dsc[g * 8 + 5], gp);
    atomicAdd(&A.dsc[g * 8 + 6], gp * gp);
    for (int kd = 0; kd < C.n_dirs; ++kd) {
      const double* dd = C.dirs + (size_t)kd * M.n;
      double val = 0.0;
      for (int k = 0; k < gs->np; ++k) val += (gs->A[k] * X - gs->B[k]) * dd[gs->bin[k]];
      val += Rv * C.dpi[kd];
      atomicAdd(&A.dsum[kd * 2 + 0], val);
      atomicAdd(&A.dsum[kd * 2 + 1], val * val);
    }
  }
}

template <typename R>
__device__ __forceinline__ void grad_init(GradState* gs, const Particle<R>& p) {
  gs->np = 1;
  gs->bin[0] = p.bin;
  gs->A[0] = 0.0;
  gs->B[0] = 0.0;
  gs->n_res = 0;
  gs->sum_x_res = 0.0;
  gs->PA = 0.0;
  gs->PB = 0.0;
}

#if MCBTE_F64
// ------------------------------------------------------------------ FP64 plain
template <int CELLS, bool GRAD>
__global__ void __launch_bounds__(256) k_steady_fp64(const GeoRun* __restrict__ geos, const uint64_t* __restrict__ offs,
                                                     MatView M, RunCfg C, Acc A) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= C.total) return;
  const int g = find_geom(offs, C.n_geoms, idx);
  const GeoRun& G = geos[g];
  const uint64_t deadline = *C.t0 + C.budget_ns;
  Particle<double> p;
  p.pid = (uint32_t)(idx - offs[g]);
  p.g = g;
  emit<double>(p, G, M, M.rec_emit, M.rec_init, nullptr, C.k0, C.k1, false, 0.0);
  GradState gs;
  if (GRAD) grad_init(&gs, p);
  double* cP = A.cellP ? A.cellP + (size_t)g * C.n_cells * 4 : nullptr;
  double* cD = A.cellD ? A.cellD + (size_t)g * (C.n_cells + 1) * 4 : nullptr;
  double* qb = C.per_bin ? A.qbin + (size_t)g * M.n : nullptr;
  const double h = (CELLS != 0) ? G.L[C.cell_axis] / (double)C.n_cells : 1.0;
  int out;
  for (;;) {
    out = step_steady<double, CELLS, GRAD>(p, G, M, M.rec_relax, nullptr, C, cP, cD, h, 1.0 / h, qb, &gs);
    if (out != STEP_ALIVE) break;
    if ((p.e & 1023u) == 0u && globaltimer_ns() > deadline) {
      atomicOr(A.flags, 1);
      out = STEP_TRUNCATED;
      break;
    }
  }
  finish_particle<double, GRAD>(p, out, idx, C, A, qb, &gs, M);
}

#endif  // MCBTE_F64
#if MCBTE_F32
// ------------------------------------------------------------------ FP32 persistent
// Every lane owns one particle at a time.  When its particle terminates the
// lane refills from a global work counter; the refills of a warp are
// aggregated into one atomicAdd (ballot of the empty lanes, leader adds the
// popcount, lanes take consecutive indices).  Lanes therefore never idle
// while work remains, whatever the event-count spread between particles.
template <int CELLS, bool GRAD>
__global__ void __launch_bounds__(512) k_steady_f32(const GeoRun* __restrict__ geos, const uint64_t* __restrict__ offs,
                                                    MatView M, RunCfg C, Acc A, SmemPlan S) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* sp = smem;
  const int n = M.n;
  const uint4* relax = M.rec_relax;
  const float4* binf = M.binf;
  double* s_qbin = nullptr;
  double* s_cP = nullptr;
  double* s_cD = nullptr;
  if (S.relax_in_smem) {
    uint4* t = reinterpret_cast<uint4*>(sp);
    for (int i = threadIdx.x; i < n; i += blockDim.x) t[i] = M.rec_relax[i];
    relax = t;
    sp += (size_t)n * sizeof(uint4);
  }
  if (S.binf_in_smem) {
    float4* t = reinterpret_cast<float4*>(sp);
    for (int i = threadIdx.x; i < n; i += blockDim.x) t[i] = M.binf[i];
    binf = t;
    sp += (size_t)n * sizeof(float4);
  }
  if (S.qbin_in_smem) {
    s_qbin = reinterpret_cast<double*>(sp);
    for (int i = threadIdx.x; i < n; i += blockDim.x) s_qbin[i] = 0.0;
    sp += (size_t)n * sizeof(double);
  }
  const int nc = C.n_cells;
  if (S.cells_in_smem) {
    s_cP = reinterpret_cast<double*>(sp);
    s_cD = s_cP + (size_t)nc * 4;
    for (int i = threadIdx.x; i < nc * 4 + (nc + 1) * 4; i += blockDim.x) s_cP[i] = 0.0;
  }
  __syncthreads();

  const unsigned lane = threadIdx.x & 31u;
  const uint64_t deadline = *C.t0 + C.budget_ns;
  Particle<float> p;
  GradState gs;
  bool alive = false;
  uint64_t idx = 0;
  double* cP = nullptr;
  double* cD = nullptr;
  double* qb = nullptr;
  float h = 1.0f, inv_h = 1.0f;
  const GeoRun* G = geos;
  for (;;) {
    const unsigned act = __activemask();
    const unsigned need = __ballot_sync(act, !alive);
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(A.work, (unsigned long long)__popc(need));
      base = __shfl_sync(act, base, leader);
      if (!alive) {
        idx = base + (unsigned long long)__popc(need & ((1u << lane) - 1u));
        if (idx >= C.total) break;
        if (*(volatile int*)A.flags & 1) break;
        const int g = find_geom(offs, C.n_geoms, idx);
        G = &geos[g];
        p.pid = (uint32_t)(idx - offs[g]);
        p.g = g;
        emit<float>(p, *G, M, M.rec_emit, M.rec_init, binf, C.k0, C.k1, false, 0.0f);
        if (GRAD) grad_init(&gs, p);
        if (CELLS) {
          cP = S.cells_in_smem ? s_cP : A.cellP + (size_t)g * nc * 4;
          cD = S.cells_in_smem ? s_cD : A.cellD + (size_t)g * (nc + 1) * 4;
          h = G->Lf[C.cell_axis] / (float)nc;
          inv_h = (float)nc / G->Lf[C.cell_axis];
        }
        qb = C.per_bin ? (S.qbin_in_smem ? s_qbin : A.qbin + (size_t)g * n) : nullptr;
        alive = true;
      }
    }
    int out = step_steady<float, CELLS ? 2 : 0, GRAD>(p, *G, M, relax, binf, C, cP, cD, h, inv_h, qb, &gs);
    if (out == STEP_ALIVE && (p.e & 255u) == 0u && globaltimer_ns() > deadline) {
      atomicOr(A.flags, 1);
      out = STEP_TRUNCATED;
    }
    if (out != STEP_ALIVE) {
      finish_particle<float, GRAD>(p, out, idx, C, A, qb, &gs, M);
      alive = false;
    }
  }
  __syncthreads();
  if (S.qbin_in_smem) {
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (s_qbin[i] != 0.0) atomicAdd(&A.qbin[i], s_qbin[i]);
  }
  if (S.cells_in_smem) {
    for (int i = threadIdx.x; i < nc * 4; i += blockDim.x)
      if (s_cP[i] != 0.0) atomicAdd(&A.cellP[i], s_cP[i]);
    for (int i = threadIdx.x; i < (nc + 1) * 4; i += blockDim.x)
      if (s_cD[i] != 0.0) atomicAdd(&A.cellD[i], s_cD[i]);
  }
}

#endif  // MCBTE_F32
#if MCBTE_F64
// ------------------------------------------------------------------ finalise
// One block per geometry: scale the raw sums into the paper's estimators
// (Eqs. temp_steady, flux_x_steady), kappa = -q / (dT/dx) and its standard
// error from the per-particle X_p (iid), and the LR gradient.
__global__ void k_finalize_steady(const GeoRun* geos, MatView M, RunCfg C, Acc A, SteadyOutDev O, int grad,
                                  const int* flags) {
  const int g = blockIdx.x;
  const GeoRun& G = geos[g];
  const int nc = C.n_cells;
  const int n = M.n;
  const double N = (double)G.n;
  const double E_eff = G.E_tot / N;
  const double C_tot = M.sums[0];
  if (nc > 0 && threadIdx.x == 0) {
    const double Vc = G.V_box / (double)nc;
    const double kT = E_eff / (C_tot * Vc);
    const double kq = E_eff / Vc;
    double run[4] = {0.0, 0.0, 0.0, 0.0};
    const double* P = A.cellP + (size_t)g * nc * 4;
    const double* D = A.cellD + (size_t)g * (nc + 1) * 4;
    for (int c = 0; c < nc; ++c) {
      double v[4];
      for (int b = 0; b < 4; ++b) {
        run[b] += D[c * 4 + b];
        v[b] = P[c * 4 + b] + run[b];
      }
      if (O.T) O.T[(size_t)g * nc + c] = (kT * v[0]) * 1e-12;
      if (O.q)
        for (int b = 0; b < 3; ++b) O.q[((size_t)g * nc + c) * 3 + b] = (kq * v[1 + b]) * 1e-9;
    }
  }
  if (O.q_bin && C.per_bin) {
    const double kb = E_eff / G.V_solid;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      O.q_bin[(size_t)g * n + i] = (kb * A.qbin[(size_t)g * n + i]) * 1e-9;
  }
  if (threadIdx.x == 0) {
    const double sx = A.dsc[g * 8 + 0], sx2 = A.dsc[g * 8 + 1];
    const double nt = (double)A.cnt[g * 4 + 3];
    const double mean = sx / nt;
    const double var = nt > 1.0 ? (sx2 - nt * mean * mean) / (nt - 1.0) : 0.0;
    const double q_mean = (E_eff / G.V_solid) * sx * 1e-9;
    const double q_se = (G.E_tot / G.V_solid) * 1e-9 * sqrt(fmax(var, 0.0) / nt);
    double* st = O.stats + (size_t)g * MCBTE_NSTATS;
    st[MCBTE_STAT_KAPPA] = -q_mean / G.kappa_grad;
    st[MCBTE_STAT_KAPPA_SE] = q_se / fabs(G.kappa_grad);
    st[MCBTE_STAT_Q_MEAN] = q_mean;
    st[MCBTE_STAT_Q_SE] = q_se;
    st[MCBTE_STAT_SUMX] = sx;
    st[MCBTE_STAT_SUMX2] = sx2;
    st[MCBTE_STAT_EVENTS] = (double)A.cnt[g * 4 + 0];
    st[MCBTE_STAT_TRUNCATED] = (double)A.cnt[g * 4 + 1];
    st[MCBTE_STAT_E_TOT] = G.E_tot;
    st[MCBTE_STAT_MAX_EVENTS] = (double)A.cnt[g * 4 + 2];
    st[MCBTE_STAT_KAPPA_CELL] = (-q_mean / G.kappa_grad) * (G.V_solid / G.V_box);
    st[MCBTE_STAT_SIGNED_EMITTED] = A.dsc[g * 8 + 2];
    st[MCBTE_STAT_SIGNED_ABSORBED] = A.dsc[g * 8 + 3];
    st[MCBTE_STAT_STATUS] = (flags[0] & 1) ? (double)MCBTE_ERR_TIMEOUT
                                           : (A.cnt[g * 4 + 1] ? (double)MCBTE_WARN_TRUNCATED : 0.0);
    st[MCBTE_STAT_N] = nt;
    st[15] = A.dsc[g * 8 + 7];
  }
  if (grad && g == 0) {
    const double scale = -(E_eff / G.V_solid) * 1e-9 / G.kappa_grad;
    const double Rs = A.dsc[4];
    for (int i = threadIdx.x; i < n; i += blockDim.x) O.dk[i] = scale * (A.G[i] + Rs * M.pi[i]);
    if (threadIdx.x == 0) {
      const double nt = (double)A.cnt[3];
      const double gm = A.dsc[5] / nt;
      const double gv = (A.dsc[6] - nt * gm * gm) / fmax(nt - 1.0, 1.0);
      const bool ok = G.pore && G.p_pore > 0.0 && G.p_pore < 1.0;
      const double nan = __longlong_as_double(0x7ff8000000000000ll);
      O.dkp[0] = ok ? scale * A.dsc[5] : nan;
      O.dkp[1] = ok ? fabs(scale) * sqrt(fmax(gv, 0.0) * nt) : nan;
      for (int k = 0; k < C.n_dirs; ++k) {
        const double dm = A.dsum[k * 2] / nt;
        const double dv = (A.dsum[k * 2 + 1] - nt * dm * dm) / fmax(nt - 1.0, 1.0);
        O.dkdir[k * 2 + 0] = scale * A.dsum[k * 2];
        O.dkdir[k * 2 + 1] = fabs(scale) * sqrt(fmax(dv, 0.0) * nt);
      }
    }
  }
}

__global__ void k_dirs_dot_pi(const double* dirs, int nd, MatView M, double* dpi) {
  const int k = threadIdx.x;
  if (k >= nd) return;
  double acc = 0.0;
  for (int i = 0; i < M.n; ++i) acc += dirs[(size_t)k * M.n + i] * M.pi[i];
  dpi[k] = acc;
}

#endif  // MCBTE_F64
#if MCBTE_F32
template <int CELLS, bool GRAD>
cudaError_t launch_f32(const GeoRun* geos, const uint64_t* offs, const MatView& M, const RunCfg& C, const Acc& A,
                       int threads, int bps, cudaStream_t s) {
  const SmemPlan S = plan_smem_f32(M.n, C.n_geoms, C.n_cells, C.per_bin, 200 * 1024);
  auto kern = k_steady_f32<CELLS, GRAD>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.bytes);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, S.bytes);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int b = (bps > 0 && bps < occ) ? bps : occ;
  kern<<<sm_count() * b, threads, S.bytes, s>>>(geos, offs, M, C, A, S);
  return cudaGetLastError();
}

#endif  // MCBTE_F32
#if MCBTE_F64
template <int CELLS, bool GRAD>
cudaError_t launch_f64(const GeoRun* geos, const uint64_t* offs, const MatView& M, const RunCfg& C, const Acc& A,
                       cudaStream_t s) {
  const uint64_t blocks = (C.total + 255) / 256;
  k_steady_fp64<CELLS, GRAD><<<(unsigned)blocks, 256, 0, s>>>(geos, offs, M, C, A);
  return cudaGetLastError();
}

#endif  // MCBTE_F64
}  // namespace

#if MCBTE_F64
SmemPlan plan_smem_f32(int n_bins, int n_geoms, int n_cells, int per_bin, size_t budget) {
  SmemPlan S{0, 0, 0, 0, 0};
  size_t used = 0;
  const size_t cells = (size_t)(n_cells * 4 + (n_cells + 1) * 4) * sizeof(double);
  if (n_cells > 0 && n_geoms == 1 && cells <= 16 * 1024) {
    S.cells_in_smem = 1;
    used += cells;
  }
  if (per_bin && n_geoms == 1 && used + (size_t)n_bins * 8 <= budget / 3) {
    S.qbin_in_smem = 1;
    used += (size_t)n_bins * 8;
  }
  if (used + (size_t)n_bins * 16 <= budget) {
    S.relax_in_smem = 1;
    used += (size_t)n_bins * 16;
  }
  if (used + (size_t)n_bins * 16 <= budget) {
    S.binf_in_smem = 1;
    used += (size_t)n_bins * 16;
  }
  S.bytes = used;
  return S;
}

int sm_count() {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    if (cached < 1) cached = 1;
  }
  return cached;
}

cudaError_t launch_setup(const SetupArgs& a, int n_geoms, const MatView& M, int transient, double t_max_s,
                         int tally_axis, GeoRun* geos, uint64_t* offs, unsigned long long* t0, cudaStream_t s) {
  k_setup<<<1, kMaxGeoms, 0, s>>>(a, n_geoms, M, transient, t_max_s, tally_axis, geos, offs, t0);
  return cudaGetLastError();
}

cudaError_t launch_steady(int precision, bool grad, const GeoRun* geos, const uint64_t* offs, const MatView& M,
                          const RunCfg& C, const Acc& A, int threads, int bps, cudaStream_t s) {
  const bool cells = C.n_cells > 0;
  if (precision == MCBTE_FP64_PLAIN) {
    if (grad) return cells ? launch_f64<1, true>(geos, offs, M, C, A, s) : launch_f64<0, true>(geos, offs, M, C, A, s);
    return cells ? launch_f64<1, false>(geos, offs, M, C, A, s) : launch_f64<0, false>(geos, offs, M, C, A, s);
  }
  return launch_steady_f32(grad, cells, geos, offs, M, C, A, threads > 0 ? threads : 256, bps, s);
}

cudaError_t launch_finalize_steady(const GeoRun* geos, const MatView& M, const RunCfg& C, const Acc& A,
                                   const SteadyOutDev& O, bool grad, const int* flags, cudaStream_t s) {
  k_finalize_steady<<<C.n_geoms, 256, 0, s>>>(geos, M, C, A, O, grad ? 1 : 0, flags);
  return cudaGetLastError();
}

cudaError_t launch_dirs_dot_pi(const double* dirs, int n_dirs, const MatView& M, double* dpi, cudaStream_t s) {
  if (n_dirs <= 0) return cudaSuccess;
  k_dirs_dot_pi<<<1, 32, 0, s>>>(dirs, n_dirs, M, dpi);
  return cudaGetLastError();
}

#endif  // MCBTE_F64

#if MCBTE_F32
cudaError_t launch_steady_f32(bool grad, bool cells, const GeoRun* geos, const uint64_t* offs, const MatView& M,
                              const RunCfg& C, const Acc& A, int threads, int bps, cudaStream_t s) {
  if (grad)
    return cells ? launch_f32<1, true>(geos, offs, M, C, A, threads, bps, s)
                 : launch_f32<0, true>(geos, offs, M, C, A, threads, bps, s);
  return cells ? launch_f32<1, false>(geos, offs, M, C, A, threads, bps, s)
               : launch_f32<0, false>(geos, offs, M, C, A, threads, bps, s);
}
#endif  // MCBTE_F32

}  // namespace mcbte
