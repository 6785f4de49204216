// Steady-state tracing (Sec. 3.6, Eq. steady_estimate): the FP64 plain
// kernel (one thread per particle, FP64 throughout) and the persistent FP32
// kernel (FP32 flights; 64-bit fixed-point tallies privatised in shared
// memory, reduced to FP64; per-lane refill from a warp-aggregated work
// counter; alias tables in shared memory), plus the finalisation kernel.
//
// This file is compiled three times: with MCBTE_F64 (FP64 kernels, no fused
// multiply-add) and with MCBTE_F32 twice, MCBTE_F32_PART 0 (the FP32 kernels
// of runs without the tail kernel, and the launch dispatch) and 1 (the FP32
// kernels that park their tail, and the tail kernels), built in parallel.
#include <atomic>

#include "launch.h"

#ifndef MCBTE_F64
#define MCBTE_F64 0
#endif
#ifndef MCBTE_F32
#define MCBTE_F32 0
#endif
#ifndef MCBTE_F32_PART
#define MCBTE_F32_PART 0
#endif

namespace mcbte {

namespace {

__device__ __forceinline__ int find_geom(const uint64_t* offs, int G, uint64_t idx) {
  int lo = 0, hi = G;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (offs[mid] <= idx) lo = mid; else hi = mid;
  }
  return lo;
}

// N_scat_max curve: a trajectory that ended (absorbed, truncated) after m <
// n_scat_max relaxations has the same final tally X in every run with
// N_scat_max > m; it enters the difference array at m + 1.
__device__ __forceinline__ void nscat_end(const RunCfg& C, int g, int m, double X) {
  if (!C.nscat_acc || m >= C.n_scat_max) return;
  double* a = nscat_slot(C, g, m + 1);
  atomicAdd(a + 2, X);
  atomicAdd(a + 3, X * X);
}

// Likelihood-ratio contributions of a finished particle with tally X: every
// relaxation period's value into G[bin], the dense resampling term R, the
// specularity score and the probe directions.
template <class Grad>
__device__ __forceinline__ void grad_finish(const Grad& gr, double X, int g, const RunCfg& C, const Acc& A,
                                            const MatView& M) {
  const int np = gr.periods();
  for (int k = 0; k < np; ++k) atomicAdd(&A.G[gr.period_bin(k)], gr.period_value(k, X));
  const double Rv = gr.resample_term(X);
  double* gs = grad_copy(A);
  atomicAdd(gs + 0, Rv);
  if (!C.mvd) {   // the measure-valued score is added after the phantom trace
    const double gp = gr.spec_term(X);
    atomicAdd(gs + 1, gp);
    atomicAdd(gs + 2, gp * gp);
  }
  for (int kd = 0; kd < C.n_dirs; ++kd) {
    const double* dd = C.dirs + (size_t)kd * M.n;
    double val = 0.0;
    for (int k = 0; k < np; ++k) val += gr.period_value(k, X) * dd[gr.period_bin(k)];
    val += Rv * C.dpi[kd];
    atomicAdd(gs + 4 + 2 * kd, val);
    atomicAdd(gs + 5 + 2 * kd, val * val);
  }
}

template <bool GRAD, class On>
struct GradPick { using type = On; };
template <class On>
struct GradPick<false, On> { using type = GradOff; };

#if MCBTE_F64
// ------------------------------------------------------------------ FP64 plain
template <bool CELLS, bool GRAD>
__global__ void __launch_bounds__(256) k_steady_fp64(const GeoRun* __restrict__ geos, const uint64_t* __restrict__ offs,
                                                     MatView M, RunCfg C, Acc A) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= C.total) return;
  const int g = find_geom(offs, C.n_geoms, idx);
  const GeoRun& G = geos[g];
  const uint64_t deadline = *C.t0 + C.budget_ns;
  Particle<double> p;
  p.pid = (uint32_t)(idx - offs[g] + G.pid0);
  p.g = g;
  const uint2 key = run_key(C);
  if (globaltimer_ns() > deadline) {   // over budget before this particle started
    atomicOr(A.flags, 1);
    return;
  }
  emit<double>(p, G, M, M.rec_emit, M.rec_init, nullptr, key.x, key.y, false, 0.0);
  typename GradPick<GRAD, GradList>::type gr;
  if constexpr (GRAD) gr.mvd = C.mvd != 0;
  if (GRAD) gr.init(p.bin);
  TallyPlain T;
  T.cP = CELLS ? A.cellP + (size_t)g * C.n_cells * 4 : nullptr;
  T.qb = C.per_bin ? A.qbin + (size_t)g * M.n : nullptr;
  T.nc = C.n_cells;
  T.ca = C.cell_axis;
  T.ta = C.tally_axis;
  T.h = CELLS ? G.L[C.cell_axis] / (double)C.n_cells : 1.0;
  T.det = C.n_regs > 0 ? A.det_raw : nullptr;
  int out;
  for (;;) {
    out = step_steady<double, typename GradPick<GRAD, GradList>::type, TallyPlain>(p, G, M, M.rec_relax, nullptr, C,
                                                                                 key.x, key.y, T, gr);
    if (out != STEP_ALIVE) break;
    if ((p.e & 1023u) == 0u && globaltimer_ns() > deadline) {
      atomicOr(A.flags, 1);
      out = STEP_TRUNCATED;
      break;
    }
  }
  T.period_end(p);
  const unsigned long long nev = (unsigned long long)p.e + 1ull;
  atomicAdd(&A.cnt[g * 4 + 0], nev);
  if (out == STEP_TRUNCATED) atomicAdd(&A.cnt[g * 4 + 1], 1ull);
  atomicMax(&A.cnt[g * 4 + 2], nev);
  atomicAdd(&A.cnt[g * 4 + 3], 1ull);
  atomicAdd(&A.dsc[g * 8 + 0], p.X);
  atomicAdd(&A.dsc[g * 8 + 1], p.X * p.X);
  atomicAdd(&A.dsc[g * 8 + 2], p.s);
  if (out == STEP_ABSORBED) {
    atomicAdd(&A.dsc[g * 8 + 3], p.s);
    atomicAdd(&A.dsc[g * 8 + 7], 1.0);
  }
  if (A.events_pp) A.events_pp[idx] = (uint32_t)nev;
  if (A.X_pp) A.X_pp[idx] = p.X;
  nscat_end(C, g, p.n_relax, p.X);
  if constexpr (GRAD) {
    grad_finish(gr, p.X, g, C, A, M);
    if (C.mvd && gr.mv.sel > 0u) {
      // measure-valued d/dp_pore: the particle again from its emission, the
      // chosen pore hit's branch flipped; nothing is tallied but its X
      const double Xn = p.X;
      gr.mv.start_phantom();
      emit<double>(p, G, M, M.rec_emit, M.rec_init, nullptr, key.x, key.y, false, 0.0);
      TallyPlain Tq;
      Tq.cP = nullptr;
      Tq.qb = nullptr;
      Tq.nc = C.n_cells;
      Tq.ca = C.cell_axis;
      Tq.ta = C.tally_axis;
      Tq.h = 1.0;
      Tq.det = nullptr;
      for (;;) {
        const int o = step_steady<double, GradList, TallyPlain>(p, G, M, M.rec_relax, nullptr, C, key.x, key.y, Tq, gr);
        if (o != STEP_ALIVE) break;
        if ((p.e & 1023u) == 0u && globaltimer_ns() > deadline) {
          atomicOr(A.flags, 1);
          break;
        }
      }
      const double D = gr.mv.score(Xn, p.X);
      double* gs = grad_copy(A);
      atomicAdd(gs + 1, D);
      atomicAdd(gs + 2, D * D);
    }
  }
}
#endif  // MCBTE_F64

#if MCBTE_F32
// ------------------------------------------------------------------ FP32 persistent
// Per-thread book-keeping of finished particles (integer / fixed-point
// fields, few registers), flushed to the geometry's global accumulators when
// the thread moves to another geometry and at exit.
struct ThreadAcct {
  int g;
  unsigned traced, trunc, absorbed, maxev;
  int s_emit, s_abs;
  unsigned long long ev;
  long long sxq;      // sum of X in units of 2^-20 nm (exact)
  double sx2;

  __device__ __forceinline__ void reset(int gg) {
    g = gg;
    traced = trunc = absorbed = maxev = 0u;
    s_emit = s_abs = 0;
    ev = 0ull;
    sxq = 0;
    sx2 = 0.0;
  }
  __device__ __forceinline__ void flush(const Acc& A) const {
    if (g < 0 || traced == 0u) return;
    atomicAdd(&A.cnt[g * 4 + 0], ev);
    if (trunc) atomicAdd(&A.cnt[g * 4 + 1], (unsigned long long)trunc);
    atomicMax(&A.cnt[g * 4 + 2], (unsigned long long)maxev);
    atomicAdd(&A.cnt[g * 4 + 3], (unsigned long long)traced);
    atomicAdd(&A.dsc[g * 8 + 0], (double)sxq * kFxInv);
    atomicAdd(&A.dsc[g * 8 + 1], sx2);
    atomicAdd(&A.dsc[g * 8 + 2], (double)s_emit);
    if (absorbed) {
      atomicAdd(&A.dsc[g * 8 + 3], (double)s_abs);
      atomicAdd(&A.dsc[g * 8 + 7], (double)absorbed);
    }
  }
};

// Gradient pass: the open period closes at the particle's end (X = X_f; a
// fused pass adds its listed periods' a X_f too), then the resampling and
// specularity terms and the directional values.
__device__ __forceinline__ void grad_finish_replay(GradReplay& gr, double X, int g, const RunCfg& C, const Acc& A) {
  gr.finish(X);
  const double Rv = gr.resample_term(X);
  double* gs = grad_copy(A);
  atomicAdd(gs + 0, Rv);
  if (!C.mvd) {   // the measure-valued score is added after the phantom trace
    const double gp = gr.spec_term(X);
    atomicAdd(gs + 1, gp);
    atomicAdd(gs + 2, gp * gp);
  }
  for (int kd = 0; kd < C.n_dirs; ++kd) {
    const double val = gr.dv[kd] + Rv * C.dpi[kd];
    atomicAdd(gs + 4 + 2 * kd, val);
    atomicAdd(gs + 5 + 2 * kd, val * val);
  }
}

// A particle the main FP32 kernel hands to the tail kernel: the state the
// FP32 steady step carries (v, 1/v and Lambda are the bin's, reloaded), its
// index in the run and, in the gradient pass, the gradient bookkeeping.  Only
// these fields are stored, so parking keeps nothing else alive in the loop.
struct ParkRec {
  int4 snap[4];   // gradient pass: the pore-hit snapshot (snap_ok)
  float x[3], u[3], d_rel, d2, s;
  int bin, n_relax, g;
  uint32_t e, pid;
  long long Xq, Xqper;
  uint64_t idx;
  // gradient pass
  double Xf, sum_x_res;
  float a, d, pa, pd;
  int bin_cur, n_res;
  uint32_t mK, mKn, msel;
  int mflags;   // bit 0 sel_spec, bit 1 phase
  double dv[kMaxDirs];
  int np;       // fused gradient pass: the listed periods
  int lb[kFusedPeriods];
  float la[kFusedPeriods];
  int snap_ok;
};

template <bool GRAD, class GradT>
__device__ __forceinline__ void park_store(ParkRec* r, const Particle<float>& p, uint64_t idx, const GradT& gr,
                                           int n_dirs) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    r->x[a] = p.x[a];
    r->u[a] = p.u[a];
  }
  r->d_rel = p.d_rel;
  r->d2 = p.d2;
  r->s = p.s;
  r->bin = p.bin;
  r->n_relax = p.n_relax;
  r->g = p.g;
  r->e = p.e;
  r->pid = p.pid;
  r->Xq = p.Xq;
  r->Xqper = p.Xqper;
  r->idx = idx;
  if constexpr (GRAD) {
    r->Xf = gr.Xf;
    r->sum_x_res = gr.sum_x_res;
    r->a = gr.a;
    r->d = gr.d;
    r->pa = gr.pa;
    r->pd = gr.pd;
    r->bin_cur = gr.bin_cur;
    r->n_res = gr.n_res;
    r->mK = gr.mv.K;
    r->mKn = gr.mv.Kn;
    r->msel = gr.mv.sel;
    r->mflags = (gr.mv.sel_spec ? 1 : 0) | (gr.mv.phase ? 2 : 0);
    for (int k = 0; k < n_dirs; ++k) r->dv[k] = gr.dv[k];
    r->np = gr.np;
    for (int k = 0; k < gr.np; ++k) {
      r->lb[k] = gr.lb[k];
      r->la[k] = gr.la[k];
    }
    r->snap_ok = gr.snap_ok ? 1 : 0;
    if (gr.snap_ok) {
#pragma unroll
      for (int k = 0; k < 4; ++k) r->snap[k] = gr.snap[k];
    }
  }
}

template <bool GRAD, class GradT>
__device__ __forceinline__ void park_load(const ParkRec* r, Particle<float>& p, uint64_t& idx, GradT& gr, int n_dirs,
                                          const MatView& M, const float4* binf) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    p.x[a] = r->x[a];
    p.u[a] = r->u[a];
  }
  p.d_rel = r->d_rel;
  p.d2 = r->d2;
  p.s = r->s;
  p.bin = r->bin;
  p.n_relax = r->n_relax;
  p.g = r->g;
  p.e = r->e;
  p.pid = r->pid;
  p.Xq = r->Xq;
  p.Xqper = r->Xqper;
  idx = r->idx;
  load_bin(p, M, binf);
  if constexpr (GRAD) {
    gr.Xf = r->Xf;
    gr.sum_x_res = r->sum_x_res;
    gr.a = r->a;
    gr.d = r->d;
    gr.pa = r->pa;
    gr.pd = r->pd;
    gr.bin_cur = r->bin_cur;
    gr.n_res = r->n_res;
    gr.mv.K = r->mK;
    gr.mv.Kn = r->mKn;
    gr.mv.sel = r->msel;
    gr.mv.sel_spec = (r->mflags & 1) != 0;
    gr.mv.phase = (r->mflags & 2) != 0;
    for (int k = 0; k < n_dirs; ++k) gr.dv[k] = r->dv[k];
    gr.np = r->np;
    for (int k = 0; k < gr.np; ++k) {
      gr.lb[k] = r->lb[k];
      gr.la[k] = r->la[k];
    }
    // without a snapshot here the phantom trace starts from the emission
    gr.snap_ok = r->snap_ok != 0 && gr.snap != nullptr;
    if (gr.snap_ok) {
#pragma unroll
      for (int k = 0; k < 4; ++k) gr.snap[k] = r->snap[k];
    }
  }
}

// The tail kernel's events of one live particle from its precomputed draws:
// slot0 holds the draws of event p.e + 1, and the slots end with event
// e_last.  A flight that ends on a periodic face draws nothing, so it is
// handled here without the event dispatch (the same operations as
// apply_event's periodic branch: ++e, the clocks run down, the particle moves
// to the opposite face).  Without the extended physics the box and the pore
// are read once into registers (GeoLean: the per-event geometry then costs no
// load on the particle's dependent chain) and a flight that ends on a box
// face takes apply_event's FP32 face branch here, from the register copy;
// relaxations, pore hits and, with the extended physics, every non-periodic
// event go through apply_event with their slot.  Returns at the particle's
// end, or ALIVE once the slots are used up.
template <class Grad, class Tally, bool EXT>
__device__ __forceinline__ int trace_slots(Particle<float>& p, const GeoRun& g, const MatView& M, const uint4* relax_tab,
                                           const float4* binf, const RunCfg& C, uint32_t k0, uint32_t k1,
                                           const Tally& T, Grad& gr, const Draw32* slot0, uint32_t e_last,
                                           uint64_t deadline, int* flags) {
  const uint32_t e0 = p.e;
  GeoLean gl;
  if constexpr (!EXT) gl.load(g);
  for (;;) {
    if (p.e + 1u >= C.max_events) return STEP_TRUNCATED;
    float db;
    int face;
    if constexpr (EXT) first_hit<float, EXT>(g, p.x, p.u, &db, &face);
    else hit_box_pore_f32(gl, p.x, p.u, &db, &face);
    const bool relax = EXT ? (p.d_rel < db && p.d_rel <= p.d2) : p.d_rel < db;
    const bool relax2 = EXT && !relax && p.d2 < db;
    const float seg = relax ? p.d_rel : (relax2 ? p.d2 : db);
    double Xb = 0.0;
    if (Grad::on) Xb = T.X(p);
    const auto c = T.segment(p, seg);
    if constexpr (EXT) {
      if (C.n_regs > 0 && T.has_det()) region_steady<float>(p, seg, C, T);
    }
    if (Grad::on) gr.flight(relax, (double)Num<float>::div(seg, p.lam), Xb, c);
#pragma unroll
    for (int a = 0; a < 3; ++a) p.x[a] = p.x[a] + seg * p.u[a];
    const bool box = !relax && !relax2 && face < 6;
    const int ty = box ? (EXT ? g.type[face] : gl.type(face)) : -1;
    int out = STEP_ALIVE;
    if (ty == MCBTE_FACE_PERIODIC) {
      ++p.e;
      p.d_rel = p.d_rel - seg;
      if constexpr (EXT) p.d2 = p.d2 - seg;
      const int a = face_axis(face);
      put3<float>(p.x, a, face_is_max(face) ? 0.0f : (EXT ? geo_L<float>(g, a) : gl.L(a)));
    } else if (!EXT && box) {
      // apply_event's FP32 face branch (isothermal: absorbed; adiabatic:
      // specular or Lambertian by the slot's draws, then a select)
      ++p.e;
      p.d_rel = p.d_rel - seg;
      const int a = face_axis(face);
      const int mx = face_is_max(face);
      put3<float>(p.x, a, mx ? gl.L(a) : 0.0f);
      if (ty == MCBTE_FACE_ISOTHERMAL) return STEP_ABSORBED;
      const Draw32& d = slot0[p.e - 1u - e0];
      const bool spec_f = (uint64_t)d.wx < g.pthr[face];
      float ud[3];
      put3_cyclic<float>(ud, a, mx ? -d.lam[0] : d.lam[0], d.lam[1], d.lam[2]);
      const float flip = -sel3(p.u, a);
#pragma unroll
      for (int b = 0; b < 3; ++b) p.u[b] = spec_f ? (b == a ? flip : p.u[b]) : ud[b];
    } else {
      out = apply_event<float, Grad, Tally, EXT, DrawSlot>(p, g, M, relax_tab, binf, C, k0, k1, relax, relax2, face,
                                                           seg, T, gr, Grad::on ? T.X(p) : 0.0,
                                                           DrawSlot{slot0 + (p.e - e0)});
      if (out != STEP_ALIVE) return out;
    }
    if ((p.e & 255u) == 0u && globaltimer_ns() > deadline) {
      atomicOr(flags, 1);
      return STEP_TRUNCATED;
    }
    if (p.e >= e_last) return STEP_ALIVE;
  }
}

// The tail loop of a particle whose flights run through unfolded periodic
// axes (forward run without cell tallies or extended physics; a box with no
// pore and no walls): trace_slots with step_steady's unfolded flight.  The
// crossings advance the event number, so the event that ends a flight may
// lie past the slots and then takes its draws inline (the same bits).
template <class Tally>
__device__ __forceinline__ int trace_unfolded(Particle<float>& p, const GeoRun& g, const MatView& M,
                                              const uint4* relax_tab, const float4* binf, const RunCfg& C, uint32_t k0,
                                              uint32_t k1, const Tally& T, const Draw32* slot0, uint32_t e_last,
                                              uint64_t deadline, int* flags, unsigned um) {
  const uint32_t e0 = p.e;
  const uint32_t nslots = e_last - e0;
  GeoLean gl;
  gl.load(g);
  GradOff off;
  for (;;) {
    if (p.e + 1u >= C.max_events) return STEP_TRUNCATED;
    float db;
    int face;
    hit_box_pore_f32(gl, p.x, p.u, &db, &face, um);
    const bool relax = p.d_rel < db;
    const float seg = relax ? p.d_rel : db;
    T.segment(p, seg);
#pragma unroll
    for (int a = 0; a < 3; ++a) p.x[a] = p.x[a] + seg * p.u[a];
    const uint32_t n = fold_periodic(p.x, gl.Lf, um);
    if (n >= C.max_events - 1u - p.e) {
      p.e = C.max_events - 1u;
      return STEP_TRUNCATED;
    }
    p.e += n;
    const uint32_t si = p.e - e0;
    const Draw32* slot = si < nslots ? slot0 + si : nullptr;
    if (!relax && face < 6) {
      // apply_event's FP32 face branch (every periodic axis is unfolded, so
      // the face is isothermal: absorbed, or adiabatic: specular or
      // Lambertian by the event's draws, then a select)
      ++p.e;
      p.d_rel = p.d_rel - seg;
      const int a = face_axis(face);
      const int mx = face_is_max(face);
      put3<float>(p.x, a, mx ? gl.L(a) : 0.0f);
      if (gl.type(face) == MCBTE_FACE_ISOTHERMAL) return STEP_ABSORBED;
      const Draw32 d = DrawSlotOr{slot}.sub0(make_uint4(p.pid, (uint32_t)p.g, p.e, 0u), k0, k1, relax_tab, M.n);
      const bool spec_f = (uint64_t)d.wx < g.pthr[face];
      float ud[3];
      put3_cyclic<float>(ud, a, mx ? -d.lam[0] : d.lam[0], d.lam[1], d.lam[2]);
      const float flip = -sel3(p.u, a);
#pragma unroll
      for (int b = 0; b < 3; ++b) p.u[b] = spec_f ? (b == a ? flip : p.u[b]) : ud[b];
    } else {
      const int out = apply_event<float, GradOff, Tally, false, DrawSlotOr>(p, g, M, relax_tab, binf, C, k0, k1,
                                                                            relax, false, face, seg, T, off, 0.0,
                                                                            DrawSlotOr{slot});
      if (out != STEP_ALIVE) return out;
    }
    if ((p.e & 255u) == 0u && globaltimer_ns() > deadline) {
      atomicOr(flags, 1);
      return STEP_TRUNCATED;
    }
    if (p.e >= e_last) return STEP_ALIVE;
  }
}

// trace_unfolded for a box whose only faces left are the pair across axis W
// (the other two axes unfolded: a film): the flight's first hit is that
// pair's, and the pair's types and specular thresholds sit in registers.
// The same operations as hit_box_pore_f32 with those axes skipped and as
// apply_event's face branch, hence the same bits as step_steady.
template <int W, class Tally>
__device__ __forceinline__ int trace_film(Particle<float>& p, const GeoRun& g, const MatView& M,
                                          const uint4* relax_tab, const float4* binf, const RunCfg& C, uint32_t k0,
                                          uint32_t k1, const Tally& T, const Draw32* slot0, uint32_t e_last,
                                          uint64_t deadline, int* flags, unsigned um) {
  const uint32_t e0 = p.e;
  const uint32_t nslots = e_last - e0;
  float Lf[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) Lf[a] = g.Lf[a];
  const int f_lo = axis_min_face(W), f_hi = axis_max_face(W);
  const bool iso_lo = g.type[f_lo] == MCBTE_FACE_ISOTHERMAL, iso_hi = g.type[f_hi] == MCBTE_FACE_ISOTHERMAL;
  const uint64_t th_lo = g.pthr[f_lo], th_hi = g.pthr[f_hi];
  GradOff off;
  for (;;) {
    if (p.e + 1u >= C.max_events) return STEP_TRUNCATED;
    const float uw = p.u[W];
    const bool up = uw > 0.0f;
    const bool ok = uw != 0.0f;
    const float d0 = Num<float>::div((up ? Lf[W] : 0.0f) - p.x[W], uw);
    const float db = ok ? (d0 < 0.0f ? 0.0f : d0) : Num<float>::big();
    const bool relax = p.d_rel < db;
    const float seg = relax ? p.d_rel : db;
    T.segment(p, seg);
#pragma unroll
    for (int a = 0; a < 3; ++a) p.x[a] = p.x[a] + seg * p.u[a];
    const uint32_t n = fold_periodic(p.x, Lf, um);
    if (n >= C.max_events - 1u - p.e) {
      p.e = C.max_events - 1u;
      return STEP_TRUNCATED;
    }
    p.e += n;
    const uint32_t si = p.e - e0;
    const Draw32* slot = si < nslots ? slot0 + si : nullptr;
    if (!relax && ok) {
      // a wall of the pair
      ++p.e;
      p.d_rel = p.d_rel - seg;
      p.x[W] = up ? Lf[W] : 0.0f;
      if (up ? iso_hi : iso_lo) return STEP_ABSORBED;
      const Draw32 d = DrawSlotOr{slot}.sub0(make_uint4(p.pid, (uint32_t)p.g, p.e, 0u), k0, k1, relax_tab, M.n);
      const bool spec_f = (uint64_t)d.wx < (up ? th_hi : th_lo);
      float ud[3];
      put3_cyclic<float>(ud, W, up ? -d.lam[0] : d.lam[0], d.lam[1], d.lam[2]);
      const float flip = -p.u[W];
#pragma unroll
      for (int b = 0; b < 3; ++b) p.u[b] = spec_f ? (b == W ? flip : p.u[b]) : ud[b];
    } else {
      const int out = apply_event<float, GradOff, Tally, false, DrawSlotOr>(p, g, M, relax_tab, binf, C, k0, k1,
                                                                            relax, false, ok ? (up ? f_hi : f_lo) : 7,
                                                                            seg, T, off, 0.0, DrawSlotOr{slot});
      if (out != STEP_ALIVE) return out;
    }
    if ((p.e & 255u) == 0u && globaltimer_ns() > deadline) {
      atomicOr(flags, 1);
      return STEP_TRUNCATED;
    }
    if (p.e >= e_last) return STEP_ALIVE;
  }
}

// Every lane owns one particle at a time.  When its particle terminates the
// lane refills from its warp's run of particle indices (WarpRun: a ballot of
// the empty lanes, which take consecutive indices of the run; the run is
// refilled from the global work counter a chunk at a time, one atomic per
// chunk).  Lanes therefore never idle while work remains, whatever the
// event-count spread between particles.
// TPB is the block size the kernel is compiled for (register budget).
// GRAD: the gradient pass.  Fused (C.fused): the forward run's tallies,
// counters and per-particle outputs and the gradient in one pass, each
// particle listing its periods until its final tally is known.  Otherwise
// the replay of the forward pass's particles with their final tallies read
// from A.X_pp: it writes the gradient accumulators only, and flags (bit 2)
// any particle whose replayed tally differs.  With the measure-valued
// d/dp_pore the lane then traces the same particle once more (phantom
// phase, the chosen pore hit flipped, resumed from the lane's snapshot of
// that hit where it has one) before it refills.
// UNF (no cell tallies, no extended physics, no gradient): flights run
// through the periodic faces of a box without pore or walls (step_steady).
// CELLS: 0 no cell tallies, 1 T and three flux components, 2 T and the
// tally-axis flux only.
//
// MODE 0: the main kernel of a run without the tail kernel.  The run's tail
// (MODE 1 and 2): once the work counter has run out, a warp of the main
// kernel (MODE 1) with at most C.tail_max particles in flight parks them
// (ParkRec, A.park) and retires, so no warp idles most of its lanes for the
// rest of the run.  The tail kernel (MODE 2, launched next on the same
// stream) takes the parked particles instead of emitting new ones; once none
// is left, a warp with at most C.tail_max particles in flight computes the
// draws of their next events on all 32 lanes at once (one Draw32 per lane,
// the warp's 32 slots shared out over its live particles, 32 / 2^ceil(log2
// live) events each) and every live lane traces that many events reading its
// slots (DrawSlot), so its dependent chain per event holds the geometry and
// the tallies only.  The draws are the inline path's, the parked state is
// resumed as it was: trajectories and tallies are bit for bit those of a
// single kernel.
template <int CELLS, bool GRAD, int TPB, bool EXT, int MODE>
__global__ void __launch_bounds__(TPB, 1) k_steady_f32(const GeoRun* __restrict__ geos,
                                                       const uint64_t* __restrict__ offs, MatView M, RunCfg C,
                                                       Acc A, SmemPlan S) {
  constexpr bool TK = MODE == 2;
  // flights through the unfolded periodic axes (step_steady)
  constexpr bool UNF = CELLS == 0 && !GRAD && !EXT;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* sp = smem;
  const int n = M.n;
  const int nc = C.n_cells;
  const uint4* relax = M.rec_relax;
  const float4* binf = M.binf;
  long long* s_qbin = nullptr;
  long long* s_cP = nullptr;
  long long* s_cD = nullptr;
  // the tail kernel's per-warp draw slots come first (16-byte aligned), 32 per warp
  Draw32* slots = nullptr;
  if (TK && S.tail_slots) {
    slots = reinterpret_cast<Draw32*>(sp) + (threadIdx.x & ~31u);
    sp += (size_t)TPB * sizeof(Draw32);
  }
  // then the pore-hit snapshots (16-byte aligned), four int4 per thread
  int4* snaps = nullptr;
  if (S.snap_in_smem) {
    snaps = reinterpret_cast<int4*>(sp) + (size_t)threadIdx.x * 4;
    sp += (size_t)TPB * 4 * sizeof(int4);
  }
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
    s_qbin = reinterpret_cast<long long*>(sp);
    for (int i = threadIdx.x; i < n; i += blockDim.x) s_qbin[i] = 0;
    sp += (size_t)n * sizeof(long long);
  }
  long long* s_grad = nullptr;
  if (S.grad_in_smem) {
    s_grad = reinterpret_cast<long long*>(sp);
    for (int i = threadIdx.x; i < n; i += blockDim.x) s_grad[i] = 0;
    sp += (size_t)n * sizeof(long long);
  }
  if (S.cells_in_smem) {
    s_cP = reinterpret_cast<long long*>(sp);
    s_cD = s_cP + (size_t)nc * 4;
    for (int i = threadIdx.x; i < nc * 4 + (nc + 1) * 4; i += blockDim.x) s_cP[i] = 0;
  }
  __syncthreads();

  const unsigned lane = threadIdx.x & 31u;
  const uint64_t deadline = *C.t0 + C.budget_ns;
  Particle<float> p;
  using GradT = typename GradPick<GRAD, GradReplay>::type;
  GradT gr;
  double gr_dv[GRAD ? kMaxDirs : 1];
  int gr_lb[GRAD ? kFusedPeriods : 1];
  float gr_la[GRAD ? kFusedPeriods : 1];
  if constexpr (GRAD) {
    gr.dv = gr_dv;
    gr.lb = gr_lb;
    gr.la = gr_la;
    gr.snap = snaps;
    gr.G = S.grad_in_smem ? s_grad : A.Gq;
    gr.fused = C.fused != 0;
    gr.n_dirs = C.n_dirs;
    gr.n_bins = n;
    gr.dirs = C.dirs;
    gr.mvd = C.mvd != 0;
  }
  ThreadAcct acct;
  acct.reset(-1);
  TallyFxT<CELLS == 2 ? 2 : 4> T;
  T.nc = nc;
  T.ca = C.cell_axis;
  T.ta = C.tally_axis;
  T.cP = T.cD = T.qb = nullptr;
  T.h = T.inv_h = 1.0f;
  T.det = (C.n_regs > 0 && !GRAD) ? A.det_q : nullptr;
  // the per-bin flux of the particle's geometry (a gradient pass tallies
  // only when fused, and never in a phantom trace)
  auto qbin_of = [&](int g) -> long long* {
    if (!C.per_bin || (GRAD && !C.fused)) return nullptr;
    return S.qbin_in_smem ? s_qbin : A.qbinq + (size_t)g * n;
  };
  bool alive = false;
  bool drained = false;   // no work left for this lane: it idles in the loop until its warp is drained
  uint64_t idx = 0;
  const GeoRun* G = geos;
  const uint2 key = run_key(C);
  const int refill_min = (C.refill_min > 1 && !TK) ? C.refill_min : 1;
  // the tail: parking (main kernel) or the draws ahead (tail kernel)
  const int tail_max = (TK ? (slots != nullptr && n <= kOneBlockBins) : (MODE == 1 && A.park_cap > 0)) ? C.tail_max : 0;
  const uint64_t n_parked = TK ? min(*(volatile unsigned long long*)A.park_n, (unsigned long long)A.park_cap) : 0;
  bool pool_dry = false;   // the same in every lane: nothing left to hand out
  WarpRun run;              // main kernel: the warp's particle indices not yet handed out
  // the tallies of the lane's geometry
  auto bind = [&](int g) {
    if (g != acct.g) {
      acct.flush(A);
      acct.reset(g);
    }
    G = &geos[g];
    if (CELLS) {
      T.cP = S.cells_in_smem ? s_cP : A.cellPq + (size_t)g * nc * 4;
      T.cD = S.cells_in_smem ? s_cD : A.cellDq + (size_t)g * (nc + 1) * 4;
      T.h = G->Lf[C.cell_axis] / (float)nc;
      T.inv_h = (float)nc / G->Lf[C.cell_axis];
    }
    T.qb = qbin_of(g);
  };
  // All 32 lanes stay in the loop until every lane of the warp is drained, so
  // the warp-wide votes below reconverge the warp at every event step.
  constexpr unsigned kAll = 0xffffffffu;
  for (;;) {
    // two votes per step: the drained lanes and the busy ones
    const unsigned dry = __ballot_sync(kAll, drained);
    if (dry == kAll) break;
    const unsigned live = __ballot_sync(kAll, alive);
    const int nlive = __popc(live);
    int out = STEP_ALIVE;
    if (MODE != 0 && pool_dry && nlive > 0 && nlive <= tail_max) {
      if constexpr (MODE == 1) {
        // park the warp's last particles for the tail kernel
        const int leader = __ffs(live) - 1;
        unsigned long long base = 0;
        if ((int)lane == leader) base = atomicAdd(A.park_n, (unsigned long long)nlive);
        base = __shfl_sync(kAll, base, leader);
        if (alive) {
          const unsigned long long slot = base + (unsigned long long)__popc(live & ((1u << lane) - 1u));
          if (slot < A.park_cap) {
            park_store<GRAD>(reinterpret_cast<ParkRec*>(A.park + slot * A.park_stride), p, idx, gr, C.n_dirs);
            alive = false;
            drained = true;
          }
        }
        continue;   // lanes the buffer could not take trace on with the next votes (park_cap reached)
      } else {
        // log2 of the slots per particle: 5 - ceil(log2(nlive)), so nlive << sh <= 32
        const int sh = 5 - (32 - __clz(nlive - 1));
        const int r = (int)(lane >> sh);                                        // the live particle this lane draws for
        unsigned mm = live;
        for (int i = 0; i < r && mm; ++i) mm &= mm - 1u;
        const int owner = mm ? __ffs(mm) - 1 : 0;
        const uint32_t e_o = __shfl_sync(kAll, p.e, owner);
        const uint32_t pid_o = __shfl_sync(kAll, p.pid, owner);
        const int g_o = __shfl_sync(kAll, p.g, owner);
        if (r < nlive) {
          Draw32 d;
          uint4 ctr = make_uint4(pid_o, (uint32_t)g_o, e_o + 1u + (lane & ((1u << sh) - 1u)), 0u);
          draw_words(d, philox(ctr, key.x, key.y), relax, n);
          d.E2 = 0.0f;
          d.mv_lo = d.mv_hi = 0u;
          if (EXT && M.imp) {
            ctr.w = 256u;
            d.E2 = draw_e2(philox(ctr, key.x, key.y));
          }
          if (GRAD && C.mvd) {
            ctr.w = 257u;
            const uint4 w7 = philox(ctr, key.x, key.y);
            d.mv_lo = w7.x;
            d.mv_hi = w7.y;
          }
          slots[lane] = d;
        }
        __syncwarp();
        if (alive) {
          const Draw32* s0 = slots + (__popc(live & ((1u << lane) - 1u)) << sh);
          const unsigned um = UNF ? unfold_mask<GradT>(*G, C) : 0u;
          const uint32_t e_l = p.e + (1u << sh);
          if (UNF && um == 3u)
            out = trace_film<2>(p, *G, M, relax, binf, C, key.x, key.y, T, s0, e_l, deadline, A.flags, um);
          else if (UNF && um == 5u)
            out = trace_film<1>(p, *G, M, relax, binf, C, key.x, key.y, T, s0, e_l, deadline, A.flags, um);
          else if (UNF && um == 6u)
            out = trace_film<0>(p, *G, M, relax, binf, C, key.x, key.y, T, s0, e_l, deadline, A.flags, um);
          else if (UNF && um)
            out = trace_unfolded(p, *G, M, relax, binf, C, key.x, key.y, T, s0, e_l, deadline, A.flags, um);
          else
            out = trace_slots<GradT, decltype(T), EXT>(p, *G, M, relax, binf, C, key.x, key.y, T, gr, s0,
                                                        p.e + (1u << sh), deadline, A.flags);
        }
        __syncwarp();   // the slots are rewritten in the next round
      }
    } else {
      const unsigned need = ~(dry | live);
      // refill once enough lanes are idle (or no lane is busy)
      if (need && !pool_dry && (__popc(need) >= refill_min || live == 0u)) {
        const unsigned cnt = __popc(need);
        const unsigned rank = __popc(need & ((1u << lane) - 1u));
        uint64_t k;
        uint64_t avail;
        if constexpr (TK) {
          const int leader = __ffs(need) - 1;
          unsigned long long base = 0;
          if ((int)lane == leader) base = atomicAdd(A.park_rd, (unsigned long long)cnt);
          base = __shfl_sync(kAll, base, leader);
          avail = n_parked;
          if (base + cnt >= avail) pool_dry = true;
          k = base + rank;
        } else {
          k = run.take(need, lane, A.work, C.total, C.take_chunk, deadline, A.flags);
          avail = C.total;
          if (run.empty()) pool_dry = true;
        }
        if (!alive && !drained) {
          if (k >= avail || (*(volatile int*)A.flags & 1)) {
            drained = true;
            continue;
          }
          if constexpr (TK) {
            // a parked particle, exactly as the main kernel left it
            park_load<GRAD>(reinterpret_cast<const ParkRec*>(A.park + k * A.park_stride), p, idx, gr, C.n_dirs, M,
                            binf);
            bind(p.g);
            if constexpr (GRAD) {
              if (gr.mv.phase) T.qb = nullptr;   // a phantom trace tallies only its own X
            }
          } else {
            idx = k;
            const int g = find_geom(offs, C.n_geoms, idx);
            bind(g);
            p.pid = (uint32_t)(idx - offs[g] + G->pid0);
            p.g = g;
            emit<float, EXT>(p, *G, M, M.rec_emit, M.rec_init, binf, key.x, key.y, false, 0.0f);
            if constexpr (GRAD) {
              gr.init(p.bin);
              if (!C.fused) gr.Xf = A.X_pp[idx];
            }
          }
          alive = true;
        }
      }
      if (!alive) {
        drained = drained || pool_dry;   // nothing left to hand out
        continue;
      }
      out = step_steady<float, GradT, decltype(T), EXT, DrawInline, UNF>(p, *G, M, relax, binf, C, key.x, key.y, T,
                                                                          gr);
      if (out == STEP_ALIVE && (p.e & 255u) == 0u && globaltimer_ns() > deadline) {
        atomicOr(A.flags, 1);
        out = STEP_TRUNCATED;
      }
    }
    if (!alive || out == STEP_ALIVE) continue;
    // the forward run's part of a finished (nominal) trace: the last period's
    // per-bin flux, the run's counters and sums, the per-particle outputs
    auto account = [&](double X) {
      T.period_end(p);
      const unsigned nev = p.e + 1u;
      acct.ev += nev;
      acct.trunc += (out == STEP_TRUNCATED) ? 1u : 0u;
      acct.maxev = nev > acct.maxev ? nev : acct.maxev;
      acct.traced += 1u;
      acct.sxq += p.Xq;
      acct.sx2 += X * X;
      const int sgn = p.s > 0.0f ? 1 : -1;
      acct.s_emit += sgn;
      if (out == STEP_ABSORBED) {
        acct.s_abs += sgn;
        acct.absorbed += 1u;
      }
      if (A.events_pp) A.events_pp[idx] = nev;
      if (A.X_pp) A.X_pp[idx] = X;
      if constexpr (EXT) nscat_end(C, p.g, p.n_relax, X);
    };
    if (GRAD) {
      const double X = T.X(p);
      if constexpr (GRAD) {
        if (!gr.mv.phase) {
          if (C.fused) account(X);
          else if (X != gr.Xf) atomicOr(A.flags, 4);
          grad_finish_replay(gr, X, p.g, C, A);
          if (C.mvd && gr.mv.sel > 0u) {
            // measure-valued d/dp_pore: the same particle again from its
            // emission, the chosen pore hit's branch flipped (Xf keeps the
            // nominal tally; the phantom tallies only its own X)
            gr.Xf = X;
            gr.mv.start_phantom();
            T.qb = nullptr;
            if (gr.snap_ok) {
              // resume at the chosen hit (the state the trace from the
              // emission would reach) and apply it with its branch flipped
              gr.restore(p);
              load_bin(p, M, binf);
              gr.mv.K = gr.mv.sel - 1u;
              apply_event<float, GradT, decltype(T), EXT>(p, *G, M, relax, binf, C, key.x, key.y, false, false, 6,
                                                          0.0f, T, gr, T.X(p));
            } else {
              emit<float, EXT>(p, *G, M, M.rec_emit, M.rec_init, binf, key.x, key.y, false, 0.0f);
            }
            continue;
          }
        } else {
          const double D = gr.mv.score(gr.Xf, X);
          double* gs = grad_copy(A);
          atomicAdd(gs + 1, D);
          atomicAdd(gs + 2, D * D);
        }
      }
    } else {
      account(T.X(p));
    }
    alive = false;
    drained = pool_dry;
  }
  if (!GRAD || C.fused) acct.flush(A);
  __syncthreads();
  if (S.qbin_in_smem) {
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (s_qbin[i] != 0) atomicAdd(reinterpret_cast<unsigned long long*>(&A.qbinq[i]), (unsigned long long)s_qbin[i]);
  }
  if (S.grad_in_smem) {
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (s_grad[i] != 0) atomicAdd(reinterpret_cast<unsigned long long*>(&A.Gq[i]), (unsigned long long)s_grad[i]);
  }
  if (S.cells_in_smem) {
    for (int i = threadIdx.x; i < nc * 4; i += blockDim.x)
      if (s_cP[i] != 0) atomicAdd(reinterpret_cast<unsigned long long*>(&A.cellPq[i]), (unsigned long long)s_cP[i]);
    for (int i = threadIdx.x; i < (nc + 1) * 4; i += blockDim.x)
      if (s_cD[i] != 0) atomicAdd(reinterpret_cast<unsigned long long*>(&A.cellDq[i]), (unsigned long long)s_cD[i]);
  }
}
#endif  // MCBTE_F32

#if MCBTE_F64
// ------------------------------------------------------------------ finalise
// One block per geometry: scale the raw sums into the paper's estimators
// (Eqs. temp_steady, flux_x_steady), kappa = -q / (dT/dx) and its standard
// error from the per-particle X_p (iid), and the LR gradient.  FP64 and
// fixed-point accumulators are both read (only one kind is non-zero).
__global__ void k_finalize_steady(const GeoRun* geos, MatView M, RunCfg C, Acc A, SteadyOutDev O, int grad,
                                  const int* flags) {
  const int g = blockIdx.x;
  const GeoRun& G = geos[g];
  const int nc = C.n_cells;
  const int n = M.n;
  const double N = (double)G.n_norm;
  const double E_eff = G.E_tot / N;
  const double C_tot = M.sums[0];
  if (nc > 0 && threadIdx.x == 0) {
    const double Vc = G.V_box / (double)nc;
    const double kT = E_eff / (C_tot * Vc);
    const double kq = E_eff / Vc;
    double run[4] = {0.0, 0.0, 0.0, 0.0};
    const double* P = A.cellP + (size_t)g * nc * 4;
    const double* D = A.cellD + (size_t)g * (nc + 1) * 4;
    const long long* Pq = A.cellPq + (size_t)g * nc * 4;
    const long long* Dq = A.cellDq + (size_t)g * (nc + 1) * 4;
    long long runq[4] = {0, 0, 0, 0};
    for (int c = 0; c < nc; ++c) {
      double v[4];
      for (int b = 0; b < 4; ++b) {
        run[b] += D[c * 4 + b];
        runq[b] += Dq[c * 4 + b];
        v[b] = P[c * 4 + b] + run[b] + (double)(Pq[c * 4 + b] + runq[b]) * kFxInv;
      }
      if (O.T) O.T[(size_t)g * nc + c] = (kT * v[0]) * 1e-12;
      if (O.q)
        for (int b = 0; b < 3; ++b) O.q[((size_t)g * nc + c) * 3 + b] = (kq * v[1 + b]) * 1e-9;
    }
  }
  if (O.det && C.n_regs > 0) {
    // detector regions: volume-averaged T and q of each detector (and bin)
    const double C_tot_d = M.sums[0];
    const size_t nb = C.det_nb > 1 ? (size_t)C.det_nb : 1;
    for (size_t s = threadIdx.x; s < (size_t)C.n_det * nb; s += blockDim.x) {
      const uint32_t d = (uint32_t)(s / nb);
      double vd = C.regs[0].v_det;
      for (int k = 0; k < C.n_regs; ++k)
        if (d >= C.regs[k].off) vd = C.regs[k].v_det;
      const double kT = E_eff / (C_tot_d * vd);
      const double kq = E_eff / vd;
      double raw[4];
      for (int b = 0; b < 4; ++b) raw[b] = A.det_raw[s * 4 + b] + (double)A.det_q[s * 4 + b] * kFxInv;
      O.det[s * 4 + 0] = (kT * raw[0]) * 1e-12;
      for (int b = 1; b < 4; ++b) O.det[s * 4 + b] = (kq * raw[b]) * 1e-9;
    }
  }
  if (O.kn && C.nscat_acc) {
    // fold the copies of the curve sums into the first
    const size_t per = (size_t)(C.n_scat_max + 1) * 4;
    const size_t stride = (size_t)C.n_geoms * per;
    double* a0 = C.nscat_acc + (size_t)g * per;
    for (size_t i = threadIdx.x; i < per; i += blockDim.x) {
      double v = a0[i];
      for (int r = 1; r < C.nscat_rep; ++r) v += a0[(size_t)r * stride + i];
      a0[i] = v;
    }
    __syncthreads();
  }
  if (O.kn && C.nscat_acc && threadIdx.x == 0) {
    // kappa and its standard error for N_scat_max = k: the tally at the k-th
    // relaxation, or the final one of trajectories that ended before it
    const int K = C.n_scat_max;
    const double nt = (double)A.cnt[g * 4 + 3];
    const double* a = C.nscat_acc + (size_t)g * (size_t)(K + 1) * 4;
    double e1 = 0.0, e2 = 0.0;
    for (int k = 1; k <= K; ++k) {
      e1 += a[(size_t)k * 4 + 2];
      e2 += a[(size_t)k * 4 + 3];
      const double s1 = a[(size_t)k * 4 + 0] + e1;
      const double s2 = a[(size_t)k * 4 + 1] + e2;
      const double mean = s1 / nt;
      const double var = nt > 1.0 ? (s2 - nt * mean * mean) / (nt - 1.0) : 0.0;
      const double qm = (E_eff / G.V_solid) * s1 * 1e-9;
      const double qs = (E_eff / G.V_solid) * 1e-9 * sqrt(fmax(var, 0.0) * nt);
      O.kn[((size_t)g * K + (k - 1)) * 2 + 0] = -qm / G.kappa_grad;
      O.kn[((size_t)g * K + (k - 1)) * 2 + 1] = qs / fabs(G.kappa_grad);
    }
  }
  if (O.q_bin && C.per_bin) {
    const double kb = E_eff / G.V_solid;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const size_t j = (size_t)g * n + i;
      O.q_bin[j] = (kb * (A.qbin[j] + (double)A.qbinq[j] * kFxInv)) * 1e-9;
    }
  }
  if (threadIdx.x == 0) {
    const double sx = A.dsc[g * 8 + 0], sx2 = A.dsc[g * 8 + 1];
    const double nt = (double)A.cnt[g * 4 + 3];
    const double mean = sx / nt;
    const double var = nt > 1.0 ? (sx2 - nt * mean * mean) / (nt - 1.0) : 0.0;
    const double q_mean = (E_eff / G.V_solid) * sx * 1e-9;
    const double q_se = (E_eff / G.V_solid) * 1e-9 * sqrt(fmax(var, 0.0) * nt);
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
    st[MCBTE_STAT_STATUS] = (flags[0] & 4)   ? (double)MCBTE_ERR_REPLAY
                            : (flags[0] & 1) ? (double)MCBTE_ERR_TIMEOUT
                                             : (A.cnt[g * 4 + 1] ? (double)MCBTE_WARN_TRUNCATED : 0.0);
    st[MCBTE_STAT_N] = nt;
    st[MCBTE_STAT_ABSORBED] = A.dsc[g * 8 + 7];
  }
  if (grad && g == 0) {
    // fold the copies of the gradient sums into the first
    double* gs = A.gsum;
    for (int i = threadIdx.x; i < kGradStride; i += blockDim.x) {
      double v = gs[i];
      for (int r = 1; r < kSumCopies; ++r) v += gs[(size_t)r * kGradStride + i];
      gs[i] = v;
    }
    __syncthreads();
    const double scale = -(E_eff / G.V_solid) * 1e-9 / G.kappa_grad;
    const double Rs = gs[0];
    for (int i = threadIdx.x; i < n; i += blockDim.x) O.dk[i] = scale * ((A.G[i] + (double)A.Gq[i] * kFxInv) + Rs * M.pi[i]);
    if (threadIdx.x == 0) {
      const double nt = (double)A.cnt[3];
      const double gm = gs[1] / nt;
      const double gv = (gs[2] - nt * gm * gm) / fmax(nt - 1.0, 1.0);
      const bool ok = G.pore && (C.mvd || (G.p_pore > 0.0 && G.p_pore < 1.0));
      const double nan = __longlong_as_double(0x7ff8000000000000ll);
      O.dkp[0] = ok ? scale * gs[1] : nan;
      O.dkp[1] = ok ? fabs(scale) * sqrt(fmax(gv, 0.0) * nt) : nan;
      for (int k = 0; k < C.n_dirs; ++k) {
        const double dm = gs[4 + 2 * k] / nt;
        const double dv = (gs[5 + 2 * k] - nt * dm * dm) / fmax(nt - 1.0, 1.0);
        O.dkdir[k * 2 + 0] = scale * gs[4 + 2 * k];
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

template <bool CELLS, bool GRAD>
cudaError_t launch_f64(const GeoRun* geos, const uint64_t* offs, const MatView& M, const RunCfg& C, const Acc& A,
                       cudaStream_t s) {
  const uint64_t blocks = (C.total + 255) / 256;
  k_steady_fp64<CELLS, GRAD><<<(unsigned)blocks, 256, 0, s>>>(geos, offs, M, C, A);
  return cudaGetLastError();
}
#endif  // MCBTE_F64

#if MCBTE_F32
// One persistent launch: SMs x resident blocks (or fewer on request).
template <int CELLS, bool GRAD, int TPB, bool EXT, int MODE>
cudaError_t launch_f32_kernel(const GeoRun* geos, const uint64_t* offs, const MatView& M, const RunCfg& C,
                              const Acc& A, int bps, cudaStream_t s) {
  // the gradient kernel keeps no cell tallies, and the per-bin flux only in
  // a fused pass
  const SmemPlan S = plan_smem_f32(M.n, C.n_geoms, GRAD ? 0 : C.n_cells, (GRAD && !C.fused) ? 0 : C.per_bin,
                                   200 * 1024, MODE == 2 ? TPB : 0, GRAD ? 1 : 0, (GRAD && C.mvd) ? TPB : 0);
  auto kern = k_steady_f32<CELLS, GRAD, TPB, EXT, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.bytes);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TPB, S.bytes);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int b = (bps > 0 && bps < occ) ? bps : occ;
  kern<<<sm_count() * b, TPB, S.bytes, s>>>(geos, offs, M, C, A, S);
  return cudaGetLastError();
}

// Part 0: the main kernel alone.  Part 1: the main kernel that parks its
// tail, then the tail kernel over the parked particles (256-thread blocks).
#if MCBTE_F32_PART == 1
constexpr int kTailThreads = 256;
#endif

template <int CELLS, bool GRAD, int TPB, bool EXT>
cudaError_t launch_f32_tpb(const GeoRun* geos, const uint64_t* offs, const MatView& M, const RunCfg& C,
                           const Acc& A, int bps, cudaStream_t s) {
#if MCBTE_F32_PART == 0
  return launch_f32_kernel<CELLS, GRAD, TPB, EXT, 0>(geos, offs, M, C, A, bps, s);
#else
  cudaError_t e = launch_f32_kernel<CELLS, GRAD, TPB, EXT, 1>(geos, offs, M, C, A, bps, s);
  if (e != cudaSuccess) return e;
  return launch_f32_kernel<CELLS, GRAD, kTailThreads, EXT, 2>(geos, offs, M, C, A, 0, s);
#endif
}

template <int CELLS, bool GRAD, bool EXT>
cudaError_t launch_f32_ext(const GeoRun* geos, const uint64_t* offs, const MatView& M, const RunCfg& C, const Acc& A,
                           int threads, int bps, cudaStream_t s) {
  switch (threads) {
    case 256: return launch_f32_tpb<CELLS, GRAD, 256, EXT>(geos, offs, M, C, A, bps, s);
    case 512: return launch_f32_tpb<CELLS, GRAD, 512, EXT>(geos, offs, M, C, A, bps, s);
    case 768: return launch_f32_tpb<CELLS, GRAD, 768, EXT>(geos, offs, M, C, A, bps, s);
    case 1024: return launch_f32_tpb<CELLS, GRAD, 1024, EXT>(geos, offs, M, C, A, bps, s);
    default: return cudaErrorInvalidValue;
  }
}

// The extended physics is compiled in only for runs that use it.
template <int CELLS, bool GRAD>
cudaError_t launch_f32(const GeoRun* geos, const uint64_t* offs, const MatView& M, const RunCfg& C, const Acc& A,
                       int threads, int bps, cudaStream_t s) {
  return C.ext ? launch_f32_ext<CELLS, GRAD, true>(geos, offs, M, C, A, threads, bps, s)
               : launch_f32_ext<CELLS, GRAD, false>(geos, offs, M, C, A, threads, bps, s);
}

cudaError_t launch_f32_variants(bool grad, bool cells, const GeoRun* geos, const uint64_t* offs, const MatView& M,
                                const RunCfg& C, const Acc& A, int threads, int bps, cudaStream_t s) {
  // the gradient pass keeps no cell or per-bin tallies
  if (grad) return launch_f32<0, true>(geos, offs, M, C, A, threads, bps, s);
  if (!cells) return launch_f32<0, false>(geos, offs, M, C, A, threads, bps, s);
  return C.cell_flux_axis ? launch_f32<2, false>(geos, offs, M, C, A, threads, bps, s)
                          : launch_f32<1, false>(geos, offs, M, C, A, threads, bps, s);
}
#endif  // MCBTE_F32

}  // namespace

#if MCBTE_F64
SmemPlan plan_smem_f32(int n_bins, int n_geoms, int n_cells, int per_bin, size_t budget, int tail_threads,
                       int grad_acc, int snap_threads) {
  // By use per event: the relaxation alias records and the per-bin
  // constants (every relaxation), the cell tallies (every flight), the
  // per-bin flux (every relaxation period), the gradient accumulator (every
  // period of a gradient pass); each is placed while room remains, then the
  // tail's draw slots (one Draw32 per thread), then the pore-hit snapshots
  // of the measure-valued d/dp (64 bytes per thread).
  SmemPlan S{0, 0, 0, 0, 0, 0, 0, 0};
  size_t used = 0;
  if (used + (size_t)n_bins * 16 <= budget) {
    S.relax_in_smem = 1;
    used += (size_t)n_bins * 16;
  }
  if (used + (size_t)n_bins * 16 <= budget) {
    S.binf_in_smem = 1;
    used += (size_t)n_bins * 16;
  }
  const size_t cells = (size_t)(n_cells * 4 + (n_cells + 1) * 4) * sizeof(long long);
  if (n_cells > 0 && n_geoms == 1 && used + cells <= budget) {
    S.cells_in_smem = 1;
    used += cells;
  }
  if (per_bin && n_geoms == 1 && used + (size_t)n_bins * 8 <= budget) {
    S.qbin_in_smem = 1;
    used += (size_t)n_bins * 8;
  }
  if (grad_acc && used + (size_t)n_bins * 8 <= budget) {
    S.grad_in_smem = 1;
    used += (size_t)n_bins * 8;
  }
  if (tail_threads > 0 && n_bins <= kOneBlockBins && used + (size_t)tail_threads * sizeof(Draw32) <= budget) {
    S.tail_slots = 1;
    used += (size_t)tail_threads * sizeof(Draw32);
  }
  if (snap_threads > 0 && used + (size_t)snap_threads * 4 * sizeof(int4) <= budget) {
    S.snap_in_smem = 1;
    used += (size_t)snap_threads * 4 * sizeof(int4);
  }
  S.bytes = used;
  return S;
}

// SM count of the current device, cached per device ordinal (grids are sized
// for the device the launch goes to).
int sm_count() {
  constexpr int kDevices = 64;
  static std::atomic<int> cached[kDevices];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < kDevices) {
    const int c = cached[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  if (v < 1) v = 1;
  if (dev >= 0 && dev < kDevices) cached[dev].store(v, std::memory_order_relaxed);
  return v;
}

cudaError_t launch_steady(int precision, bool grad, const GeoRun* geos, const uint64_t* offs, const MatView& M,
                          const RunCfg& C, const Acc& A, int threads, int bps, cudaStream_t s) {
  const bool cells = C.n_cells > 0;
  if (precision == MCBTE_FP64_PLAIN) {
    if (grad) return cells ? launch_f64<true, true>(geos, offs, M, C, A, s) : launch_f64<false, true>(geos, offs, M, C, A, s);
    return cells ? launch_f64<true, false>(geos, offs, M, C, A, s) : launch_f64<false, false>(geos, offs, M, C, A, s);
  }
  // default block: 768 threads, 512 for the gradient (its estimator state
  // takes ~128 registers per thread)
  return launch_steady_f32(grad, cells, geos, offs, M, C, A, threads > 0 ? threads : (grad ? 512 : 768), bps, s);
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

#if MCBTE_F32 && MCBTE_F32_PART == 1
cudaError_t launch_steady_f32_tail(bool grad, bool cells, const GeoRun* geos, const uint64_t* offs, const MatView& M,
                                   const RunCfg& C, const Acc& A, int threads, int bps, cudaStream_t s) {
  return launch_f32_variants(grad, cells, geos, offs, M, C, A, threads, bps, s);
}
#endif

#if MCBTE_F32 && MCBTE_F32_PART == 0
size_t park_record_bytes() { return (sizeof(ParkRec) + 15) & ~(size_t)15; }

// Runs that can park their tail (a park buffer and a threshold) take the
// kernels of part 1, the others the plain main kernel.
cudaError_t launch_steady_f32(bool grad, bool cells, const GeoRun* geos, const uint64_t* offs, const MatView& M,
                              const RunCfg& C, const Acc& A, int threads, int bps, cudaStream_t s) {
  if (A.park_cap > 0 && C.tail_max > 0)
    return launch_steady_f32_tail(grad, cells, geos, offs, M, C, A, threads, bps, s);
  return launch_f32_variants(grad, cells, geos, offs, M, C, A, threads, bps, s);
}
#endif  // MCBTE_F32

}  // namespace mcbte
