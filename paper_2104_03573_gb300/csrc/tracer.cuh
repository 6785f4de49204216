// Particle emission and the event step of the deviational tracer, shared by
// the FP64 plain kernels and the FP32 persistent kernels.
//
// Event contract (identical for every precision; the random words are the
// same, only their real-valued maps differ in width):
//   counter = (particle id within its geometry, geometry index, event index, sub-block)
//   key     = (seed low, seed high)
//   emission (event 0): sub 0 {source, alias column, alias threshold lo, hi}
//                       sub 1 {direction mu, phi, flight -ln R lo, hi}
//                       sub 2 {body sign, emission time}
//                       sub 3+k {position attempt k; Gaussian: Box-Muller words}
//   relaxation event  : sub 0 {alias column, threshold lo, mu, phi}
//                       sub 1 {threshold hi, flight -ln R lo, hi}
//                       FP32 path with at most kOneBlockBins bins: sub 0 only,
//                       {alias column and its 32-bit test word, flight -ln R, mu, phi}
//   adiabatic / pore  : sub 0 {specular test, -, mu, phi}
//   isothermal / periodic walls draw nothing.
#pragma once

#include "mcbte_device.cuh"

namespace mcbte {

// Fixed-point unit of the FP32 path's tallies: 2^-20 nm (lengths) and
// 2^-20 ps (times).  64-bit integer sums are exact and independent of the
// order of the atomic adds.
constexpr float kFx = 1048576.0f;
constexpr double kFxInv = 9.5367431640625e-07;

struct RunCfg {
  uint32_t k0, k1;
  int n_scat_max;
  uint32_t max_events;
  int n_cells, cell_axis, tally_axis, per_bin;
  int n_geoms;
  uint64_t total;
  const unsigned long long* t0;   // device timestamp (ns) written by the setup kernel
  uint64_t budget_ns;             // wall-clock budget of the tracing kernel
  const unsigned long long* seed_dev;   // optional device-resident Philox key (overrides k0, k1)
  int refill_min;                 // FP32 tracer: refill a warp once this many lanes are idle
  // gradient
  int n_dirs;
  const double* dirs;    // [n_dirs][n_bins]
  const double* dpi;     // [n_dirs] dirs . pi
  // transient
  double t_max_ps;
  int n_times;
  const double* t_meas_ps;
  int grid[3];
  int cell_flux_axis;   // FP32 cell tallies: T and the tally-axis flux only
  int ext;              // extended physics in use (two-phonon clock, walls, per-bin d, general gradient)
  // transient detector regions (none: the whole box split by grid)
  const struct DetRegion* regs;
  int n_regs;
  uint32_t n_det;
  int time_average;     // bin averages over [t_{m-1}, t_m) instead of snapshots
  // FP32 transient time windows: this launch takes the snapshots with index
  // < win_end; the first window emits, later ones resume saved particles
  int win_first, win_last, win_end;
  int mvd;              // gradient: measure-valued d kappa / d p_pore (phantom traces)
  // N_scat_max convergence curve, or null: per geometry and k = 1..n_scat_max,
  // [0] sum of X at the k-th relaxation, [1] its square, [2] sum of the final
  // X of trajectories with exactly k - 1 relaxations, [3] its square; in
  // nscat_rep copies (a power of two), block b adding to copy b % nscat_rep
  double* nscat_acc;    // [nscat_rep][G][n_scat_max + 1][4]
  int nscat_rep;
  int det_nb;           // steady detector sums per detector (1) or per detector and bin (n_bins)
  int tail_max;         // FP32 steady tracer: the tail's draw slots serve warps with at most
                        // this many particles in flight once the work counter has run out (0: off)
  int fused;            // FP32 gradient: the forward tallies and the gradient in one pass
  // particle indices a warp takes from the work counter at once (WarpRun):
  // 1024 for a batch of geometries (a warp stays on one geometry longer),
  // 256 otherwise (a shorter drain); 0 counts as 32
  unsigned take_chunk;
};

// Transient detector region (Sec. 4.5): a closed axis-aligned cuboid split
// into n[0] x n[1] x n[2] detectors numbered from `off`, x fastest.
struct DetRegion {
  double lo[3], hi[3], h[3];   // nm; h = (hi - lo) / n
  float lof[3], hif[3], cinvf[3];
  int n[3];
  uint32_t off;
  double v_det;                // m^3 per detector
  int hi_closed[3];            // upper face on (or beyond) the box's upper face
};

// Time the path x(tau) = x0 + w (tau - t0) (w in nm/ps) spends in each
// detector of region r between ta < tb: the interval clipped to the region's
// box, then a cell-by-cell walk of the grid in time order (crossing times
// from the grid planes; ties advance every axis that crosses); at most
// nx + ny + nz + 3 steps.  add(detector index within the region, duration).
template <typename R, class Add>
__device__ __forceinline__ void region_track(const DetRegion& r, const R x0[3], const R w[3], R t0, R ta, R tb,
                                             Add add) {
  R lo[3], hi[3], h[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = sizeof(R) == 8 ? (R)r.lo[a] : (R)r.lof[a];
    hi[a] = sizeof(R) == 8 ? (R)r.hi[a] : (R)r.hif[a];
    h[a] = sizeof(R) == 8 ? (R)r.h[a] : (hi[a] - lo[a]) / (R)r.n[a];
  }
  R t_in = ta, t_out = tb;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R p = x0[a] + w[a] * (ta - t0);
    if (w[a] == R(0)) {
      if (!(p >= lo[a] && (p < hi[a] || (r.hi_closed[a] && p <= hi[a])))) return;
      continue;
    }
    R c0 = t0 + (lo[a] - x0[a]) / w[a];
    R c1 = t0 + (hi[a] - x0[a]) / w[a];
    if (c0 > c1) {
      const R tmp = c0;
      c0 = c1;
      c1 = tmp;
    }
    t_in = t_in > c0 ? t_in : c0;
    t_out = t_out < c1 ? t_out : c1;
  }
  if (!(t_in < t_out)) return;
  int i3[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R p = x0[a] + w[a] * (t_in - t0);
    int ia;
    if constexpr (sizeof(R) == 8) ia = (int)floor((p - lo[a]) / h[a]);
    else ia = (int)floorf((p - lo[a]) / h[a]);
    if (w[a] < R(0) && (R)ia * h[a] + lo[a] == p) ia = ia - 1;
    i3[a] = min(max(ia, 0), r.n[a] - 1);
  }
  R tau = t_in;
  const int max_steps = r.n[0] + r.n[1] + r.n[2] + 3;
  for (int step = 0; step < max_steps && tau < t_out; ++step) {
    R tn = t_out;
    R tc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      tc[a] = Num<R>::inf();
      if (w[a] > R(0)) tc[a] = t0 + ((lo[a] + (R)(i3[a] + 1) * h[a]) - x0[a]) / w[a];
      else if (w[a] < R(0)) tc[a] = t0 + ((lo[a] + (R)i3[a] * h[a]) - x0[a]) / w[a];
      if (tc[a] < tn) tn = tc[a];
    }
    if (tn < tau) tn = tau;
    add(((uint32_t)i3[2] * (uint32_t)r.n[1] + (uint32_t)i3[1]) * (uint32_t)r.n[0] + (uint32_t)i3[0], tn - tau);
    tau = tn;
    if (!(tau < t_out)) break;
    bool out_of = false;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (tc[a] <= tn) {
        i3[a] += w[a] > R(0) ? 1 : -1;
        if (i3[a] < 0 || i3[a] >= r.n[a]) out_of = true;
      }
    if (out_of) break;
  }
}

// Raw accumulators of a run (device).
// Sums that every particle adds to (the gradient sums, a transient run's
// counters) are kept in kSumCopies copies, block b adding to copy
// b % kSumCopies, so that those same-address atomics do not serialise in one
// L2 slice; the finalising kernel folds the copies.
constexpr int kSumCopies = 64;
// Gradient sums of one run (one geometry): [0] the resampling term R, [1] the
// d kappa / d p_pore score, [2] its square, [3] unused, [4 + 2k] the value
// along probe direction k, [5 + 2k] its square.
constexpr int kGradStride = 4 + 2 * kMaxDirs;

struct Acc {
  double* cellP;              // [G][nc][4]   per-cell direct / partial-cell sums (FP64 path)
  double* cellD;              // [G][nc+1][4] difference array of full-cell sums (FP64 path)
  double* qbin;               // [G][n_bins]  (FP64 path)
  long long* cellPq;          // [G][nc][4]   fixed-point counterparts (FP32 path)
  long long* cellDq;          // [G][nc+1][4]
  long long* qbinq;           // [G][n_bins]
  double* dsc;                // [G][8] (transient: [kSumCopies][8]): sumX, sumX2, signed emitted,
                              // signed absorbed, -, -, -, absorbed
  unsigned long long* cnt;    // [G][4] (transient: [kSumCopies][4]): events, truncated, max events, traced
  double* G;                  // [n_bins] sparse part of the LR gradient (FP64 path)
  long long* Gq;              // [n_bins] its fixed-point counterpart (FP32 gradient pass)
  double* gsum;               // [kSumCopies][kGradStride] gradient sums
  double* snap;               // [n_times][cells][4] transient
  uint4* tstate;              // [total][3] particle state between transient time windows, or null
  double* det_raw;            // [n_det][4] steady detector sums (FP64 path)
  long long* det_q;           // [n_det][4] the same in fixed point (FP32 path)
  uint32_t* events_pp;        // [total] or null
  double* X_pp;               // [total] or null
  unsigned long long* work;   // [1] persistent work counter
  int* flags;                 // [1] bit 0: time budget hit
  // FP32 steady tracer's tail: particles the main kernel hands to the tail
  // kernel (records of park_stride bytes), how many it parked, how many the
  // tail kernel has taken
  unsigned char* park;
  unsigned long long* park_n;
  unsigned long long* park_rd;
  size_t park_stride;
  uint64_t park_cap;          // records the buffer holds (0: no tail kernel)
};

__device__ __forceinline__ size_t sum_copy() { return (size_t)(blockIdx.x & (unsigned)(kSumCopies - 1)); }

__device__ __forceinline__ double* grad_copy(const Acc& A) { return A.gsum + sum_copy() * kGradStride; }

template <typename R>
struct Particle {
  R x[3], u[3];
  R d_rel;          // remaining relaxation distance (nm), three-phonon clock
  R d2;             // remaining two-phonon distance (nm), +inf without that clock
  R v, inv_v, lam;  // current bin
  R t;              // ps (transient)
  R s;              // sign
  int bin;
  uint32_t e;
  int n_relax;
  uint32_t pid;
  int g;
  int mi;           // next measurement index (transient)
  double X;         // sum s l u_tally (nm), FP64 path
  double Xper;      // X at the start of the current relaxation period
  long long Xq;     // the same in fixed point, FP32 path
  long long Xqper;
};

template <typename R>
__device__ __forceinline__ void load_bin(Particle<R>& p, const MatView& M, const float4* binf) {
  if (sizeof(R) == 8) {
    p.v = (R)M.v_d[p.bin];
    p.inv_v = (R)M.inv_v_d[p.bin];
    p.lam = (R)M.lam_d[p.bin];
  } else {
    const float4 b = binf[p.bin];
    p.v = (R)b.x;
    p.inv_v = (R)b.y;
    p.lam = (R)b.z;
  }
}

// Shared resampling step of emissions and relaxations: bin from an alias
// table (~C v or ~C at emission, Eqs. iso_flux / grad_flux_sim / Nbin;
// ~C/tau at relaxation, Eq. n_scatt), direction with polar cosine
// mu = sqrt(R) about a face normal or the gradient (Lambertian, Eq. wall_dir)
// or mu = 1 - 2R (isotropic, Eq. angle_gen), new relaxation distance
// Lambda (-ln R) (Eq. time_to_scat).  w, w1 are the event's sub-blocks 0 and 1.
// axis 3: Lambertian about the frame `fr` (control gradient in a general
// direction; the frame already carries the sign).
template <typename R, bool EXT = true>
__device__ __forceinline__ void resample(Particle<R>& p, const MatView& M, const uint4* rec, const float4* binf,
                                         uint4 w, uint4 w1, bool lambert, int axis, R sgn,
                                         const R* fr = nullptr) {
  p.bin = alias_draw(rec, M.n, w.x, w.y, w1.x);
  const R mu = lambert ? Num<R>::sqrt_(Num<R>::oc(w.z)) : R(1) - R(2) * Num<R>::oc(w.z);
  if (EXT && axis == 3) dir_about_frame<R>(p.u, fr, mu, w.w);
  else dir_about_axis<R>(p.u, axis, sgn, mu, w.w);
  load_bin(p, M, binf);
  p.d_rel = p.lam * (-Num<R>::log_(Num<R>::oc53(w1.y, w1.z)));
}

// FP32 relaxation from one Philox block (tables of at most kOneBlockBins
// bins, draw_words): word 0 times n gives the alias column (high half) and a
// 32-bit uniform for its test (low half, compared with the threshold's high
// word: the acceptance is off by at most n / 2^32), word 1 the flight, words
// 2 and 3 the isotropic direction.  A 24-bit flight uniform is all FP32
// resolves.
constexpr int kOneBlockBins = 65536;

// ------------------------------------------------------------------ FP32 event draws
// What the words of one event decide whatever the particle's state (FP32
// path, tables of at most kOneBlockBins bins): from sub-block 0 the test
// word, the relaxation's bin (alias draw ~ C/tau, Eq. n_scatt), its flight
// factor -ln R (Eq. time_to_scat) and isotropic direction (Eq. angle_gen),
// and the Lambertian direction about a surface normal in the normal's frame
// (mu = sqrt(R), Eq. wall_dir); the two-phonon factor -ln R2 from sub-block
// 256 and the measure-valued reservoir word from sub-block 257 when those are
// in use.  12 words, stored as three 16-byte vectors.
struct __align__(16) Draw32 {
  uint32_t wx;             // sub 0 word 0: specular / alias test word
  int bin;                 // relaxation bin
  float E;                 // -ln R of the relaxation flight
  float iso[3];            // isotropic unit vector
  float lam[3];            // (mu, s cos phi, s sin phi), s = sqrt(1 - mu^2)
  float E2;                // -ln R2 (sub-block 256)
  uint32_t mv_lo, mv_hi;   // sub-block 257 words 0 and 1
};

// Sub-block 0 of an event: one Philox block, one alias lookup, ln, two square
// roots and one sincos.  Products that meet a sum are written with explicit
// roundings so every caller computes the same bits.
__device__ __forceinline__ void draw_words(Draw32& d, uint4 w, const uint4* rec, int n) {
  d.wx = w.x;
  const uint64_t m = (uint64_t)w.x * (uint64_t)n;
  const int col = (int)(m >> 32);
  const uint4 a = rec[col];
  d.bin = ((uint32_t)m < a.y) ? col : (int)a.z;
  d.E = -Num<float>::log_(Num<float>::oc(w.y));
  float sn, cs;
  Num<float>::sincos2pi(Num<float>::co(w.w), &sn, &cs);
  const float mi = 1.0f - 2.0f * Num<float>::oc(w.z);      // exact
  const float si = sqrtf(fmaxf(0.0f, __fmaf_rn(-mi, mi, 1.0f)));
  d.iso[0] = __fmul_rn(si, cs);
  d.iso[1] = __fmul_rn(si, sn);
  d.iso[2] = mi;
  const float ml = sqrtf(Num<float>::oc(w.z));
  const float sl = sqrtf(fmaxf(0.0f, __fmaf_rn(-ml, ml, 1.0f)));
  d.lam[0] = ml;
  d.lam[1] = __fmul_rn(sl, cs);
  d.lam[2] = __fmul_rn(sl, sn);
}

// Two-phonon factor -ln R2 from the words of sub-block 256.
__device__ __forceinline__ float draw_e2(uint4 w) { return -Num<float>::log_(Num<float>::oc53(w.x, w.y)); }

// Where an FP32 event takes its draws.  DrawInline computes them from the
// event's Philox blocks when the event needs them; DrawSlot reads the ones a
// warp computed beforehand for this event (the same functions, so the same
// bits).  ctr is (particle, geometry, event, 0).
struct DrawInline {
  __device__ __forceinline__ Draw32 sub0(uint4 ctr, uint32_t k0, uint32_t k1, const uint4* rec, int n) const {
    Draw32 d;
    draw_words(d, philox(ctr, k0, k1), rec, n);
    return d;
  }
  __device__ __forceinline__ float e2(uint4 ctr, uint32_t k0, uint32_t k1) const {
    ctr.w = 256u;
    return draw_e2(philox(ctr, k0, k1));
  }
  __device__ __forceinline__ unsigned long long mv(uint4 ctr, uint32_t k0, uint32_t k1) const {
    ctr.w = 257u;
    const uint4 r = philox(ctr, k0, k1);
    return (unsigned long long)r.x | ((unsigned long long)r.y << 32);
  }
};

struct DrawSlot {
  const Draw32* s;   // this event's draws (shared memory)
  __device__ __forceinline__ Draw32 sub0(uint4, uint32_t, uint32_t, const uint4*, int) const { return *s; }
  __device__ __forceinline__ float e2(uint4, uint32_t, uint32_t) const { return s->E2; }
  __device__ __forceinline__ unsigned long long mv(uint4, uint32_t, uint32_t) const {
    return (unsigned long long)s->mv_lo | ((unsigned long long)s->mv_hi << 32);
  }
};

// The slot when the event has one (s non-null), else the inline draws: an
// unfolded flight can end on an event past the slots computed for it.
struct DrawSlotOr {
  const Draw32* s;
  __device__ __forceinline__ Draw32 sub0(uint4 ctr, uint32_t k0, uint32_t k1, const uint4* rec, int n) const {
    return s ? *s : DrawInline().sub0(ctr, k0, k1, rec, n);
  }
  __device__ __forceinline__ float e2(uint4 ctr, uint32_t k0, uint32_t k1) const {
    return s ? s->E2 : DrawInline().e2(ctr, k0, k1);
  }
  __device__ __forceinline__ unsigned long long mv(uint4 ctr, uint32_t k0, uint32_t k1) const {
    return s ? DrawSlot{s}.mv(ctr, k0, k1) : DrawInline().mv(ctr, k0, k1);
  }
};

// Two-phonon clock (Sec. 3.3): a new exponential distance with the current
// bin's mean free path v tau_imp, from sub-block 256 of the particle's
// current event; +inf without impurity scattering.
template <typename R, class Src = DrawInline>
__device__ __forceinline__ R draw_d2(const Particle<R>& p, const MatView& M, const float4* binf, uint32_t k0,
                                     uint32_t k1, const Src& src = Src()) {
  if (!M.imp) return Num<R>::inf();
  const R lam2 = sizeof(R) == 8 ? (R)M.lam2_d[p.bin] : (R)binf[p.bin].w;
  if (isinf(lam2)) return Num<R>::inf();
  if constexpr (sizeof(R) == 4) {
    return lam2 * src.e2(make_uint4(p.pid, (uint32_t)p.g, p.e, 0u), k0, k1);
  } else {
    const uint4 w = philox(make_uint4(p.pid, (uint32_t)p.g, p.e, 256u), k0, k1);
    return lam2 * (-Num<R>::log_(Num<R>::oc53(w.x, w.y)));
  }
}

// Emission-only part of event 0 (Sec. 3.2: source by cumulative energy,
// sub 1 word 3; Secs. 3.2.1-3.2.3: sign, emission time, position from sub 2,
// further body-position attempts from sub 2 + j, Box-Muller from sub 3).
// Returns the direction law for resample(): table (0 ~C v, 1 ~C), Lambertian
// or isotropic, axis and sign.
template <typename R, bool EXT = true>
__device__ __forceinline__ void emit_prologue(Particle<R>& p, const GeoRun& g, uint32_t k0, uint32_t k1,
                                              bool transient, R t_max_ps, uint4 w1, int* table, bool* lambert,
                                              int* axis, R* sgn) {
  uint4 ctr = make_uint4(p.pid, (uint32_t)p.g, 0u, 2u);
  const uint4 w2 = philox(ctr, k0, k1);
  int k = 0;
  while ((uint64_t)w1.w >= g.src_thr[k]) ++k;
  const int kind = g.src_kind[k];
  p.t = R(0);
  if (kind == 0) {
    const int f = g.src_face[k];
    const int a = face_axis(f);
    const int mx = face_is_max(f);
    p.s = (R)g.face_sign[f];
    *table = 0;
    *lambert = true;
    *axis = a;
    *sgn = mx ? R(-1) : R(1);
    if (transient) p.t = Num<R>::co(w2.w) * t_max_ps;
    const int a1 = (a == 2) ? 0 : a + 1;
    const int a2 = (a == 0) ? 2 : (a == 1 ? 0 : 1);
    put3_cyclic<R>(p.x, a, mx ? geo_L<R>(g, a) : R(0), Num<R>::mid(w2.x) * geo_L<R>(g, a1),
                   Num<R>::mid(w2.y) * geo_L<R>(g, a2));
  } else if (kind == 1) {
    p.s = (w2.w < 0x80000000u) ? R(1) : R(-1);
    *table = 0;
    *lambert = true;
    *axis = (EXT && g.grad_general) ? 3 : g.grad_axis;
    // positive particles travel down the control gradient, negative ones up it
    *sgn = (p.s > R(0)) ? (R)(-g.grad_sign) : (R)g.grad_sign;
    const R cx = sizeof(R) == 8 ? (R)g.cx : (R)g.cxf;
    const R cy = sizeof(R) == 8 ? (R)g.cy : (R)g.cyf;
    const R r2 = sizeof(R) == 8 ? (R)g.r2 : (R)g.r2f;
    uint4 w3 = w2;
    for (uint32_t j = 0;; ++j) {
      if (j > 0) {
        ctr.w = 2u + j;
        w3 = philox(ctr, k0, k1);
      }
      p.x[0] = Num<R>::mid(w3.x) * geo_L<R>(g, 0);
      p.x[1] = Num<R>::mid(w3.y) * geo_L<R>(g, 1);
      p.x[2] = Num<R>::mid(w3.z) * geo_L<R>(g, 2);
      bool inside = false;
      if (g.pore) {
        const R dx = p.x[0] - cx, dy = p.x[1] - cy;
        inside = dx * dx + dy * dy < r2;
      }
      if (EXT && !inside && g.n_inner > 0) inside = in_hole<R>(g, p.x[0], p.x[1]);
      if (!inside) break;
      if (j + 1 >= 64u) break;
    }
  } else {
    p.s = (R)g.gauss_sign;
    *table = 1;
    *lambert = false;
    *axis = 2;
    *sgn = R(1);
    ctr.w = 3u;
    const uint4 w3 = philox(ctr, k0, k1);
    const R m1 = Num<R>::sqrt_(R(-2) * Num<R>::log_(Num<R>::oc(w3.x)));
    const R m2 = Num<R>::sqrt_(R(-2) * Num<R>::log_(Num<R>::oc(w3.z)));
    R s1, c1, s2, c2;
    Num<R>::sincos2pi(Num<R>::co(w3.y), &s1, &c1);
    Num<R>::sincos2pi(Num<R>::co(w3.w), &s2, &c2);
    const R nrm[3] = {m1 * c1, m1 * s1, m2 * c2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const R La = geo_L<R>(g, a);
      R c = (R)g.gauss_c[a] + (R)g.gauss_sigma * nrm[a];
      if (c < R(0)) c = -c;
      if (c > La) c = R(2) * La - c;
      if (c < R(0)) c = R(0);
      if (c > La) c = La;
      p.x[a] = c;
    }
  }
}

__device__ __forceinline__ void particle_reset_counters(Particle<float>& p) {
  p.e = 0u;
  p.n_relax = 0;
  p.X = 0.0;
  p.Xper = 0.0;
  p.Xq = 0;
  p.Xqper = 0;
}
__device__ __forceinline__ void particle_reset_counters(Particle<double>& p) {
  p.e = 0u;
  p.n_relax = 0;
  p.X = 0.0;
  p.Xper = 0.0;
  p.Xq = 0;
  p.Xqper = 0;
}

// Emission of particle (pid, g) at event 0: the emission prologue, then the
// shared resampling step with the source's bin law and direction law.
// EXT: the run uses extended physics (a two-phonon clock, internal walls,
// per-bin specularity, a control gradient off the axes); without it those
// paths are compiled out.
template <typename R, bool EXT = true>
__device__ __forceinline__ void emit(Particle<R>& p, const GeoRun& g, const MatView& M, const uint4* rec_emit,
                                     const uint4* rec_init, const float4* binf, uint32_t k0, uint32_t k1,
                                     bool transient, R t_max_ps) {
  uint4 ctr = make_uint4(p.pid, (uint32_t)p.g, 0u, 0u);
  const uint4 w = philox(ctr, k0, k1);
  ctr.w = 1u;
  const uint4 w1 = philox(ctr, k0, k1);
  int table;
  bool lambert;
  int axis;
  R sgn;
  emit_prologue<R, EXT>(p, g, k0, k1, transient, t_max_ps, w1, &table, &lambert, &axis, &sgn);
  const int fi = sgn > R(0) ? 1 : 0;
  const R* fr = nullptr;
  if constexpr (sizeof(R) == 8) fr = reinterpret_cast<const R*>(g.gframe[fi]);
  else fr = reinterpret_cast<const R*>(g.gframef[fi]);
  resample<R, EXT>(p, M, table ? rec_init : rec_emit, binf, w, w1, lambert, axis, sgn, fr);
  particle_reset_counters(p);
  if constexpr (EXT) p.d2 = draw_d2(p, M, binf, k0, k1);
}

// ------------------------------------------------------------------ tally policies
// FP64 plain path: every cell the segment crosses gets its own path length,
// added with global FP64 atomics (the plain definition of the track-length
// estimator, Eqs. temp_steady and flux_x_steady).
struct TallyPlain {
  double* cP;      // [nc][4] of this particle's geometry, or null
  double* qb;      // [n_bins], or null
  int nc, ca, ta;
  double h;
  double* det = nullptr;   // [n_det][4] steady detector-region sums, or null

  __device__ __forceinline__ bool has_det() const { return det != nullptr; }
  __device__ __forceinline__ void det_add(size_t c, double a0, double a1, double a2, double a3) const {
    atomicAdd(det + c + 0, a0);
    atomicAdd(det + c + 1, a1);
    atomicAdd(det + c + 2, a2);
    atomicAdd(det + c + 3, a3);
  }

  __device__ __forceinline__ double X(const Particle<double>& p) const { return p.X; }

  __device__ __forceinline__ double segment(Particle<double>& p, double seg) const {
    const double contrib = (p.s * seg) * sel3(p.u, ta);
    p.X += contrib;
    if (!cP) return contrib;
    const double z0 = sel3(p.x, ca);
    const double uc = sel3(p.u, ca);
    const double z1 = z0 + seg * uc;
    if (uc == 0.0) {
      int c = (int)floor(z0 / h);
      c = min(max(c, 0), nc - 1);
      atomicAdd(&cP[c * 4 + 0], (p.s * seg) * p.inv_v);
#pragma unroll
      for (int b = 0; b < 3; ++b) atomicAdd(&cP[c * 4 + 1 + b], (p.s * seg) * p.u[b]);
      return contrib;
    }
    const double zlo = z0 < z1 ? z0 : z1;
    const double zhi = z0 < z1 ? z1 : z0;
    const int clo = min(max((int)floor(zlo / h), 0), nc - 1);
    const int chi = min(max((int)floor(zhi / h), 0), nc - 1);
    const double au = fabs(uc);
    for (int c = clo; c <= chi; ++c) {
      double lo = fmax(zlo, c * h);
      double hi = fmin(zhi, (c + 1) * h);
      if (c == nc - 1) hi = zhi;
      if (c == 0) lo = zlo;
      const double ov = hi - lo;
      if (ov <= 0.0) continue;
      const double l = ov / au;
      atomicAdd(&cP[c * 4 + 0], (p.s * l) * p.inv_v);
#pragma unroll
      for (int b = 0; b < 3; ++b) atomicAdd(&cP[c * 4 + 1 + b], (p.s * l) * p.u[b]);
    }
    return contrib;
  }

  __device__ __forceinline__ void period_end(Particle<double>& p) const {
    if (qb) {
      atomicAdd(&qb[p.bin], p.X - p.Xper);
      p.Xper = p.X;
    }
  }
};

// Out-of-line 64-bit conversion for the rare contributions beyond 2^31
// fixed-point units (kept out of line so the common path never issues it).
static __device__ __noinline__ long long fx_wide(float s) { return __float2ll_rn(s); }

// v in fixed point (units of 2^-20), rounded to nearest; the common case
// fits a 32-bit conversion, larger values take the 64-bit one.
__device__ __forceinline__ long long fx(float v) {
  const float s = v * kFx;
  if (fabsf(s) < 2.0e9f) return (long long)__float2int_rn(s);
  return fx_wide(s);
}

// Integer add to a tally that lives in shared or global memory (a generic
// atomic: the hardware resolves the address space).
__device__ __forceinline__ void red_s64(long long* a, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(a), (unsigned long long)v);
}

// Adds f_i * d to a[i] (i < 4) in fixed point; one range test for the
// group (values below 2e9 in fixed point take the 32-bit conversion, as fx).
__device__ __forceinline__ void fx_add4(long long* a, float f0, float f1, float f2, float f3, float d) {
  const float v0 = (f0 * d) * kFx, v1 = (f1 * d) * kFx, v2 = (f2 * d) * kFx, v3 = (f3 * d) * kFx;
  if (fmaxf(fmaxf(fabsf(v0), fabsf(v1)), fmaxf(fabsf(v2), fabsf(v3))) < 2.0e9f) {
    red_s64(a + 0, (long long)__float2int_rn(v0));
    red_s64(a + 1, (long long)__float2int_rn(v1));
    red_s64(a + 2, (long long)__float2int_rn(v2));
    red_s64(a + 3, (long long)__float2int_rn(v3));
  } else {
    red_s64(a + 0, fx_wide(v0));
    red_s64(a + 1, fx_wide(v1));
    red_s64(a + 2, fx_wide(v2));
    red_s64(a + 3, fx_wide(v3));
  }
}

// The same for {a[0], a[1 + ax]} only (cell tallies of T and the flux along
// one axis).
__device__ __forceinline__ void fx_add2(long long* a, int ax, float f0, float fa, float d) {
  const float v0 = (f0 * d) * kFx, va = (fa * d) * kFx;
  if (fmaxf(fabsf(v0), fabsf(va)) < 2.0e9f) {
    red_s64(a, (long long)__float2int_rn(v0));
    red_s64(a + 1 + ax, (long long)__float2int_rn(va));
  } else {
    red_s64(a, fx_wide(v0));
    red_s64(a + 1 + ax, fx_wide(va));
  }
}

// FP32 path: fixed-point tallies.  Cells use a difference array: the (up to)
// two partial end cells go to P, the run of full cells in between is one
// +/- pair in D, and the per-cell value is P[c] + sum_{c' <= c} D[c'];
// at most 4 x 4 integer atomics per segment whatever the number of cells
// crossed.  The frequency-resolved flux is added once per relaxation
// period (the bin is constant over a period).  NQ = 4: cells tally T and
// q_x, q_y, q_z; NQ = 2: T and the flux along the tally axis only.
template <int NQ = 4>
struct TallyFxT {
  long long* cP;   // [nc][4] (shared memory or global), or null
  long long* cD;   // [nc+1][4]
  long long* qb;   // [n_bins], or null
  int nc, ca, ta;
  float h, inv_h;
  long long* det = nullptr;   // [n_det][4] steady detector-region sums (fixed point), or null

  __device__ __forceinline__ bool has_det() const { return det != nullptr; }
  __device__ __forceinline__ void det_add(size_t c, float a0, float a1, float a2, float a3) const {
    red_s64(det + c + 0, fx(a0));
    red_s64(det + c + 1, fx(a1));
    red_s64(det + c + 2, fx(a2));
    red_s64(det + c + 3, fx(a3));
  }

  __device__ __forceinline__ double X(const Particle<float>& p) const { return (double)p.Xq * kFxInv; }

  __device__ __forceinline__ float segment(Particle<float>& p, float seg) const {
    const float contrib = (p.s * seg) * sel3(p.u, ta);
    p.Xq += __float2ll_rn(contrib * kFx);   // fx(contrib) without its range branch (same rounding)
    if (!cP) return contrib;
    const float z0 = sel3(p.x, ca);
    const float uz = sel3(p.u, ca);
    if (uz == 0.0f) {
      const int c = min(max((int)(z0 * inv_h), 0), nc - 1);
      const float sl = p.s * seg;
      add(cP + c * 4, sl * p.inv_v, sl * p.u[0], sl * p.u[1], sl * p.u[2], 1.0f);
      return contrib;
    }
    const float z1 = z0 + seg * uz;
    const float zlo = fminf(z0, z1);
    const float zhi = fmaxf(z0, z1);
    const int clo = min(max((int)(zlo * inv_h), 0), nc - 1);
    const int chi = min(max((int)(zhi * inv_h), 0), nc - 1);
    const float k = copysignf(__frcp_rn(fabsf(uz)), p.s);   // s / |u_z| exactly (s = +-1): per unit axial length
    const float f0 = k * p.inv_v, f1 = k * p.u[0], f2 = k * p.u[1], f3 = k * p.u[2];
    // the lower end's partial cell always (the whole flight when it stays in
    // one cell); the upper end's and the run of full cells only when needed
    add(cP + clo * 4, f0, f1, f2, f3, (clo == chi ? zhi : (float)(clo + 1) * h) - zlo);
    if (clo == chi) return contrib;
    add(cP + chi * 4, f0, f1, f2, f3, zhi - (float)chi * h);
    if (chi > clo + 1) {
      add(cD + (clo + 1) * 4, f0, f1, f2, f3, h);
      add(cD + chi * 4, f0, f1, f2, f3, -h);
    }
    return contrib;
  }

  __device__ __forceinline__ void add(long long* a, float f0, float f1, float f2, float f3, float d) const {
    if constexpr (NQ == 4) fx_add4(a, f0, f1, f2, f3, d);
    else fx_add2(a, ta, f0, ta == 0 ? f1 : (ta == 1 ? f2 : f3), d);
  }

  __device__ __forceinline__ void period_end(Particle<float>& p) const {
    if (qb) {
      red_s64(qb + p.bin, p.Xq - p.Xqper);
      p.Xqper = p.Xq;
    }
  }
};
using TallyFx = TallyFxT<4>;

// No steady tallies (transient runs).
struct TallyNone {
  template <typename R>
  __device__ __forceinline__ void period_end(Particle<R>&) const {}
  template <typename R>
  __device__ __forceinline__ double X(const Particle<R>&) const { return 0.0; }
};

// ------------------------------------------------------------------ likelihood-ratio policies
// Scores of the sampled laws (no gradient in the paper; derived from them):
//   flight ended by relaxation   -1 + l / Lambda   (density of Eq. time_to_scat)
//   flight ended by a boundary        l / Lambda   (survival)
//   resampling into bin i        -delta_ij + pi_j  (law ~ C/tau of Eq. n_scatt)
//   specular / diffuse pore hit   1/p, -1/(1-p)    (Sec. 3.5.3)
// Each score multiplies the tally still to come (causal form).  Per particle
// and relaxation period k (bin b_k): G[b_k] += A_k X - B_k with A_k the sum
// of its scores and B_k the sum of score x tally-so-far; the dense pi_j part
// is R pi_j with R = n_res X - sum of X at each resampling.
//
// Measure-valued alternative for the pore specularity: the weak derivative
// of the Bernoulli(p) draw of Eq. specular is the difference of its two
// branches.  In the nominal trace (phase 0) pore hit j of the particle takes
// the choice with probability 1/j (reservoir draw: the 64-bit word of
// sub-block 257 of its event is at most floor((2^64 - 1) / j)), so the chosen
// hit is uniform over the K hits; the phantom trace (phase 1) is the same
// particle from its emission with the chosen hit's branch flipped; the score
// is K (X_spec - X_diff).
struct MvdState {
  uint32_t K;      // pore hits of this trace so far
  uint32_t Kn;     // the nominal trace's K (phantom phase)
  uint32_t sel;    // chosen hit (1-based), 0: none
  bool sel_spec;   // the nominal branch at the chosen hit
  bool phase;      // false: nominal trace, true: phantom trace

  __device__ __forceinline__ void reset() {
    K = Kn = sel = 0u;
    sel_spec = false;
    phase = false;
  }
  // word(): the 64-bit reservoir word of this event (sub-block 257), drawn
  // only in the nominal trace
  template <class Word>
  __device__ __forceinline__ bool branch(bool spec, Word word) {
    ++K;
    if (phase) return K == sel ? !spec : spec;
    const unsigned long long v = word();
    // v <= floor((2^64 - 1) / K) exactly when the product v K is below
    // 2^64, i.e. when its high 64 bits are zero (no 64-bit division)
    if (__umul64hi(v, (unsigned long long)K) == 0ull) {
      sel = K;
      sel_spec = spec;
    }
    return spec;
  }
  // the phantom trace starts; the nominal trace's K is kept
  __device__ __forceinline__ void start_phantom() {
    Kn = K;
    K = 0u;
    phase = true;
  }
  __device__ __forceinline__ double score(double X_nominal, double X_phantom) const {
    return (double)Kn * (sel_spec ? X_nominal - X_phantom : X_phantom - X_nominal);
  }
};

struct GradOff {
  static constexpr bool on = false;
  __device__ __forceinline__ void init(int) {}
  template <typename C>
  __device__ __forceinline__ void flight(bool, double, double, C) {}
  __device__ __forceinline__ void resampled(int, double) {}
  template <class Word>
  __device__ __forceinline__ bool pore_branch(bool spec, double, double, Word) { return spec; }
  template <typename R>
  __device__ __forceinline__ void pore_hit(const Particle<R>&) {}
  __device__ __forceinline__ int periods() const { return 0; }
  __device__ __forceinline__ int period_bin(int) const { return 0; }
  __device__ __forceinline__ double period_value(int, double) const { return 0.0; }
  __device__ __forceinline__ double resample_term(double) const { return 0.0; }
  __device__ __forceinline__ double spec_term(double) const { return 0.0; }
};

// FP64 path: the per-segment form, kept operation for operation with the
// CPU implementation of the same scores.
struct GradList {
  static constexpr bool on = true;
  int np;
  int bin[kMaxPeriods];
  double A[kMaxPeriods];
  double B[kMaxPeriods];
  int n_res;
  double sum_x_res;
  double PA, PB;
  bool mvd;         // measure-valued d/dp (set by the kernel)
  MvdState mv;

  __device__ __forceinline__ void init(int b) {
    mv.reset();
    np = 1;
    bin[0] = b;
    A[0] = 0.0;
    B[0] = 0.0;
    n_res = 0;
    sum_x_res = 0.0;
    PA = 0.0;
    PB = 0.0;
  }
  // ratio = l / Lambda of the flight; Xb = tally before it
  __device__ __forceinline__ void flight(bool relax, double ratio, double Xb, double) {
    if (mv.phase) return;
    double score = ratio;
    if (relax) score = score - 1.0;
    A[np - 1] += score;
    B[np - 1] += score * Xb;
  }
  __device__ __forceinline__ void resampled(int b, double Xnow) {
    if (mv.phase) return;
    if (np < kMaxPeriods) {
      bin[np] = b;
      A[np] = -1.0;
      B[np] = -Xnow;
      np++;
    }
    n_res++;
    sum_x_res += Xnow;
  }
  template <class Word>
  __device__ __forceinline__ bool pore_branch(bool spec, double p, double Xnow, Word word) {
    if (mvd) return mv.branch(spec, word);
    const double sc = spec ? 1.0 / p : -1.0 / (1.0 - p);
    PA += sc;
    PB += sc * Xnow;
    return spec;
  }
  __device__ __forceinline__ double period_value(int k, double X) const { return A[k] * X - B[k]; }
  __device__ __forceinline__ int periods() const { return np; }
  __device__ __forceinline__ int period_bin(int k) const { return bin[k]; }
  __device__ __forceinline__ double resample_term(double X) const { return (double)n_res * X - sum_x_res; }
  __device__ __forceinline__ double spec_term(double X) const { return PA * X - PB; }
  template <typename R>
  __device__ __forceinline__ void pore_hit(const Particle<R>&) {}
};

// Relaxation periods a particle of the one-pass FP32 gradient can list
// (runs with N_scat_max up to this many).
constexpr int kFusedPeriods = 16;

// FP32 path.  Each relaxation period k adds A_k X_f - B_k = a (X_f - X_k) + d
// to the gradient of its bin, a being the period's score sum, d the running
// sum of (score so far) x (segment tally) (FP32 registers) and X_k the tally
// when the period closes.
// Replay (second pass): the forward pass stored every particle's final tally
// X_f; this pass traces the same particle again (same random words, same
// fixed-point tally, so the same trajectory) and adds the whole term the
// moment the period closes.  Nothing is stored per period.
// Fused (one pass, N_scat_max <= kFusedPeriods): X_f is known only at the
// particle's end, so a closing period adds d - a X_k at once and lists
// (bin, a); the end adds a X_f for every listed period.
struct GradReplay {
  static constexpr bool on = true;
  double Xf;
  long long* G;         // [n_bins] gradient accumulator (shared or global memory, 2^-20 fixed point: order-free sums)
  int bin_cur;
  float a, d;
  float pa, pd;
  int n_res;
  double sum_x_res;
  int n_dirs, n_bins;
  const double* dirs;
  // The arrays live outside the struct (the kernel's own local arrays): a
  // struct holding a dynamically indexed array stays in local memory as a
  // whole, and the per-flight scalars above would go with it.
  double* dv;           // [kMaxDirs] per direction: sum over closed periods of value x dirs[bin]
  bool mvd;             // measure-valued d/dp (set by the kernel)
  bool fused;           // one pass (set by the kernel)
  int np;               // fused: listed periods
  int* lb;              // [kFusedPeriods] fused: their bins
  float* la;            // [kFusedPeriods] fused: their score sums
  // Measure-valued d/dp: the particle as it reached the chosen pore hit
  // (position on the wall, incoming direction, clocks, tally, counters), so
  // the phantom trace resumes there instead of tracing again from the
  // emission: the same state, hence the same bits.  Null: no snapshot.
  int4* snap;           // [4] this lane's record (shared memory)
  bool snap_ok;
  MvdState mv;

  __device__ __forceinline__ void init(int b) {
    mv.reset();
    bin_cur = b;
    a = d = pa = pd = 0.0f;
    n_res = 0;
    sum_x_res = 0.0;
    np = 0;
    snap_ok = false;
    for (int k = 0; k < n_dirs; ++k) dv[k] = 0.0;
  }
  // after the pore branch of a hit: the hit just chosen (nominal trace) is
  // recorded; p has reached the wall and not yet turned
  template <typename R>
  __device__ __forceinline__ void pore_hit(const Particle<R>& p) {
    if constexpr (sizeof(R) == 4) {
      if (!mvd || mv.phase || mv.sel != mv.K || snap == nullptr) return;
      snap[0] = make_int4(__float_as_int(p.x[0]), __float_as_int(p.x[1]), __float_as_int(p.x[2]),
                          __float_as_int(p.u[0]));
      snap[1] = make_int4(__float_as_int(p.u[1]), __float_as_int(p.u[2]), __float_as_int(p.d_rel),
                          __float_as_int(p.d2));
      snap[2] = make_int4((int)(unsigned)p.Xq, (int)(p.Xq >> 32), (int)(unsigned)p.Xqper, (int)(p.Xqper >> 32));
      snap[3] = make_int4((int)p.e, p.bin, p.n_relax, __float_as_int(p.s));
      snap_ok = true;
    }
  }
  // the particle back at the chosen hit, its event not yet applied (e one
  // less); the caller reloads the bin's constants and applies the event
  __device__ __forceinline__ void restore(Particle<float>& p) const {
    const int4 a = snap[0], b = snap[1], c = snap[2], d = snap[3];
    p.x[0] = __int_as_float(a.x);
    p.x[1] = __int_as_float(a.y);
    p.x[2] = __int_as_float(a.z);
    p.u[0] = __int_as_float(a.w);
    p.u[1] = __int_as_float(b.x);
    p.u[2] = __int_as_float(b.y);
    p.d_rel = __int_as_float(b.z);
    p.d2 = __int_as_float(b.w);
    p.Xq = (long long)(((unsigned long long)(unsigned)c.y << 32) | (unsigned)c.x);
    p.Xqper = (long long)(((unsigned long long)(unsigned)c.w << 32) | (unsigned)c.z);
    p.e = (uint32_t)d.x - 1u;
    p.bin = d.y;
    p.n_relax = d.z;
    p.s = __int_as_float(d.w);
  }
  __device__ __forceinline__ void flight(bool relax, double ratio, double, float c) {
    if (mv.phase) return;
    a += (float)ratio - (relax ? 1.0f : 0.0f);
    d = fmaf(a, c, d);
    pd = fmaf(pa, c, pd);
  }
  __device__ __forceinline__ void add(int b, double val) {
    red_s64(&G[b], __double2ll_rn(val * kFx));
    for (int k = 0; k < n_dirs; ++k) dv[k] += val * dirs[(size_t)k * n_bins + b];
  }
  __device__ __forceinline__ void close_period(double Xnow) {
    if (fused) {
      add(bin_cur, (double)d - (double)a * Xnow);
      if (np < kFusedPeriods) {   // always: the host runs this pass only for N_scat_max <= kFusedPeriods
        lb[np] = bin_cur;
        la[np] = a;
        ++np;
      }
    } else {
      add(bin_cur, (double)a * (Xf - Xnow) + (double)d);
    }
  }
  // the particle's end, X its final tally: the open period (X_k = X_f: its
  // term is d), and in a fused pass the listed periods' a X_f
  __device__ __forceinline__ void finish(double X) {
    if (!fused) {
      close_period(X);
      return;
    }
    add(bin_cur, (double)d);
    for (int k = 0; k < np; ++k) add(lb[k], (double)la[k] * X);
  }
  __device__ __forceinline__ void resampled(int b, double Xnow) {
    if (mv.phase) return;
    close_period(Xnow);
    bin_cur = b;
    a = -1.0f;
    d = 0.0f;
    n_res++;
    sum_x_res += Xnow;
  }
  template <class Word>
  __device__ __forceinline__ bool pore_branch(bool spec, double p, double, Word word) {
    if (mvd) return mv.branch(spec, word);
    pa += spec ? (float)(1.0 / p) : (float)(-1.0 / (1.0 - p));
    return spec;
  }
  __device__ __forceinline__ double resample_term(double X) const { return (double)n_res * X - sum_x_res; }
  __device__ __forceinline__ double spec_term(double) const { return (double)pd; }
};

// A warp's run of particle indices [cb, ce), taken from the run's work
// counter `chunk` at a time (RunCfg::take_chunk): one returning atomic on
// that single address per chunk instead of one per warp refill.  take()
// (called by the whole warp) returns this lane's index among the lanes in
// `need` (the others' values are meaningless) and checks the time budget at
// every take of the counter (particles shorter than the per-event check
// interval would otherwise never look).  dry: the counter has run out; with
// cb >= ce the warp has nothing left to hand out.
struct WarpRun {
  uint64_t cb = 0, ce = 0;
  bool dry = false;
  __device__ __forceinline__ uint64_t take(unsigned need, unsigned lane, unsigned long long* work, uint64_t total,
                                           unsigned chunk, uint64_t deadline, int* flags) {
    const unsigned cnt = __popc(need);
    const unsigned rank = __popc(need & ((1u << lane) - 1u));
    const uint64_t left = cb < ce ? ce - cb : 0;
    if (left >= cnt) {
      const uint64_t k = cb + rank;
      cb += cnt;
      return k;
    }
    chunk = chunk < 32u ? 32u : chunk;   // at least a warp's refill
    unsigned long long nb = 0;
    if (lane == 0) {
      nb = atomicAdd(work, (unsigned long long)chunk);
      if (globaltimer_ns() > deadline) atomicOr(flags, 1);
    }
    nb = __shfl_sync(0xffffffffu, nb, 0);
    const uint64_t k = rank < left ? cb + rank : nb + (rank - left);
    cb = nb + (cnt - left);
    ce = nb + chunk < total ? nb + chunk : total;
    if (nb + chunk >= total) dry = true;
    return k;
  }
  __device__ __forceinline__ bool empty() const { return dry && cb >= ce; }
};

// Philox key of the run: the host seed, or the device-resident one.
__device__ __forceinline__ uint2 run_key(const RunCfg& C) {
  if (C.seed_dev) {
    const unsigned long long s = *C.seed_dev;
    return make_uint2((uint32_t)s, (uint32_t)(s >> 32));
  }
  return make_uint2(C.k0, C.k1);
}

// Outcome of one event step.
enum { STEP_ALIVE = 0, STEP_ABSORBED = 1, STEP_DONE = 2, STEP_TRUNCATED = 3 };

// The event that ends a flight (Sec. 3.3 cases i/iii; Secs. 3.5.2-3.5.6):
// relaxation (bin redrawn ~ C/tau, isotropic direction, new clock, sign
// kept), or the boundary `face` (isothermal: absorbed; periodic: translated
// to the opposite face; adiabatic / pore: specular with probability p, else
// Lambertian about the inward normal).  The particle has already moved.
// `Xnow` is the particle's tally so far (gradient bookkeeping only).
// Slot k of geometry g's N_scat_max curve sums in this block's copy.
__device__ __forceinline__ double* nscat_slot(const RunCfg& C, int g, int k) {
  const size_t rep = (size_t)(blockIdx.x & (unsigned)(C.nscat_rep - 1));
  return C.nscat_acc + ((rep * (size_t)C.n_geoms + (size_t)g) * (size_t)(C.n_scat_max + 1) + (size_t)k) * 4;
}

template <typename R, class Grad, class Tally, bool EXT = true, class Src = DrawInline>
__device__ __forceinline__ int apply_event(Particle<R>& p, const GeoRun& g, const MatView& M, const uint4* rec_relax,
                                           const float4* binf, const RunCfg& C, uint32_t k0, uint32_t k1,
                                           bool relax, bool relax2, int face, R seg, const Tally& T, Grad& gr,
                                           double Xnow, const Src& src = Src()) {
  ++p.e;
  uint4 ctr = make_uint4(p.pid, (uint32_t)p.g, p.e, 0u);
  if (relax) {
    ++p.n_relax;
    if constexpr (EXT) {
      if (C.nscat_acc) {
        // a run with N_scat_max = n_relax would end the particle here with this tally
        const double x = T.X(p);
        double* a = nscat_slot(C, p.g, p.n_relax);
        atomicAdd(a + 0, x);
        atomicAdd(a + 1, x * x);
      }
    }
    if (C.n_scat_max > 0 && p.n_relax >= C.n_scat_max) return STEP_DONE;
    // the relaxation period in this bin is over: frequency-resolved flux
    T.period_end(p);
    if (sizeof(R) == 4 && M.n <= kOneBlockBins) {
      const Draw32 d = src.sub0(ctr, k0, k1, rec_relax, M.n);
      p.bin = d.bin;
#pragma unroll
      for (int b = 0; b < 3; ++b) p.u[b] = (R)d.iso[b];
      load_bin(p, M, binf);
      p.d_rel = p.lam * (R)d.E;
    } else {
      const uint4 w = philox(ctr, k0, k1);
      ctr.w = 1u;
      const uint4 w1 = philox(ctr, k0, k1);
      resample<R>(p, M, rec_relax, binf, w, w1, false, 2, R(1));
    }
    if constexpr (EXT) p.d2 = draw_d2(p, M, binf, k0, k1, src);   // both clocks restart in the new mode (Sec. 3.3 (i))
    if (Grad::on) gr.resampled(p.bin, Xnow);
    return STEP_ALIVE;
  }
  p.d_rel = p.d_rel - seg;
  if constexpr (EXT) {
    if (relax2) {
      // two-phonon scattering (Sec. 3.5.1, Sec. 3.3 (ii)): same mode, new
      // isotropic direction, new two-phonon clock; the three-phonon clock runs on
      if constexpr (sizeof(R) == 4) {
        const Draw32 d = src.sub0(ctr, k0, k1, rec_relax, M.n);
#pragma unroll
        for (int b = 0; b < 3; ++b) p.u[b] = (R)d.iso[b];
      } else {
        const uint4 w = philox(ctr, k0, k1);
        dir_about_axis<R>(p.u, 2, R(1), R(1) - R(2) * Num<R>::oc(w.z), w.w);
      }
      p.d2 = draw_d2(p, M, binf, k0, k1, src);
      return STEP_ALIVE;
    }
    p.d2 = p.d2 - seg;
  }
  if (face < 6) {
    const int a = face_axis(face);
    const int mx = face_is_max(face);
    const R La = geo_L<R>(g, a);
    const int ty = g.type[face];
    if (ty == MCBTE_FACE_ISOTHERMAL) {
      put3<R>(p.x, a, mx ? La : R(0));
      return STEP_ABSORBED;
    }
    if (ty == MCBTE_FACE_PERIODIC) {
      put3<R>(p.x, a, mx ? R(0) : La);
      return STEP_ALIVE;
    }
    put3<R>(p.x, a, mx ? La : R(0));
    if constexpr (sizeof(R) == 4) {
      // FP32: both outcomes, then a select (no branch on the draw)
      const Draw32 d = src.sub0(ctr, k0, k1, rec_relax, M.n);
      const bool spec_f = (uint64_t)d.wx < ((EXT && ((g.fbin >> face) & 1)) ? M.spec_thr[p.bin] : g.pthr[face]);
      R ud[3];
      put3_cyclic<R>(ud, a, mx ? -d.lam[0] : d.lam[0], d.lam[1], d.lam[2]);
      const R flip = -sel3(p.u, a);
#pragma unroll
      for (int b = 0; b < 3; ++b) p.u[b] = spec_f ? (b == a ? flip : p.u[b]) : ud[b];
    } else {
      const uint4 w = philox(ctr, k0, k1);
      const bool spec_f = (uint64_t)w.x < ((EXT && ((g.fbin >> face) & 1)) ? M.spec_thr[p.bin] : g.pthr[face]);
      if (spec_f) put3<R>(p.u, a, -sel3(p.u, a));
      else dir_about_axis<R>(p.u, a, mx ? R(-1) : R(1), Num<R>::sqrt_(Num<R>::oc(w.z)), w.w);
    }
    return STEP_ALIVE;
  }
  if constexpr (sizeof(R) == 4) {
    // FP32 pore or internal wall: both outcomes, then a select (no branch on
    // the draw); explicit roundings keep every draw source's bits equal
    const Draw32 d = src.sub0(ctr, k0, k1, rec_relax, M.n);
    float nx, ny;
    bool spec;
    if (EXT && face >= 7) {
      // internal wall (Sec. 4.2): onto its line, then reflect about its normal
      const int k = face - 7;
      nx = g.snxf[k];
      ny = g.snyf[k];
      const float dn = __fmaf_rn(p.x[0] - g.sx1f[k], nx, __fmul_rn(p.x[1] - g.sy1f[k], ny));
      p.x[0] = __fmaf_rn(-dn, nx, p.x[0]);
      p.x[1] = __fmaf_rn(-dn, ny, p.x[1]);
      spec = (uint64_t)d.wx < (((g.sbin >> k) & 1) ? M.spec_thr[p.bin] : g.sthr[k]);
    } else {
      // pore wall: the cylinder's outward normal points into the solid
      nx = p.x[0] - g.cxf;
      ny = p.x[1] - g.cyf;
      // unit normal by the hardware reciprocal square root (the two
      // quotients of a correctly rounded normalisation sat on the chain)
      const float il = rsqrtf(__fmaf_rn(nx, nx, __fmul_rn(ny, ny)));
      nx = nx * il;
      ny = ny * il;
      spec = (uint64_t)d.wx < g.pthr_pore;
      if (Grad::on) {
        spec = gr.pore_branch(spec, g.p_pore, Xnow, [&] { return src.mv(ctr, k0, k1); });
        gr.pore_hit(p);
      }
    }
    const float two_un = 2.0f * __fmaf_rn(p.u[0], nx, __fmul_rn(p.u[1], ny));
    const float s0 = __fmaf_rn(-two_un, nx, p.u[0]);
    const float s1 = __fmaf_rn(-two_un, ny, p.u[1]);
    const float l0 = __fmaf_rn(d.lam[0], nx, -__fmul_rn(d.lam[1], ny));
    const float l1 = __fmaf_rn(d.lam[0], ny, __fmul_rn(d.lam[1], nx));
    p.u[0] = spec ? s0 : l0;
    p.u[1] = spec ? s1 : l1;
    p.u[2] = spec ? p.u[2] : d.lam[2];
    return STEP_ALIVE;
  } else {
    R nx, ny;
    bool spec;
    const uint4 w = philox(ctr, k0, k1);
    if (EXT && face >= 7) {
      // internal wall (Sec. 4.2): onto its line, then reflect about its normal
      const int k = face - 7;
      nx = (R)g.snx[k];
      ny = (R)g.sny[k];
      const R dn = (p.x[0] - (R)g.sx1[k]) * nx + (p.x[1] - (R)g.sy1[k]) * ny;
      p.x[0] = p.x[0] - dn * nx;
      p.x[1] = p.x[1] - dn * ny;
      spec = (uint64_t)w.x < (((g.sbin >> k) & 1) ? M.spec_thr[p.bin] : g.sthr[k]);
    } else {
      // pore wall: the cylinder's outward normal points into the solid
      nx = p.x[0] - (R)g.cx;
      ny = p.x[1] - (R)g.cy;
      const R len = Num<R>::sqrt_(nx * nx + ny * ny);
      nx = nx / len;
      ny = ny / len;
      spec = (uint64_t)w.x < g.pthr_pore;
      if (Grad::on) spec = gr.pore_branch(spec, g.p_pore, Xnow, [&] { return DrawInline().mv(ctr, k0, k1); });
    }
    if (spec) {
      const R un = p.u[0] * nx + p.u[1] * ny;
      p.u[0] = p.u[0] - (R(2) * un) * nx;
      p.u[1] = p.u[1] - (R(2) * un) * ny;
    } else {
      const R mu = Num<R>::sqrt_(Num<R>::oc(w.z));
      const R sn = Num<R>::sqrt_(Num<R>::fmax_(R(0), R(1) - mu * mu));
      R sphi, cphi;
      Num<R>::sincos2pi(Num<R>::co(w.w), &sphi, &cphi);
      const R sc = sn * cphi;
      p.u[0] = mu * nx - sc * ny;
      p.u[1] = mu * ny + sc * nx;
      p.u[2] = sn * sphi;
    }
    return STEP_ALIVE;
  }
}

// Steady detector regions (Sec. 4.5): the flight's track length in every
// detector it crosses, s dt for T (ps) and s v dt u for q (nm), dt the time
// spent in the detector (the time integral of Eqs. temp_steady, flux_x_steady).
template <typename R, class Tally>
__device__ __forceinline__ void region_steady(const Particle<R>& p, R seg, const RunCfg& C, const Tally& T) {
  const R v = p.v;
  const R w3[3] = {v * p.u[0], v * p.u[1], v * p.u[2]};
  const R dt = sizeof(R) == 8 ? seg / v : seg * p.inv_v;
  for (int k = 0; k < C.n_regs; ++k) {
    const DetRegion& r = C.regs[k];
    region_track<R>(r, p.x, w3, R(0), R(0), dt, [&](uint32_t d, R dur) {
      T.det_add((((size_t)r.off + d) * (size_t)C.det_nb + (C.det_nb > 1 ? (size_t)p.bin : 0)) * 4, p.s * dur, ((p.s * v) * dur) * p.u[0], ((p.s * v) * dur) * p.u[1],
                ((p.s * v) * dur) * p.u[2]);
    });
  }
}

// One flight + event of a steady (or gradient) particle: first hit vs the
// remaining relaxation distance (boundary wins ties, Sec. 3.3 case iii),
// track-length tallies of the flight (Eqs. temp_steady, flux_x_steady), then
// the event.
// Periodic axes an FP32 forward flight runs through (no extended physics,
// no pore, no walls; never the cell axis, whose tallies follow the position).
// A gradient pass keeps stopping at them: its causal scores depend on where
// flights are cut.
template <class Grad>
__device__ __forceinline__ unsigned unfold_mask(const GeoRun& g, const RunCfg& C) {
  if (Grad::on) return 0u;
  return (unsigned)g.unfold & ~(C.n_cells > 0 ? (1u << C.cell_axis) : 0u);
}

// UNF: the kernel compiles the unfolded flight in (FP32 kernels without
// cell tallies; the others keep their registers for the tallies).
template <typename R, class Grad, class Tally, bool EXT = true, class Src = DrawInline, bool UNF = false>
__device__ __forceinline__ int step_steady(Particle<R>& p, const GeoRun& g, const MatView& M, const uint4* rec_relax,
                                           const float4* binf, const RunCfg& C, uint32_t k0, uint32_t k1,
                                           const Tally& T, Grad& gr, const Src& src = Src()) {
  if (p.e + 1u >= C.max_events) return STEP_TRUNCATED;
  if constexpr (UNF && sizeof(R) == 4 && !EXT && !Grad::on) {
    const unsigned um = unfold_mask<Grad>(g, C);
    if (um) {
      // the flight runs to the nearest face off the periodic axes (or the
      // relaxation), crossing periodic faces on its way; the crossings are
      // counted as the events they are, so the event that ends the flight
      // keeps its number and its random words
      float db;
      int face;
      hit_box_pore_f32(g, p.x, p.u, &db, &face, um);
      const bool relax = p.d_rel < db;
      const float seg = relax ? p.d_rel : db;
      T.segment(p, seg);
#pragma unroll
      for (int a = 0; a < 3; ++a) p.x[a] = p.x[a] + seg * p.u[a];
      const uint32_t n = fold_periodic(p.x, g.Lf, um);
      if (n >= C.max_events - 1u - p.e) {
        p.e = C.max_events - 1u;
        return STEP_TRUNCATED;
      }
      p.e += n;
      return apply_event<R, Grad, Tally, EXT, Src>(p, g, M, rec_relax, binf, C, k0, k1, relax, false, face, seg, T,
                                                   gr, 0.0, src);
    }
  }
  R db;
  int face;
  first_hit<R, EXT>(g, p.x, p.u, &db, &face);
  // nearest of the two scattering clocks and the boundary (Sec. 3.3): the
  // boundary wins ties, the three-phonon clock wins a tie with the two-phonon one
  const bool relax = EXT ? (p.d_rel < db && p.d_rel <= p.d2) : p.d_rel < db;
  const bool relax2 = EXT && !relax && p.d2 < db;
  const R seg = relax ? p.d_rel : (relax2 ? p.d2 : db);
  double Xb = 0.0;
  if (Grad::on) Xb = T.X(p);
  const auto c = T.segment(p, seg);
  if constexpr (EXT) {
    if (C.n_regs > 0 && T.has_det()) region_steady<R>(p, seg, C, T);
  }
  if (Grad::on) gr.flight(relax, (double)Num<R>::div(seg, p.lam), Xb, c);
#pragma unroll
  for (int a = 0; a < 3; ++a) p.x[a] = p.x[a] + seg * p.u[a];
  return apply_event<R, Grad, Tally, EXT, Src>(p, g, M, rec_relax, binf, C, k0, k1, relax, relax2, face, seg, T, gr,
                                                 Grad::on ? T.X(p) : 0.0, src);
}

// One flight + event of a transient particle: the flight also ends at
// t_max (Sec. 3.5.6); every measurement time t_m inside the flight's
// interval [t, t_end) (closed at t_max) adds the particle's snapshot to its
// detector cell (Eq. sampling, Sec. 3.4).
// One snapshot into tally entry c: FP64 atomics, or (FP32 path) the exact
// signed count and the flux in 2^-20 nm/ps fixed point.
template <typename R>
__device__ __forceinline__ void snap_add(double* snap, size_t c, R s, R sv, const R u[3], R v) {
  if constexpr (sizeof(R) == 8) {
    atomicAdd(&snap[c + 0], (double)s);
    atomicAdd(&snap[c + 1], (double)(sv * u[0]));
    atomicAdd(&snap[c + 2], (double)(sv * u[1]));
    atomicAdd(&snap[c + 3], (double)(sv * u[2]));
  } else {
    long long* q = reinterpret_cast<long long*>(snap) + c;
    red_s64(q + 0, s > R(0) ? 1ll : -1ll);
    red_s64(q + 1, fx((float)(sv * u[0])));
    red_s64(q + 2, fx((float)(sv * u[1])));
    red_s64(q + 3, fx((float)(sv * u[2])));
  }
  (void)v;
}

// `tmeas`: the measurement times in ps (FP64 path: the global array; FP32
// path: a float copy in shared memory).  `cinv`: cells per nm along x, y, z
// (FP32 path only; the FP64 path divides by the cell size, the CPU reference form).
template <typename R, bool EXT = true>
__device__ __forceinline__ int step_transient(Particle<R>& p, const GeoRun& g, const MatView& M,
                                              const uint4* rec_relax, const float4* binf, const RunCfg& C,
                                              uint32_t k0, uint32_t k1, double* snap, const R* tmeas,
                                              const R* cinv) {
  if (p.e + 1u >= C.max_events) return STEP_TRUNCATED;
  R db;
  int face;
  first_hit<R, EXT>(g, p.x, p.u, &db, &face);
  const R v = p.v;
  const R tmax = (R)C.t_max_ps;
  const R d_end = (tmax - p.t) * v;
  bool fin = false, relax = false, relax2 = false;
  R seg;
  if (d_end <= p.d_rel && d_end <= db && (!EXT || d_end <= p.d2)) { fin = true; seg = d_end; }
  else if (p.d_rel < db && (!EXT || p.d_rel <= p.d2)) { relax = true; seg = p.d_rel; }
  else if (EXT && p.d2 < db) { relax2 = true; seg = p.d2; }
  else { seg = db; }
  // the flight ended by t_max ends at t_max exactly (Sec. 3.5.6), so a
  // measurement at t_max samples every particle still alive
  const R t_end = fin ? tmax : ((sizeof(R) == 8) ? p.t + seg / v : p.t + seg * p.inv_v);
  const int nx = C.grid[0], ny = C.grid[1], nz = C.grid[2];
  const size_t ncell = (size_t)nx * ny * nz;
  if (C.time_average) {
    // bin averages over [t_{m-1}, t_m): the flight's time in each detector
    // during each bin it overlaps, over the bin's length
    const R w3[3] = {v * p.u[0], v * p.u[1], v * p.u[2]};
    while (p.mi < C.n_times) {
      const R b0 = p.mi == 0 ? R(0) : tmeas[p.mi - 1];
      const R b1 = tmeas[p.mi];
      if (!(b0 < t_end)) break;
      const R ta = p.t > b0 ? p.t : b0;
      const R tb = t_end < b1 ? t_end : b1;
      if (ta < tb) {
        const R wb = R(1) / (b1 - b0);
        for (int k = 0; k < C.n_regs; ++k) {
          const DetRegion& r = C.regs[k];
          const size_t base = (size_t)p.mi * C.n_det + r.off;
          region_track<R>(r, p.x, w3, p.t, ta, tb, [&](uint32_t det, R dur) {
            const size_t c = (base + det) * 4;
            const R f = (p.s * dur) * wb;
            if constexpr (sizeof(R) == 8) {
              atomicAdd(&snap[c + 0], (double)f);
              atomicAdd(&snap[c + 1], (double)((f * v) * p.u[0]));
              atomicAdd(&snap[c + 2], (double)((f * v) * p.u[1]));
              atomicAdd(&snap[c + 3], (double)((f * v) * p.u[2]));
            } else {
              // FP32 path: every component in 2^-20 fixed point (the weights are fractions)
              long long* q = reinterpret_cast<long long*>(snap) + c;
              red_s64(q + 0, fx((float)f));
              red_s64(q + 1, fx((float)((f * v) * p.u[0])));
              red_s64(q + 2, fx((float)((f * v) * p.u[1])));
              red_s64(q + 3, fx((float)((f * v) * p.u[2])));
            }
          });
        }
      }
      if (b1 <= t_end) ++p.mi;
      else break;
    }
  } else
  while (p.mi < C.n_times) {
    const R tm = tmeas[p.mi];
    if (!(tm < t_end || (fin && tm <= t_end))) break;
    const R dist = v * (tm - p.t);
    R pm[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) pm[a] = p.x[a] + dist * p.u[a];
    int ix, iy, iz;
    if constexpr (sizeof(R) == 8) {
      ix = (int)floor(pm[0] / (geo_L<R>(g, 0) / (R)nx));
      iy = (int)floor(pm[1] / (geo_L<R>(g, 1) / (R)ny));
      iz = (int)floor(pm[2] / (geo_L<R>(g, 2) / (R)nz));
    } else {
      ix = (int)floorf(pm[0] * cinv[0]);
      iy = (int)floorf(pm[1] * cinv[1]);
      iz = (int)floorf(pm[2] * cinv[2]);
    }
    ix = min(max(ix, 0), nx - 1);
    iy = min(max(iy, 0), ny - 1);
    iz = min(max(iz, 0), nz - 1);
    const R sv = p.s * v;
    if (C.n_regs > 0) {
      // detector regions: every half-open cuboid [lo, hi) containing the
      // position (closed on the box's upper faces)
      for (int k = 0; k < C.n_regs; ++k) {
        const DetRegion& r = C.regs[k];
        int i3[3];
        bool in = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const R lo = sizeof(R) == 8 ? (R)r.lo[a] : (R)r.lof[a];
          const R hi = sizeof(R) == 8 ? (R)r.hi[a] : (R)r.hif[a];
          in = in && pm[a] >= lo && (pm[a] < hi || (pm[a] == hi && pm[a] >= geo_L<R>(g, a)));
          int ia;
          if constexpr (sizeof(R) == 8) ia = (int)floor((pm[a] - lo) / (R)r.h[a]);
          else ia = (int)floorf((pm[a] - lo) * r.cinvf[a]);
          i3[a] = min(max(ia, 0), r.n[a] - 1);
        }
        if (!in) continue;
        const size_t c = ((size_t)p.mi * C.n_det + r.off + ((size_t)i3[2] * r.n[1] + i3[1]) * r.n[0] + i3[0]) * 4;
        snap_add<R>(snap, c, p.s, sv, p.u, v);
      }
      ++p.mi;
      continue;
    }
    const size_t c = ((size_t)p.mi * ncell + ((size_t)iz * ny + iy) * nx + ix) * 4;
    if (sizeof(R) == 8) {
      atomicAdd(&snap[c + 0], (double)p.s);
      atomicAdd(&snap[c + 1], (double)(sv * p.u[0]));
      atomicAdd(&snap[c + 2], (double)(sv * p.u[1]));
      atomicAdd(&snap[c + 3], (double)(sv * p.u[2]));
    } else {
      // FP32 path: the signed count exactly, the flux in 2^-20 nm/ps units;
      // |s v u_a| <= v (1 + rounding), so for v below 2^10 nm/ps every
      // component is below 2^30 in fixed point and the 32-bit conversion
      // gives the value fx gives, without its range test
      long long* q = reinterpret_cast<long long*>(snap) + c;
      red_s64(q + 0, p.s > R(0) ? 1ll : -1ll);
      if ((float)v < 1024.0f) {
        red_s64(q + 1, (long long)__float2int_rn((float)(sv * p.u[0]) * kFx));
        red_s64(q + 2, (long long)__float2int_rn((float)(sv * p.u[1]) * kFx));
        red_s64(q + 3, (long long)__float2int_rn((float)(sv * p.u[2]) * kFx));
      } else {
        red_s64(q + 1, fx((float)(sv * p.u[0])));
        red_s64(q + 2, fx((float)(sv * p.u[1])));
        red_s64(q + 3, fx((float)(sv * p.u[2])));
      }
    }
    ++p.mi;
  }
  p.t = t_end;
#pragma unroll
  for (int a = 0; a < 3; ++a) p.x[a] = p.x[a] + seg * p.u[a];
  if (fin) return STEP_DONE;
  GradOff off;
  return apply_event<R, GradOff, TallyNone, EXT>(p, g, M, rec_relax, binf, C, k0, k1, relax, relax2, face, seg, TallyNone(), off,
                                            0.0);
}

}  // namespace mcbte
