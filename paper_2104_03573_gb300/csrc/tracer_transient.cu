// Transient tracing (Secs. 3.2-3.5): wall sources emit at t0 = R t_max, the
// initial condition at t0 = 0 (Sec. 3.2); every measurement time inside a
// particle's life adds its snapshot to the detector grid (Eq. sampling).
// FP64 plain kernel (one thread per particle) and persistent FP32 kernel
// (per-lane refill, alias tables in shared memory, FP64 L2 atomics into the
// [time][cell][T, qx, qy, qz] tally, which is far larger than shared memory).
#include "launch.h"

#ifndef MCBTE_F64
#define MCBTE_F64 0
#endif
#ifndef MCBTE_F32
#define MCBTE_F32 0
#endif

namespace mcbte {

namespace {

// First measurement index still ahead of the particle: for snapshots the
// first t_m >= t0, for bin averages the bin [t_{m-1}, t_m) containing t0.
template <typename R>
__device__ __forceinline__ void transient_start(Particle<R>& p, const RunCfg& C) {
  p.mi = 0;
  if (C.time_average) {
    while (p.mi < C.n_times && (R)C.t_meas_ps[p.mi] <= p.t) ++p.mi;
  } else {
    while (p.mi < C.n_times && (R)C.t_meas_ps[p.mi] < p.t) ++p.mi;
  }
}

template <typename R>
__device__ __forceinline__ void transient_finish(const Particle<R>& p, int out, uint64_t idx, const Acc& A) {
  const unsigned long long nev = (unsigned long long)p.e + 1ull;
  unsigned long long* cnt = A.cnt + sum_copy() * 4;
  double* dsc = A.dsc + sum_copy() * 8;
  atomicAdd(cnt + 0, nev);
  if (out == STEP_TRUNCATED) atomicAdd(cnt + 1, 1ull);
  atomicMax(cnt + 2, nev);
  atomicAdd(cnt + 3, 1ull);
  atomicAdd(dsc + 2, (double)p.s);
  if (out == STEP_ABSORBED) {
    atomicAdd(dsc + 3, (double)p.s);
    atomicAdd(dsc + 7, 1.0);
  }
  if (A.events_pp) A.events_pp[idx] = (uint32_t)nev;
}

#if MCBTE_F64
__global__ void __launch_bounds__(256) k_transient_fp64(const GeoRun* __restrict__ geos, MatView M, RunCfg C, Acc A) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= C.total) return;
  const GeoRun& G = geos[0];
  const uint64_t deadline = *C.t0 + C.budget_ns;
  Particle<double> p;
  p.pid = (uint32_t)idx;
  p.g = 0;
  const uint2 key = run_key(C);
  if (globaltimer_ns() > deadline) {   // over budget before this particle started
    atomicOr(A.flags, 1);
    return;
  }
  emit<double>(p, G, M, M.rec_emit, M.rec_init, nullptr, key.x, key.y, true, C.t_max_ps);
  transient_start(p, C);
  int out;
  for (;;) {
    out = step_transient<double>(p, G, M, M.rec_relax, nullptr, C, key.x, key.y, A.snap, C.t_meas_ps, nullptr);
    if (out != STEP_ALIVE) break;
    if ((p.e & 1023u) == 0u && globaltimer_ns() > deadline) {
      atomicOr(A.flags, 1);
      out = STEP_TRUNCATED;
      break;
    }
  }
  transient_finish(p, out, idx, A);
}

#endif  // MCBTE_F64
#if MCBTE_F32
// Particle state between time windows, 48 bytes: {x, t}, {u, d_rel},
// {event index, bin | sign bit, next measurement index | live bit, d2}
// (transient runs have no N_scat^max, so the relaxation count is not kept).
// Streaming (evict-first) accesses keep the window's tally slice in L2.
constexpr uint32_t kLive = 0x80000000u;

__device__ __forceinline__ void save_state(uint4* st, uint64_t idx, const Particle<float>& p) {
  uint4* q = st + idx * 3;
  __stcs(q + 0, make_uint4(__float_as_uint(p.x[0]), __float_as_uint(p.x[1]), __float_as_uint(p.x[2]),
                           __float_as_uint(p.t)));
  __stcs(q + 1, make_uint4(__float_as_uint(p.u[0]), __float_as_uint(p.u[1]), __float_as_uint(p.u[2]),
                           __float_as_uint(p.d_rel)));
  __stcs(q + 2, make_uint4(p.e, (uint32_t)p.bin | (p.s < 0.0f ? 0x80000000u : 0u), (uint32_t)p.mi | kLive,
                           __float_as_uint(p.d2)));
}

__device__ __forceinline__ void mark_done(uint4* st, uint64_t idx) { __stcs(st + idx * 3 + 2, make_uint4(0, 0, 0, 0)); }

// false: the particle ended in an earlier window, or it has nothing to
// sample before `win_end` (then its saved state stays as it is)
__device__ __forceinline__ bool load_state(const uint4* st, uint64_t idx, Particle<float>& p, const MatView& M,
                                           const float4* binf, const RunCfg& C) {
  const uint4* q = st + idx * 3;
  const uint4 c = __ldcs(q + 2);
  if (!(c.z & kLive)) return false;
  if (!C.win_last && (int)(c.z & ~kLive) >= C.win_end) return false;
  const uint4 a = __ldcs(q + 0);
  const uint4 b = __ldcs(q + 1);
  p.x[0] = __uint_as_float(a.x);
  p.x[1] = __uint_as_float(a.y);
  p.x[2] = __uint_as_float(a.z);
  p.t = __uint_as_float(a.w);
  p.u[0] = __uint_as_float(b.x);
  p.u[1] = __uint_as_float(b.y);
  p.u[2] = __uint_as_float(b.z);
  p.d_rel = __uint_as_float(b.w);
  p.e = c.x;
  p.bin = (int)(c.y & 0x7fffffffu);
  p.s = (c.y & 0x80000000u) ? -1.0f : 1.0f;
  p.mi = (int)(c.z & ~kLive);
  p.d2 = __uint_as_float(c.w);
  p.n_relax = 0;
  p.pid = (uint32_t)idx;
  p.g = 0;
  load_bin(p, M, binf);
  return true;
}

// Snapshots of a warp's flights, shared out over its 32 lanes.  Lane i
// takes k_i snapshots this step (measurement indices p.mi .. p.mi + k_i - 1
// of the flight that starts at p.x at time p.t); a lane's count depends on
// its flight's length, so a per-lane loop would leave most lanes idle while
// the longest flights sample.  Here the warp's k_1 + ... + k_32 snapshots are
// taken 32 at a time: each lane finds the owner of its snapshot by a binary
// search of the inclusive prefix sums and reads the owner's state by
// shuffles.  Every lane of the warp must call this (k = 0 for idle lanes).
// The arithmetic per snapshot is the per-lane loop's (Eq. sampling, Sec. 3.4).
__device__ __forceinline__ void warp_snapshots(int k, const Particle<float>& p, const float* tmeas, const float* cinv,
                                               const RunCfg& C, double* snap) {
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = (int)(threadIdx.x & 31u);
  int incl = k;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kAll, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(kAll, incl, 31);
  const int nx = C.grid[0], ny = C.grid[1], nz = C.grid[2];
  const size_t ncell = (size_t)nx * ny * nz;
  for (int base = 0; base < total; base += 32) {
    const int j = base + lane;
    // owner: the first lane whose inclusive sum exceeds j (always in 0..31)
    int own = 0;
#pragma unroll
    for (int st = 16; st >= 1; st >>= 1) {
      const int v = __shfl_sync(kAll, incl, own + st - 1);
      if (v <= j) own += st;
    }
    const int first = __shfl_sync(kAll, incl - k, own);
    const int mi0 = __shfl_sync(kAll, p.mi, own);
    const float x0 = __shfl_sync(kAll, p.x[0], own), x1 = __shfl_sync(kAll, p.x[1], own),
                x2 = __shfl_sync(kAll, p.x[2], own);
    const float u0 = __shfl_sync(kAll, p.u[0], own), u1 = __shfl_sync(kAll, p.u[1], own),
                u2 = __shfl_sync(kAll, p.u[2], own);
    const float t0 = __shfl_sync(kAll, p.t, own), v = __shfl_sync(kAll, p.v, own),
                s = __shfl_sync(kAll, p.s, own);
    if (j < total) {
      const int m = mi0 + (j - first);
      const float dist = v * (tmeas[m] - t0);
      const float pm0 = x0 + dist * u0, pm1 = x1 + dist * u1, pm2 = x2 + dist * u2;
      const int ix = min(max((int)floorf(pm0 * cinv[0]), 0), nx - 1);
      const int iy = min(max((int)floorf(pm1 * cinv[1]), 0), ny - 1);
      const int iz = min(max((int)floorf(pm2 * cinv[2]), 0), nz - 1);
      const size_t c = ((size_t)m * ncell + ((size_t)iz * ny + iy) * nx + ix) * 4;
      long long* q = reinterpret_cast<long long*>(snap) + c;
      const float sv = s * v;
      red_s64(q + 0, s > 0.0f ? 1ll : -1ll);
      if (v < 1024.0f) {
        red_s64(q + 1, (long long)__float2int_rn((sv * u0) * kFx));
        red_s64(q + 2, (long long)__float2int_rn((sv * u1) * kFx));
        red_s64(q + 3, (long long)__float2int_rn((sv * u2) * kFx));
      } else {
        red_s64(q + 1, fx(sv * u0));
        red_s64(q + 2, fx(sv * u1));
        red_s64(q + 3, fx(sv * u2));
      }
    }
  }
}

// Time-bin averages of a warp's flights, shared out over its 32 lanes in the
// same way: lane i contributes to the k_i bins m = p.mi .. p.mi + k_i - 1
// that its flight [p.t, t_end) overlaps; each (flight, bin) pair is one item,
// and the warp takes its items 32 at a time, every lane walking its item's
// piece of flight through the detector grids (region_track) with the
// owner's state read by shuffles.  Every lane of the warp must call this.
// The arithmetic per item is the per-lane loop's in step_transient.
__device__ __forceinline__ void warp_bin_averages(int k, float t_end, const Particle<float>& p, const float* tmeas,
                                                  const RunCfg& C, double* snap) {
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = (int)(threadIdx.x & 31u);
  int incl = k;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kAll, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(kAll, incl, 31);
  for (int base = 0; base < total; base += 32) {
    const int j = base + lane;
    int own = 0;
#pragma unroll
    for (int st = 16; st >= 1; st >>= 1) {
      const int v = __shfl_sync(kAll, incl, own + st - 1);
      if (v <= j) own += st;
    }
    const int first = __shfl_sync(kAll, incl - k, own);
    const int mi0 = __shfl_sync(kAll, p.mi, own);
    const float x[3] = {__shfl_sync(kAll, p.x[0], own), __shfl_sync(kAll, p.x[1], own),
                        __shfl_sync(kAll, p.x[2], own)};
    const float u0 = __shfl_sync(kAll, p.u[0], own), u1 = __shfl_sync(kAll, p.u[1], own),
                u2 = __shfl_sync(kAll, p.u[2], own);
    const float t0 = __shfl_sync(kAll, p.t, own), te = __shfl_sync(kAll, t_end, own),
                v = __shfl_sync(kAll, p.v, own), s = __shfl_sync(kAll, p.s, own);
    if (j < total) {
      const int m = mi0 + (j - first);
      const float b0 = m == 0 ? 0.0f : tmeas[m - 1];
      const float b1 = tmeas[m];
      const float ta = t0 > b0 ? t0 : b0;
      const float tb = te < b1 ? te : b1;
      if (ta < tb) {
        const float wb = 1.0f / (b1 - b0);
        const float w3[3] = {v * u0, v * u1, v * u2};
        for (int r = 0; r < C.n_regs; ++r) {
          const DetRegion& reg = C.regs[r];
          const size_t base_c = (size_t)m * C.n_det + reg.off;
          region_track<float>(reg, x, w3, t0, ta, tb, [&](uint32_t det, float dur) {
            long long* q = reinterpret_cast<long long*>(snap) + (base_c + det) * 4;
            const float f = (s * dur) * wb;
            red_s64(q + 0, fx(f));
            red_s64(q + 1, fx((f * v) * u0));
            red_s64(q + 2, fx((f * v) * u1));
            red_s64(q + 3, fx((f * v) * u2));
          });
        }
      }
    }
  }
}

// Shared memory: the measurement times as float (always), then the relaxation
// alias records and per-bin constants where the plan has room.
// TAVG: the run tallies time-bin averages (compiled apart, so that the
// snapshot variant carries none of that code).
template <int TPB, bool EXT, bool TAVG>
__global__ void __launch_bounds__(TPB, 1) k_transient_f32(const GeoRun* __restrict__ geos, MatView M, RunCfg C,
                                                          Acc A, SmemPlan S) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* sp = smem;
  const int n = M.n;
  const uint4* relax = M.rec_relax;
  const float4* binf = M.binf;
  float* tmeas = reinterpret_cast<float*>(sp);
  for (int i = threadIdx.x; i < C.n_times; i += TPB) tmeas[i] = (float)C.t_meas_ps[i];
  sp += ((size_t)C.n_times * sizeof(float) + 15) & ~(size_t)15;
  if (S.relax_in_smem) {
    uint4* t = reinterpret_cast<uint4*>(sp);
    for (int i = threadIdx.x; i < n; i += TPB) t[i] = M.rec_relax[i];
    relax = t;
    sp += (size_t)n * sizeof(uint4);
  }
  if (S.binf_in_smem) {
    float4* t = reinterpret_cast<float4*>(sp);
    for (int i = threadIdx.x; i < n; i += TPB) t[i] = M.binf[i];
    binf = t;
  }
  __syncthreads();
  const GeoRun& G = geos[0];
  float cinv[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) cinv[a] = (float)((double)C.grid[a] / G.L[a]);
  const uint64_t deadline = *C.t0 + C.budget_ns;
  const unsigned lane = threadIdx.x & 31u;
  const uint2 key = run_key(C);
  WarpRun run;   // the warp's particle indices not yet handed out
  Particle<float> p;
  bool alive = false;
  bool drained = false;   // as in the steady tracer: idle lanes stay until the warp is drained
  uint64_t idx = 0;
  constexpr unsigned kAll = 0xffffffffu;
  if (TAVG || C.n_regs == 0) {
    // Snapshots on the whole-box grid: every lane of a warp runs every step
    // (no lane skips ahead to the next refill), so that the warp can share
    // out its snapshots (warp_snapshots).  Flight and event as in
    // step_transient.
    for (;;) {
      if (__all_sync(kAll, drained)) break;
      const unsigned need = __ballot_sync(kAll, !alive && !drained);
      if (need) {
        const uint64_t k = run.take(need, lane, A.work, C.total, C.take_chunk, deadline, A.flags);
        if (!alive && !drained) {
          idx = k;
          if (idx >= C.total || (*(volatile int*)A.flags & 1)) {
            drained = true;
          } else if (C.win_first) {
            p.pid = (uint32_t)idx;
            p.g = 0;
            emit<float, EXT>(p, G, M, M.rec_emit, M.rec_init, binf, key.x, key.y, true, (float)C.t_max_ps);
            transient_start(p, C);
            if (!C.win_last && p.mi >= C.win_end) save_state(A.tstate, idx, p);   // emitted after this window
            else alive = true;
          } else if (load_state(A.tstate, idx, p, M, binf, C)) {
            alive = true;
          }
        }
      }
      // the flight: nearest of t_max, the clocks and the boundary (Sec. 3.3,
      // Sec. 3.5.6), and how many measurement times it covers
      int out = STEP_ALIVE, k = 0, face = 0, mi_next = 0;
      bool fin = false, rlx = false, rlx2 = false;
      float seg = 0.0f, t_end = 0.0f;
      if (alive) {
        if (p.e + 1u >= C.max_events) {
          out = STEP_TRUNCATED;
        } else {
          float db;
          first_hit<float, EXT>(G, p.x, p.u, &db, &face);
          const float tmax = (float)C.t_max_ps;
          const float d_end = (tmax - p.t) * p.v;
          if (d_end <= p.d_rel && d_end <= db && (!EXT || d_end <= p.d2)) { fin = true; seg = d_end; }
          else if (p.d_rel < db && (!EXT || p.d_rel <= p.d2)) { rlx = true; seg = p.d_rel; }
          else if (EXT && p.d2 < db) { rlx2 = true; seg = p.d2; }
          else { seg = db; }
          t_end = fin ? tmax : p.t + seg * p.inv_v;
          if constexpr (TAVG) {
            // the bins [t_{m-1}, t_m) the flight overlaps: m = p.mi up to the
            // first m whose end t_m lies beyond t_end (the flight's last bin,
            // where the particle stays), by bisection
            int lo = p.mi, hi = C.n_times;
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (tmeas[mid] <= t_end) lo = mid + 1; else hi = mid;
            }
            mi_next = lo;
            k = p.mi < C.n_times ? (lo < C.n_times ? lo : C.n_times - 1) - p.mi + 1 : 0;
          } else {
            // the measurement times in [t, t_end) (closed at t_max): the first
            // index from p.mi on that is not covered, by bisection
            int lo = p.mi, hi = C.n_times;
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              const bool cov = fin ? (tmeas[mid] <= t_end) : (tmeas[mid] < t_end);
              if (cov) lo = mid + 1; else hi = mid;
            }
            k = lo - p.mi;
          }
        }
      }
      if constexpr (TAVG) warp_bin_averages(k, t_end, p, tmeas, C, A.snap);
      else warp_snapshots(k, p, tmeas, cinv, C, A.snap);
      if (!alive) continue;
      if (out == STEP_ALIVE) {
        if constexpr (TAVG) p.mi = mi_next;
        else p.mi += k;
        p.t = t_end;
#pragma unroll
        for (int a = 0; a < 3; ++a) p.x[a] = p.x[a] + seg * p.u[a];
        if (fin) {
          out = STEP_DONE;
        } else {
          GradOff off;
          out = apply_event<float, GradOff, TallyNone, EXT>(p, G, M, relax, binf, C, key.x, key.y, rlx, rlx2, face, seg,
                                                            TallyNone(), off, 0.0);
        }
      }
      if (out == STEP_ALIVE && (p.e & 255u) == 0u && globaltimer_ns() > deadline) {
        atomicOr(A.flags, 1);
        out = STEP_TRUNCATED;
      }
      if (out != STEP_ALIVE) {
        transient_finish(p, out, idx, A);
        if (!C.win_last) mark_done(A.tstate, idx);
        alive = false;
      } else if (!C.win_last && p.mi >= C.win_end) {
        save_state(A.tstate, idx, p);
        alive = false;
      }
    }
    return;
  }
  // snapshots into detector regions: the per-lane loop
  if constexpr (!TAVG) {
    for (;;) {
      if (__all_sync(kAll, drained)) break;
      const unsigned need = __ballot_sync(kAll, !alive && !drained);
      if (need) {
        const uint64_t k = run.take(need, lane, A.work, C.total, C.take_chunk, deadline, A.flags);
        if (!alive && !drained) {
          idx = k;
          if (idx >= C.total || (*(volatile int*)A.flags & 1)) {
            drained = true;
            continue;
          }
          if (C.win_first) {
            p.pid = (uint32_t)idx;
            p.g = 0;
            emit<float, EXT>(p, G, M, M.rec_emit, M.rec_init, binf, key.x, key.y, true, (float)C.t_max_ps);
            transient_start(p, C);
            if (!C.win_last && p.mi >= C.win_end) {   // emitted after this window's last snapshot
              save_state(A.tstate, idx, p);
              continue;
            }
          } else if (!load_state(A.tstate, idx, p, M, binf, C)) {
            continue;
          }
          alive = true;
        }
      }
      if (!alive) continue;
      int out = step_transient<float, EXT>(p, G, M, relax, binf, C, key.x, key.y, A.snap, tmeas, cinv);
      if (out == STEP_ALIVE && (p.e & 255u) == 0u && globaltimer_ns() > deadline) {
        atomicOr(A.flags, 1);
        out = STEP_TRUNCATED;
      }
      if (out != STEP_ALIVE) {
        transient_finish(p, out, idx, A);
        if (!C.win_last) mark_done(A.tstate, idx);
        alive = false;
      } else if (!C.win_last && p.mi >= C.win_end) {
        // this window's snapshots are taken: park the particle at its event
        save_state(A.tstate, idx, p);
        alive = false;
      }
    }
  }
}

#endif  // MCBTE_F32
#if MCBTE_F64
// Scale the raw snapshot sums: T = s E_eff / (C V_cell), q = s E_eff V_g / V_cell.
// `fixed`: the sums are the FP32 path's integers (signed count; flux in
// 2^-20 nm/ps units), converted here in place.
__global__ void k_finalize_transient(const GeoRun* geos, MatView M, RunCfg C, Acc A, double* tally, double* stats,
                                     size_t n_cells_total, int fixed) {
  const GeoRun& G = geos[0];
  const double E_eff = G.E_tot / (double)G.n;
  const double Vc = G.V_box / (double)((size_t)C.grid[0] * C.grid[1] * C.grid[2]);
  const size_t total = (size_t)C.n_times * n_cells_total;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    // volume of this entry's detector (its region's split, or the grid cell)
    double vd = Vc;
    if (C.n_regs > 0) {
      const uint32_t det = (uint32_t)(i % n_cells_total);
      for (int k = 0; k < C.n_regs; ++k)
        if (det >= C.regs[k].off) vd = C.regs[k].v_det;
    }
    const double kT = E_eff / (M.sums[0] * vd);
    const double kq = E_eff / vd;
    const double* r = A.snap + i * 4;
    double* o = tally + i * 4;
    double a0, a1, a2, a3;
    if (fixed) {
      const long long* q = reinterpret_cast<const long long*>(r);
      a0 = C.time_average ? (double)q[0] * kFxInv : (double)q[0];
      a1 = (double)q[1] * kFxInv;
      a2 = (double)q[2] * kFxInv;
      a3 = (double)q[3] * kFxInv;
    } else {
      a0 = r[0];
      a1 = r[1];
      a2 = r[2];
      a3 = r[3];
    }
    o[0] = kT * a0;
    o[1] = (kq * a1) * 1e3;
    o[2] = (kq * a2) * 1e3;
    o[3] = (kq * a3) * 1e3;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // fold the copies of the run counters
    unsigned long long c[4] = {0ull, 0ull, 0ull, 0ull};
    double d[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int r = 0; r < kSumCopies; ++r) {
      c[0] += A.cnt[r * 4 + 0];
      c[1] += A.cnt[r * 4 + 1];
      c[2] = c[2] > A.cnt[r * 4 + 2] ? c[2] : A.cnt[r * 4 + 2];
      c[3] += A.cnt[r * 4 + 3];
      for (int k = 0; k < 8; ++k) d[k] += A.dsc[r * 8 + k];
    }
    for (int k = 0; k < MCBTE_NSTATS; ++k) stats[k] = 0.0;
    stats[MCBTE_STAT_EVENTS] = (double)c[0];
    stats[MCBTE_STAT_TRUNCATED] = (double)c[1];
    stats[MCBTE_STAT_MAX_EVENTS] = (double)c[2];
    stats[MCBTE_STAT_N] = (double)c[3];
    stats[MCBTE_STAT_E_TOT] = G.E_tot;
    stats[MCBTE_STAT_SIGNED_EMITTED] = d[2];
    stats[MCBTE_STAT_SIGNED_ABSORBED] = d[3];
    stats[MCBTE_STAT_ABSORBED] = d[7];
    stats[MCBTE_STAT_STATUS] = (A.flags[0] & 1) ? (double)MCBTE_ERR_TIMEOUT
                                                : (c[1] ? (double)MCBTE_WARN_TRUNCATED : 0.0);
  }
}

#endif  // MCBTE_F64
}  // namespace

#if MCBTE_F64
cudaError_t launch_transient(int precision, const GeoRun* geos, const MatView& M, const RunCfg& C, const Acc& A,
                             int threads, int bps, cudaStream_t s) {
  if (precision == MCBTE_FP64_PLAIN) {
    const uint64_t blocks = (C.total + 255) / 256;
    k_transient_fp64<<<(unsigned)blocks, 256, 0, s>>>(geos, M, C, A);
    return cudaGetLastError();
  }
  return launch_transient_f32(geos, M, C, A, threads > 0 ? threads : 1024, bps, s);
}

#endif  // MCBTE_F64
#if MCBTE_F32
namespace {
template <int TPB, bool EXT, bool TAVG>
cudaError_t launch_transient_tav(const GeoRun* geos, const MatView& M, const RunCfg& C, const Acc& A, int bps,
                                 cudaStream_t s) {
  const size_t tm_bytes = ((size_t)C.n_times * sizeof(float) + 15) & ~(size_t)15;
  SmemPlan S = plan_smem_f32(M.n, 1, 0, 0, 200 * 1024 - tm_bytes);
  S.bytes += tm_bytes;
  auto kern = k_transient_f32<TPB, EXT, TAVG>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.bytes);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TPB, S.bytes);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int b = (bps > 0 && bps < occ) ? bps : occ;
  kern<<<sm_count() * b, TPB, S.bytes, s>>>(geos, M, C, A, S);
  return cudaGetLastError();
}
template <int TPB, bool EXT>
cudaError_t launch_transient_tpb(const GeoRun* geos, const MatView& M, const RunCfg& C, const Acc& A, int bps,
                                 cudaStream_t s) {
  return C.time_average ? launch_transient_tav<TPB, EXT, true>(geos, M, C, A, bps, s)
                        : launch_transient_tav<TPB, EXT, false>(geos, M, C, A, bps, s);
}
}  // namespace

cudaError_t launch_transient_f32(const GeoRun* geos, const MatView& M, const RunCfg& C, const Acc& A, int threads,
                                 int bps, cudaStream_t s) {
  const bool imp = C.ext != 0;   // the extended physics is compiled in only when used
  switch (threads) {
    case 256: return imp ? launch_transient_tpb<256, true>(geos, M, C, A, bps, s)
                         : launch_transient_tpb<256, false>(geos, M, C, A, bps, s);
    case 512: return imp ? launch_transient_tpb<512, true>(geos, M, C, A, bps, s)
                         : launch_transient_tpb<512, false>(geos, M, C, A, bps, s);
    case 768: return imp ? launch_transient_tpb<768, true>(geos, M, C, A, bps, s)
                         : launch_transient_tpb<768, false>(geos, M, C, A, bps, s);
    case 1024: return imp ? launch_transient_tpb<1024, true>(geos, M, C, A, bps, s)
                          : launch_transient_tpb<1024, false>(geos, M, C, A, bps, s);
    default: return cudaErrorInvalidValue;
  }
}

#endif  // MCBTE_F32
#if MCBTE_F64
cudaError_t launch_finalize_transient(const GeoRun* geos, const MatView& M, const RunCfg& C, const Acc& A,
                                      double* tally, double* stats, size_t n_cells_total, bool fixed,
                                      cudaStream_t s) {
  k_finalize_transient<<<sm_count() * 4, 256, 0, s>>>(geos, M, C, A, tally, stats, n_cells_total, fixed ? 1 : 0);
  return cudaGetLastError();
}

#endif  // MCBTE_F64

}  // namespace mcbte
