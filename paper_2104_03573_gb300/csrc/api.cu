// C ABI of the MCBTE GB300 library: handle management, argument checks,
// workspace layout and the launch sequence of every run.  No numerical step
// of the method runs here; this file only validates, lays out memory and
// launches kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "launch.h"

using namespace mcbte;

namespace {

thread_local std::string g_err;

mcbte_status fail(mcbte_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

// Caller-owned timing event around the trace kernel. Inside a stream capture
// it becomes an external event-record node, so that it fires at every replay
// of the graph; outside a capture it is a plain record.
cudaError_t record_trace_event(void* ev, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) return e;
  if (cs == cudaStreamCaptureStatusActive)
    return cudaEventRecordWithFlags((cudaEvent_t)ev, s, cudaEventRecordExternal);
  return cudaEventRecord((cudaEvent_t)ev, s);
}

mcbte_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? MCBTE_ERR_OOM : MCBTE_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(call)                                 \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// Bump allocator over one device buffer (256-byte aligned pieces).
struct Carve {
  size_t off = 0;
  char* base = nullptr;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// Small host data (detector regions, measurement times) reaches the device
// as kernel parameters, 4000 bytes per launch: the parameters are copied
// when the launch is issued, so the host buffer may go away at once, and a
// stream capture records the bytes themselves (a copy from host memory would
// record the host address, read again at every replay).
constexpr unsigned kParamChunk = 4000;
struct ParamChunk {
  unsigned char b[kParamChunk];
};

__global__ void k_param_copy(unsigned char* dst, ParamChunk c, unsigned n) {
  for (unsigned i = threadIdx.x; i < n; i += blockDim.x) dst[i] = c.b[i];
}

cudaError_t param_upload(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  const unsigned char* from = static_cast<const unsigned char*>(src);
  unsigned char* to = static_cast<unsigned char*>(dst);
  for (size_t off = 0; off < bytes; off += kParamChunk) {
    const unsigned n = (unsigned)std::min<size_t>(kParamChunk, bytes - off);
    ParamChunk c;
    std::memcpy(c.b, from + off, n);
    k_param_copy<<<1, 256, 0, s>>>(to + off, c, n);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

struct mcbte_material {
  int n;
  void* block;
  MatView view;
  MatBuild b;
};

struct mcbte_geometry {
  mcbte_geometry_desc host;
  mcbte_geometry_desc* dev;
};

extern "C" {

int mcbte_last_error(char* buf, size_t n) {
  if (buf && n > 0) {
    size_t k = g_err.size() < n - 1 ? g_err.size() : n - 1;
    std::memcpy(buf, g_err.data(), k);
    buf[k] = '\0';
  }
  return (int)g_err.size();
}

int mcbte_version(void) { return 10000; }

// ------------------------------------------------------------------ material
mcbte_status mcbte_material_create(const mcbte_material_desc* d, mcbte_material** out) {
  if (!d || !out) return fail(MCBTE_ERR_INVALID_ARG, "material_create: null argument");
  *out = nullptr;
  const int n = d->n_bins;
  if (n < 1 || n > (1 << 24)) return fail(MCBTE_ERR_INVALID_ARG, "material_create: n_bins out of range");
  if (!d->omega || !d->v || !d->tau) return fail(MCBTE_ERR_INVALID_ARG, "material_create: omega, v, tau required");
  const bool fmt2 = d->C != nullptr;
  if (!fmt2 && (!d->D || !d->domega))
    return fail(MCBTE_ERR_INVALID_ARG, "material_create: give C (format 2) or D and domega (format 1)");
  if (!fmt2 && !finite_pos(d->T_lin)) return fail(MCBTE_ERR_INVALID_ARG, "material_create: T_lin must be > 0");
  for (int i = 0; i < n; ++i) {
    if (!finite_pos(d->v[i])) return fail(MCBTE_ERR_INVALID_ARG, "material_create: v must be > 0");
    if (!finite_pos(d->tau[i])) return fail(MCBTE_ERR_INVALID_ARG, "material_create: tau must be > 0");
    if (!std::isfinite(d->omega[i]) || d->omega[i] <= 0.0)
      return fail(MCBTE_ERR_INVALID_ARG, "material_create: omega must be > 0");
    if (fmt2 && !(std::isfinite(d->C[i]) && d->C[i] >= 0.0))
      return fail(MCBTE_ERR_INVALID_ARG, "material_create: C must be >= 0");
    if (!fmt2 && !(std::isfinite(d->D[i]) && d->D[i] >= 0.0 && std::isfinite(d->domega[i]) && d->domega[i] >= 0.0))
      return fail(MCBTE_ERR_INVALID_ARG, "material_create: D and domega must be >= 0");
    if (d->tau_imp && !(d->tau_imp[i] > 0.0))
      return fail(MCBTE_ERR_INVALID_ARG, "material_create: tau_imp must be > 0 (+inf: no two-phonon scattering)");
    if (d->spec_bin && !(d->spec_bin[i] >= 0.0 && d->spec_bin[i] <= 1.0))
      return fail(MCBTE_ERR_INVALID_ARG, "material_create: spec_bin must be in [0, 1]");
  }
  Carve c;
  auto layout = [&](MatBuild& b) {
    b.n = n;
    double* omega = c.take<double>(n);
    double* v = c.take<double>(n);
    double* tau = c.take<double>(n);
    double* Cin = c.take<double>(n);
    double* D = c.take<double>(n);
    double* dw = c.take<double>(n);
    b.omega = omega; b.v = v; b.tau = tau;
    b.C_in = fmt2 ? Cin : nullptr;
    b.D = D; b.domega = dw;
    b.T_lin = d->T_lin;
    b.C = c.take<double>(n);
    b.w_emit = c.take<double>(n);
    b.w_init = c.take<double>(n);
    b.w_relax = c.take<double>(n);
    b.v_nm = c.take<double>(n);
    b.inv_v = c.take<double>(n);
    b.lam = c.take<double>(n);
    b.pi = c.take<double>(n);
    b.lam2 = c.take<double>(n);
    double* ti = c.take<double>(n);
    b.tau_imp = d->tau_imp ? ti : nullptr;
    double* sb = c.take<double>(n);
    b.spec_bin = d->spec_bin ? sb : nullptr;
    b.spec_thr = c.take<uint64_t>(n);
    b.sums = c.take<double>(4);
    b.prob = c.take<double>(3 * (size_t)n);
    b.thr = c.take<uint64_t>(3 * (size_t)n);
    b.alias = c.take<int32_t>(3 * (size_t)n);
    b.rec = c.take<uint4>(3 * (size_t)n);
    b.binf = c.take<float4>(n);
    b.scratch_p = c.take<double>(3 * (size_t)n);
    b.scratch_small = c.take<int>(3 * (size_t)n);
    b.scratch_large = c.take<int>(3 * (size_t)n);
  };
  MatBuild probe{};
  layout(probe);
  const size_t bytes = c.off;
  void* block = nullptr;
  // stream-ordered pool allocation (a plain cudaMalloc costs far more than
  // the table build for a few thousand bins)
  CUDA_TRY(cudaMallocAsync(&block, bytes, 0));
  c.off = 0;
  c.base = static_cast<char*>(block);
  MatBuild b{};
  layout(b);
  auto cleanup = [&]() {
    cudaFreeAsync(block, 0);
    cudaStreamSynchronize(0);
  };
  const size_t nb = (size_t)n * sizeof(double);
  cudaError_t e = cudaMemcpy((void*)b.omega, d->omega, nb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy((void*)b.v, d->v, nb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy((void*)b.tau, d->tau, nb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && d->tau_imp) e = cudaMemcpy((void*)b.tau_imp, d->tau_imp, nb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && d->spec_bin) e = cudaMemcpy((void*)b.spec_bin, d->spec_bin, nb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && fmt2) e = cudaMemcpy((void*)b.C_in, d->C, nb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !fmt2) e = cudaMemcpy((void*)b.D, d->D, nb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !fmt2) e = cudaMemcpy((void*)b.domega, d->domega, nb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_material_build(b, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  double sums[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(sums, b.sums, 3 * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "material_create");
  }
  if (!(sums[0] > 0.0) || !(sums[2] > 0.0)) {
    cleanup();
    return fail(MCBTE_ERR_INVALID_ARG, "material_create: total heat capacity is zero");
  }
  mcbte_material* m = new mcbte_material();
  m->n = n;
  m->block = block;
  m->b = b;
  MatView& v = m->view;
  v.n = n;
  v.rec_emit = b.rec;
  v.rec_init = b.rec + n;
  v.rec_relax = b.rec + 2 * (size_t)n;
  v.binf = b.binf;
  v.v_d = b.v_nm;
  v.inv_v_d = b.inv_v;
  v.lam_d = b.lam;
  v.pi = b.pi;
  v.sums = b.sums;
  v.lam2_d = b.lam2;
  v.imp = d->tau_imp ? 1 : 0;
  v.spec_thr = d->spec_bin ? b.spec_thr : nullptr;
  *out = m;
  return MCBTE_OK;
}

void mcbte_material_destroy(mcbte_material* m) {
  if (!m) return;
  // the block returns to the pool once the work queued before this call is done
  cudaDeviceSynchronize();
  cudaFreeAsync(m->block, 0);
  cudaStreamSynchronize(0);
  delete m;
}

int mcbte_material_n_bins(const mcbte_material* m) { return m ? m->n : 0; }

mcbte_status mcbte_material_tables(const mcbte_material* m, double* C, double* prob, uint64_t* thr, int32_t* alias,
                                   double* sums) {
  if (!m) return fail(MCBTE_ERR_INVALID_ARG, "material_tables: null material");
  const size_t n = (size_t)m->n;
  if (C) CUDA_TRY(cudaMemcpy(C, m->b.C, n * sizeof(double), cudaMemcpyDeviceToHost));
  if (prob) CUDA_TRY(cudaMemcpy(prob, m->b.prob, 3 * n * sizeof(double), cudaMemcpyDeviceToHost));
  if (thr) CUDA_TRY(cudaMemcpy(thr, m->b.thr, 3 * n * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  if (alias) CUDA_TRY(cudaMemcpy(alias, m->b.alias, 3 * n * sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (sums) CUDA_TRY(cudaMemcpy(sums, m->b.sums, 3 * sizeof(double), cudaMemcpyDeviceToHost));
  return MCBTE_OK;
}

// ------------------------------------------------------------------ geometry
mcbte_status mcbte_geometry_create(const mcbte_geometry_desc* d, mcbte_geometry** out) {
  if (!d || !out) return fail(MCBTE_ERR_INVALID_ARG, "geometry_create: null argument");
  *out = nullptr;
  for (int a = 0; a < 3; ++a)
    if (!finite_pos(d->L[a])) return fail(MCBTE_ERR_INVALID_ARG, "geometry_create: L must be > 0");
  for (int f = 0; f < 6; ++f) {
    if (d->face_type[f] < 0 || d->face_type[f] > 2) return fail(MCBTE_ERR_INVALID_ARG, "geometry_create: face type");
    if (d->face_type[f] == MCBTE_FACE_ADIABATIC && !(d->face_p[f] <= 1.0))   // < 0: per-bin d(omega)
      return fail(MCBTE_ERR_INVALID_ARG, "geometry_create: specularity above 1");
    if (d->face_type[f] == MCBTE_FACE_ISOTHERMAL && !finite_pos(d->face_T[f]))
      return fail(MCBTE_ERR_INVALID_ARG, "geometry_create: isothermal T_b must be > 0");
  }
  const int lo[3] = {3, 0, 4}, hi[3] = {1, 2, 5};
  for (int a = 0; a < 3; ++a) {
    const bool pl = d->face_type[lo[a]] == MCBTE_FACE_PERIODIC, ph = d->face_type[hi[a]] == MCBTE_FACE_PERIODIC;
    if (pl != ph) return fail(MCBTE_ERR_INVALID_ARG, "geometry_create: periodic faces must come in pairs");
  }
  if (!finite_pos(d->T_eq)) return fail(MCBTE_ERR_INVALID_ARG, "geometry_create: T_eq must be > 0");
  int ng = 0;
  for (int a = 0; a < 3; ++a) {
    if (!std::isfinite(d->grad_T[a])) return fail(MCBTE_ERR_INVALID_ARG, "geometry_create: grad_T not finite");
    if (d->grad_T[a] != 0.0) ++ng;
  }
  (void)ng;   // any direction (Sec. 3.2.3); a single component keeps the axis-aligned emission
  if (d->pore) {
    const double r = d->pore_r, cx = d->pore_c[0], cy = d->pore_c[1];
    if (!finite_pos(r) || !(cx - r > 0.0) || !(cx + r < d->L[0]) || !(cy - r > 0.0) || !(cy + r < d->L[1]))
      return fail(MCBTE_ERR_INVALID_ARG, "geometry_create: pore must lie strictly inside the cell");
    if (!(d->pore_p >= 0.0 && d->pore_p <= 1.0))
      return fail(MCBTE_ERR_INVALID_ARG, "geometry_create: pore specularity outside [0,1]");
    if (3.141592653589793 * r * r > 0.9 * d->L[0] * d->L[1])
      return fail(MCBTE_ERR_INVALID_ARG, "geometry_create: porosity above 0.9");
  }
  if (d->gauss && !finite_pos(d->gauss_sigma))
    return fail(MCBTE_ERR_INVALID_ARG, "geometry_create: gauss_sigma must be > 0");
  if (d->n_inner < 0 || d->n_inner > MCBTE_MAX_INNER)
    return fail(MCBTE_ERR_INVALID_ARG, "geometry_create: n_inner in [0, MCBTE_MAX_INNER]");
  for (int k = 0; k < d->n_inner; ++k) {
    const double* s4 = d->inner[k];
    for (int c = 0; c < 4; ++c)
      if (!(std::isfinite(s4[c]) && s4[c] >= 0.0 && s4[c] <= d->L[c & 1]))
        return fail(MCBTE_ERR_INVALID_ARG, "geometry_create: internal walls must lie in the cell");
    if (s4[0] == s4[2] && s4[1] == s4[3]) return fail(MCBTE_ERR_INVALID_ARG, "geometry_create: empty internal wall");
    const double nn = d->inner_n[k][0] * d->inner_n[k][0] + d->inner_n[k][1] * d->inner_n[k][1];
    if (!(std::fabs(nn - 1.0) < 1e-9)) return fail(MCBTE_ERR_INVALID_ARG, "geometry_create: wall normals must be unit");
    if (!(d->inner_p[k] <= 1.0)) return fail(MCBTE_ERR_INVALID_ARG, "geometry_create: wall specularity above 1");
  }
  mcbte_geometry_desc* dev = nullptr;
  CUDA_TRY(cudaMalloc(&dev, sizeof(mcbte_geometry_desc)));
  cudaError_t e = cudaMemcpy(dev, d, sizeof(mcbte_geometry_desc), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(dev);
    return cuda_fail(e, "geometry_create");
  }
  mcbte_geometry* g = new mcbte_geometry();
  g->host = *d;
  g->dev = dev;
  *out = g;
  return MCBTE_OK;
}

void mcbte_geometry_destroy(mcbte_geometry* g) {
  if (!g) return;
  cudaFree(g->dev);
  delete g;
}

}  // extern "C"

// ------------------------------------------------------------------ steady runs
namespace {

bool has_isothermal_source(const mcbte_geometry_desc& d) {
  for (int f = 0; f < 6; ++f)
    if (d.face_type[f] == MCBTE_FACE_ISOTHERMAL && d.face_T[f] != d.T_eq) return true;
  return false;
}

// A face or internal wall that takes the material's per-bin specularity.
bool uses_spec_bin(const mcbte_geometry_desc& d) {
  for (int f = 0; f < 6; ++f)
    if (d.face_type[f] == MCBTE_FACE_ADIABATIC && d.face_p[f] < 0.0) return true;
  for (int k = 0; k < d.n_inner; ++k)
    if (d.inner_p[k] < 0.0) return true;
  return false;
}

// The run needs the tracers' extended paths: a two-phonon clock, internal
// walls, per-bin specularity or a control gradient off the axes.
bool uses_ext(const mcbte_material* m, const mcbte_geometry_desc& d) {
  int nz = 0;
  for (int a = 0; a < 3; ++a) nz += d.grad_T[a] != 0.0;
  return m->view.imp || d.n_inner > 0 || uses_spec_bin(d) || nz > 1;
}

// Detector regions (Sec. 4.5): validation and the device records, derived
// with the CPU reference's arithmetic.
mcbte_status check_regions(int n, const double* regions, const int* grid, const char* who) {
  if (n < 0 || n > MCBTE_MAX_REGIONS) return fail(MCBTE_ERR_INVALID_ARG, std::string(who) + ": n_regions in [0, 16]");
  if (n > 0 && (!regions || !grid)) return fail(MCBTE_ERR_INVALID_ARG, std::string(who) + ": regions and region_grid required");
  uint64_t nd = 0;
  for (int k = 0; k < n; ++k) {
    uint64_t cnt = 1;
    for (int a = 0; a < 3; ++a) {
      const double lo = regions[6 * k + 2 * a], hi = regions[6 * k + 2 * a + 1];
      const int g = grid[3 * k + a];
      if (!(std::isfinite(lo) && std::isfinite(hi) && hi > lo))
        return fail(MCBTE_ERR_INVALID_ARG, std::string(who) + ": region bounds must satisfy min < max");
      if (g < 1 || g > 4096) return fail(MCBTE_ERR_INVALID_ARG, std::string(who) + ": region_grid in [1, 4096]");
      cnt *= (uint64_t)g;
    }
    nd += cnt;
  }
  if (nd > (1ull << 28)) return fail(MCBTE_ERR_INVALID_ARG, std::string(who) + ": too many detectors");
  return MCBTE_OK;
}

uint64_t region_detectors(int n, const int* grid) {
  uint64_t nd = 0;
  for (int k = 0; k < n; ++k) nd += (uint64_t)grid[3 * k] * grid[3 * k + 1] * grid[3 * k + 2];
  return nd;
}

// Steady detector sums: one per detector, or one per detector and bin.
uint64_t steady_det_slots(const mcbte_steady_params* p, int n_bins) {
  return region_detectors(p->n_regions, p->region_grid) * (p->det_per_bin ? (uint64_t)n_bins : 1ull);
}

// Records of n regions (whole: the box split by `grid` as one region).
std::vector<DetRegion> build_regions(int n, const double* regions, const int* rgrid, bool whole, const int grid[3],
                                     const double Lbox[3]) {
  std::vector<DetRegion> rg(n);
  uint32_t off = 0;
  for (int k = 0; k < n; ++k) {
    DetRegion& r = rg[k];
    double vol = 1.0;
    int cnt = 1;
    for (int a = 0; a < 3; ++a) {
      const double lo_m = whole ? 0.0 : regions[6 * k + 2 * a];
      const double hi_m = whole ? Lbox[a] : regions[6 * k + 2 * a + 1];
      r.n[a] = whole ? grid[a] : rgrid[3 * k + a];
      r.hi_closed[a] = (hi_m * 1e9) >= (Lbox[a] * 1e9);
      r.lo[a] = lo_m * 1e9;
      r.hi[a] = hi_m * 1e9;
      r.h[a] = (r.hi[a] - r.lo[a]) / (double)r.n[a];
      r.lof[a] = (float)r.lo[a];
      r.hif[a] = (float)r.hi[a];
      r.cinvf[a] = (float)((double)r.n[a] / (r.hi[a] - r.lo[a]));
      vol = vol * (hi_m - lo_m);
      cnt *= r.n[a];
    }
    r.v_det = vol / (double)cnt;
    r.off = off;
    off += (uint32_t)cnt;
  }
  return rg;
}

bool has_gradient(const mcbte_geometry_desc& d) {
  return d.grad_T[0] != 0.0 || d.grad_T[1] != 0.0 || d.grad_T[2] != 0.0;
}

struct SteadyWs {
  GeoRun* geos;
  uint64_t* offs;
  char* zero_begin;
  double* cellP;
  double* cellD;
  double* qbin;
  long long* cellPq;
  long long* cellDq;
  long long* qbinq;
  double* dsc;
  unsigned long long* cnt;
  double* G;
  long long* Gq;
  double* gsum;
  unsigned long long* work;
  int* flags;
  unsigned long long* t0;
  unsigned long long* park_n;   // FP32 tail: particles parked, and taken by the tail kernel
  unsigned long long* park_rd;
  char* zero_end;
  double* dirs;
  double* dpi;
  // host-output staging
  double *T, *q, *q_bin, *stats;
  uint32_t* events_pp;
  double* X_pp;
  double *dk, *dkp, *dkdir;
  double* xrep;   // FP32 gradient: final tally of every particle (forward -> replay)
  DetRegion* regs;      // steady detector regions
  double* det_raw;      // [n_det][4] FP64 path sums (zeroed)
  long long* det_q;     // [n_det][4] FP32 path fixed-point sums (zeroed)
  double* det;          // host staging of the outputs
  double* nscat;        // [R][G][K + 1][4] N_scat_max curve sums, R = nscat_replicas (zeroed)
  double* kn;           // host staging of the curve
  unsigned char* park;  // FP32 tail: park_cap records of park_record_bytes() (last, not zeroed)
  uint64_t park_cap;
  size_t bytes;
};

// Records the FP32 steady tracer can park for its tail kernel: at most
// tail_max per resident warp of the main kernel (64 warps per SM), and never
// more than the run's particles.
uint64_t park_capacity(const mcbte_steady_params* p, uint64_t total) {
  if (p->precision != MCBTE_FP32_TRACE || p->tail_lanes < 0) return 0;
  const uint64_t tail = p->tail_lanes == 0 ? 8 : (uint64_t)p->tail_lanes;
  const uint64_t cap = (uint64_t)sm_count() * 64ull * tail;
  return cap < total ? cap : total;
}

// Copies of the N_scat_max curve sums: every relaxation adds to one of K + 1
// slots per geometry, and one copy for the whole grid serialises those
// same-address atomics in a few L2 slices.  Up to 64 copies (a power of
// two), fewer where the curve is long or the batch large, so that they stay
// within 8 MiB.
int nscat_replicas(int G, int K) {
  const size_t per = (size_t)G * (size_t)(K + 1) * 4 * sizeof(double);
  int r = 64;
  while (r > 1 && (size_t)r * per > ((size_t)8 << 20)) r >>= 1;
  return r;
}

SteadyWs layout_steady(char* base, int G, int n, int nc, uint64_t total, bool grad, bool replay, int nd,
                       bool host_out, bool want_ev, bool want_x, bool want_T, bool want_q, bool want_qbin,
                       uint64_t n_det = 0, int nscat = 0, uint64_t park_cap = 0) {
  Carve c;
  c.base = base;
  SteadyWs w{};
  w.geos = c.take<GeoRun>(G);
  w.offs = c.take<uint64_t>(G + 1);
  c.off = (c.off + 255) & ~(size_t)255;
  w.zero_begin = base ? base + c.off : nullptr;
  w.cellP = nc > 0 ? c.take<double>((size_t)G * nc * 4) : nullptr;
  w.cellD = nc > 0 ? c.take<double>((size_t)G * (nc + 1) * 4) : nullptr;
  w.qbin = c.take<double>((size_t)G * n);
  w.cellPq = nc > 0 ? c.take<long long>((size_t)G * nc * 4) : nullptr;
  w.cellDq = nc > 0 ? c.take<long long>((size_t)G * (nc + 1) * 4) : nullptr;
  w.qbinq = c.take<long long>((size_t)G * n);
  w.dsc = c.take<double>((size_t)G * 8);
  w.cnt = c.take<unsigned long long>((size_t)G * 4);
  w.G = grad ? c.take<double>(n) : nullptr;
  w.Gq = grad ? c.take<long long>(n) : nullptr;
  w.gsum = grad ? c.take<double>((size_t)kSumCopies * kGradStride) : nullptr;
  w.work = c.take<unsigned long long>(1);
  w.flags = c.take<int>(2);
  w.t0 = c.take<unsigned long long>(1);
  w.park_n = c.take<unsigned long long>(1);
  w.park_rd = c.take<unsigned long long>(1);
  w.det_raw = n_det ? c.take<double>(4 * n_det) : nullptr;
  w.det_q = n_det ? c.take<long long>(4 * n_det) : nullptr;
  w.nscat = nscat ? c.take<double>((size_t)nscat_replicas(G, nscat) * G * (size_t)(nscat + 1) * 4) : nullptr;
  c.off = (c.off + 255) & ~(size_t)255;
  w.zero_end = base ? base + c.off : nullptr;
  w.regs = n_det ? c.take<DetRegion>(MCBTE_MAX_REGIONS) : nullptr;
  w.det = (host_out && n_det) ? c.take<double>(4 * n_det) : nullptr;
  w.dirs = (grad && nd > 0) ? c.take<double>((size_t)nd * n) : nullptr;
  w.dpi = (grad && nd > 0) ? c.take<double>(nd) : nullptr;
  w.xrep = replay ? c.take<double>(total) : nullptr;
  if (host_out) {
    w.T = (want_T && nc > 0) ? c.take<double>((size_t)G * nc) : nullptr;
    w.q = (want_q && nc > 0) ? c.take<double>((size_t)G * nc * 3) : nullptr;
    w.q_bin = want_qbin ? c.take<double>((size_t)G * n) : nullptr;
    w.stats = c.take<double>((size_t)G * MCBTE_NSTATS);
    w.events_pp = want_ev ? c.take<uint32_t>(total) : nullptr;
    w.X_pp = want_x ? c.take<double>(total) : nullptr;
    w.dk = grad ? c.take<double>(n) : nullptr;
    w.dkp = grad ? c.take<double>(2) : nullptr;
    w.dkdir = (grad && nd > 0) ? c.take<double>(2 * (size_t)nd) : nullptr;
    w.kn = nscat ? c.take<double>((size_t)G * (size_t)nscat * 2) : nullptr;
  }
  w.park_cap = park_cap;
  w.park = park_cap ? c.take<unsigned char>(park_cap * park_record_bytes()) : nullptr;
  w.bytes = c.off + 256;
  return w;
}

mcbte_status check_steady(const mcbte_material* m, const mcbte_geometry* const* geoms, int G,
                          const mcbte_steady_params* p, uint64_t* total) {
  if (!m || !geoms || !p) return fail(MCBTE_ERR_INVALID_ARG, "run_steady: null argument");
  if (G < 1 || G > kMaxGeoms) return fail(MCBTE_ERR_INVALID_ARG, "run_steady: n_geoms must be in [1, 128]");
  if (!p->n_particles) return fail(MCBTE_ERR_INVALID_ARG, "run_steady: n_particles required");
  if (p->precision != MCBTE_FP64_PLAIN && p->precision != MCBTE_FP32_TRACE)
    return fail(MCBTE_ERR_INVALID_ARG, "run_steady: precision");
  if (p->n_cells < 0 || p->n_cells > 4096) return fail(MCBTE_ERR_INVALID_ARG, "run_steady: n_cells in [0, 4096]");
  if (p->cell_axis < 0 || p->cell_axis > 2 || p->tally_axis < 0 || p->tally_axis > 2)
    return fail(MCBTE_ERR_INVALID_ARG, "run_steady: axis must be 0, 1 or 2");
  if (p->n_scat_max < 0) return fail(MCBTE_ERR_INVALID_ARG, "run_steady: n_scat_max < 0");
  if (p->refill_threshold < 0 || p->refill_threshold > 32)
    return fail(MCBTE_ERR_INVALID_ARG, "run_steady: refill_threshold in [0, 32]");
  if (p->tail_lanes < -1 || p->tail_lanes > 32)
    return fail(MCBTE_ERR_INVALID_ARG, "run_steady: tail_lanes in [-1, 32]");
  if (p->threads_per_block != 0 && p->threads_per_block != 256 && p->threads_per_block != 512 &&
      p->threads_per_block != 768 && p->threads_per_block != 1024)
    return fail(MCBTE_ERR_INVALID_ARG, "run_steady: threads_per_block must be 0, 256, 512, 768 or 1024");
  uint64_t t = 0;
  for (int g = 0; g < G; ++g) {
    if (!geoms[g]) return fail(MCBTE_ERR_INVALID_ARG, "run_steady: null geometry");
    const uint64_t ng = p->n_particles[g];
    if (ng < 1 || ng >= (1ull << 32)) return fail(MCBTE_ERR_INVALID_ARG, "run_steady: n_particles in [1, 2^32)");
    const uint64_t b = p->pid_begin ? p->pid_begin[g] : 0;
    const uint64_t nt = p->n_total ? p->n_total[g] : ng;
    if (b + ng > (1ull << 32) || b + ng > nt)
      return fail(MCBTE_ERR_INVALID_ARG, "run_steady: pid_begin + n_particles must be <= n_total and <= 2^32");
    t += ng;
    const mcbte_geometry_desc& d = geoms[g]->host;
    if (d.gauss) return fail(MCBTE_ERR_INVALID_ARG, "run_steady: an initial condition needs a transient run");
    if (!has_isothermal_source(d) && !has_gradient(d))
      return fail(MCBTE_ERR_INVALID_ARG, "run_steady: geometry has no source (no isothermal wall off T_eq, no grad_T)");
    if (uses_spec_bin(d) && !m->view.spec_thr)
      return fail(MCBTE_ERR_INVALID_ARG, "run_steady: a per-bin specularity needs the material's spec_bin");
  }
  {
    const mcbte_status rs = check_regions(p->n_regions, p->regions, p->region_grid, "run_steady");
    if (rs != MCBTE_OK) return rs;
    if (p->n_regions > 0 && G != 1) return fail(MCBTE_ERR_INVALID_ARG, "run_steady: detector regions need one geometry");
  }
  if (p->det_per_bin && p->n_regions < 1)
    return fail(MCBTE_ERR_INVALID_ARG, "run_steady: det_per_bin needs detector regions");
  if (p->nscat_curve && (p->n_scat_max < 1 || p->n_scat_max > MCBTE_MAX_NSCAT_CURVE))
    return fail(MCBTE_ERR_INVALID_ARG, "run_steady: nscat_curve needs n_scat_max in [1, MCBTE_MAX_NSCAT_CURVE]");
  if (t >= (1ull << 40)) return fail(MCBTE_ERR_INVALID_ARG, "run_steady: too many particles");
  *total = t;
  return MCBTE_OK;
}

// An FP32 gradient run is one pass (forward tallies and gradient together,
// GradReplay's fused mode) when every particle's relaxation periods fit its
// list and the run keeps no cell or detector tallies; otherwise a forward
// pass stores every particle's final tally and a second pass replays it.
bool grad_fused(const mcbte_steady_params* p) {
  return p->precision == MCBTE_FP32_TRACE && p->n_scat_max >= 1 && p->n_scat_max <= kFusedPeriods &&
         p->n_cells == 0 && p->n_regions == 0 && !p->nscat_curve;
}

mcbte_status steady_impl(const mcbte_material* m, const mcbte_geometry* const* geoms, int G,
                         const mcbte_steady_params* p, const mcbte_steady_out* out, const mcbte_grad_out* gout,
                         void* workspace, size_t ws_bytes, cudaStream_t s) {
  uint64_t total = 0;
  mcbte_status st = check_steady(m, geoms, G, p, &total);
  if (st != MCBTE_OK) return st;
  if (!out || !out->stats) return fail(MCBTE_ERR_INVALID_ARG, "run_steady: out->stats required");
  const bool grad = gout != nullptr;
  const int n = m->n;
  const int nc = p->n_cells;
  const int nd = grad ? gout->n_dirs : 0;
  if (grad) {
    if (G != 1) return fail(MCBTE_ERR_INVALID_ARG, "grad: one geometry");
    if (p->n_scat_max < 1) return fail(MCBTE_ERR_INVALID_ARG, "grad: n_scat_max must be >= 1");
    if (p->precision == MCBTE_FP64_PLAIN && p->n_scat_max > kMaxPeriods - 1)
      return fail(MCBTE_ERR_INVALID_ARG, "grad: FP64 n_scat_max must be in [1, 64]");
    if (nd < 0 || nd > kMaxDirs || (nd > 0 && !gout->dirs))
      return fail(MCBTE_ERR_INVALID_ARG, "grad: n_dirs in [0, 16] with dirs");
    if (!gout->dkappa_dlogtau || !gout->dkappa_dp || (nd > 0 && !gout->dkappa_dir))
      return fail(MCBTE_ERR_INVALID_ARG, "grad: output pointers required");
    if (gout->on_host != out->on_host) return fail(MCBTE_ERR_INVALID_ARG, "grad: on_host must match");
    if (gout->dp_estimator < 0 || gout->dp_estimator > 2)
      return fail(MCBTE_ERR_INVALID_ARG, "grad: dp_estimator must be 0, 1 or 2");
    if (p->nscat_curve) return fail(MCBTE_ERR_INVALID_ARG, "grad: nscat_curve is an output of run_steady");
  }
  if (p->nscat_curve && !out->kappa_nscat)
    return fail(MCBTE_ERR_INVALID_ARG, "run_steady: nscat_curve needs out->kappa_nscat");
  const int nscat = p->nscat_curve ? p->n_scat_max : 0;
  const bool host_out = out->on_host != 0;
  const bool fused = grad && grad_fused(p);
  const bool replay = grad && p->precision == MCBTE_FP32_TRACE && !fused;
  const uint64_t n_det = region_detectors(p->n_regions, p->region_grid);
  const uint64_t det_slots = steady_det_slots(p, n);
  // the tail kernel's park buffer when the workspace has room for it (a
  // caller's workspace sized without it still runs, without the tail kernel)
  uint64_t park_cap = park_capacity(p, total);
  SteadyWs w = layout_steady(nullptr, G, n, nc, total, grad, replay, nd, host_out, out->events_pp, out->X_pp, out->T,
                             out->q, out->q_bin, det_slots, nscat, park_cap);
  char* base = static_cast<char*>(workspace);
  if (base && ws_bytes < w.bytes && park_cap) {
    park_cap = 0;
    w = layout_steady(nullptr, G, n, nc, total, grad, replay, nd, host_out, out->events_pp, out->X_pp, out->T, out->q,
                      out->q_bin, det_slots, nscat, 0);
  }
  const size_t need = w.bytes;
  bool own = false;
  if (!base) {
    CUDA_TRY(cudaMallocAsync((void**)&base, need, s));
    own = true;
  } else if (ws_bytes < need) {
    return fail(MCBTE_ERR_WORKSPACE, "run_steady: workspace too small");
  }
  char* aligned = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(base) + 255) & ~(uintptr_t)255);
  w = layout_steady(aligned, G, n, nc, total, grad, replay, nd, host_out, out->events_pp, out->X_pp, out->T, out->q,
                    out->q_bin, det_slots, nscat, park_cap);
  auto release = [&]() {
    if (own) cudaFreeAsync(base, s);
  };
#define RUN_TRY(call)                      \
  do {                                     \
    cudaError_t e_ = (call);               \
    if (e_ != cudaSuccess) {               \
      release();                           \
      return cuda_fail(e_, #call);         \
    }                                      \
  } while (0)
  RUN_TRY(cudaMemsetAsync(w.zero_begin, 0, (size_t)(w.zero_end - w.zero_begin), s));
  SetupArgs a;
  std::memset(&a, 0, sizeof(a));
  for (int g = 0; g < G; ++g) {
    a.desc[g] = geoms[g]->dev;
    a.n[g] = p->n_particles[g];
    a.pid0[g] = p->pid_begin ? p->pid_begin[g] : 0;
    a.n_norm[g] = p->n_total ? p->n_total[g] : p->n_particles[g];
  }
  RUN_TRY(launch_setup(a, G, m->view, 0, 0.0, p->tally_axis, w.geos, w.offs, w.t0, s));
  RunCfg C{};
  C.k0 = (uint32_t)p->seed;
  C.k1 = (uint32_t)(p->seed >> 32);
  C.n_scat_max = p->n_scat_max;
  C.max_events = (p->max_events == 0 || p->max_events > 0xFFFFFFFFull) ? 0xFFFFFFFFu : (uint32_t)p->max_events;
  C.n_cells = nc;
  C.cell_axis = p->cell_axis;
  C.tally_axis = p->tally_axis;
  C.per_bin = p->per_bin ? 1 : 0;
  C.n_geoms = G;
  C.total = total;
  C.t0 = w.t0;
  C.budget_ns = (uint64_t)((p->time_budget_s > 0 ? p->time_budget_s : 120.0) * 1e9);
  C.seed_dev = reinterpret_cast<const unsigned long long*>(p->seed_device);
  C.refill_min = p->refill_threshold;
  C.tail_max = p->tail_lanes == 0 ? 8 : (p->tail_lanes < 0 ? 0 : p->tail_lanes);
  C.fused = fused ? 1 : 0;
  C.take_chunk = G > 1 ? 1024u : 256u;
  C.cell_flux_axis = p->cell_flux_axis ? 1 : 0;
  C.ext = (p->n_regions > 0 || nscat > 0) ? 1 : 0;
  for (int g = 0; g < G; ++g) C.ext |= uses_ext(m, geoms[g]->host) ? 1 : 0;
  C.nscat_acc = w.nscat;
  C.nscat_rep = nscat ? nscat_replicas(G, nscat) : 1;
  C.n_regs = p->n_regions;
  C.n_det = (uint32_t)n_det;
  C.det_nb = p->det_per_bin ? n : 1;
  C.regs = w.regs;
  if (grad && geoms[0]->host.pore) {
    // d kappa / d p_pore: the measure-valued estimator on request, and where
    // the likelihood-ratio score is undefined
    const double pp = geoms[0]->host.pore_p;
    C.mvd = (gout->dp_estimator == 2 || (gout->dp_estimator == 0 && (pp <= 0.0 || pp >= 1.0))) ? 1 : 0;
  }
  if (p->n_regions > 0) {
    const std::vector<DetRegion> rg =
        build_regions(p->n_regions, p->regions, p->region_grid, false, nullptr, geoms[0]->host.L);
    RUN_TRY(param_upload(w.regs, rg.data(), rg.size() * sizeof(DetRegion), s));
  }
  Acc A{};
  A.cellP = w.cellP;
  A.cellD = w.cellD;
  A.qbin = w.qbin;
  A.cellPq = w.cellPq;
  A.cellDq = w.cellDq;
  A.qbinq = w.qbinq;
  A.dsc = w.dsc;
  A.cnt = w.cnt;
  A.G = w.G;
  A.Gq = w.Gq;
  A.gsum = w.gsum;
  A.work = w.work;
  A.flags = w.flags;
  A.det_raw = w.det_raw;
  A.det_q = w.det_q;
  A.park = w.park;
  A.park_n = w.park_n;
  A.park_rd = w.park_rd;
  A.park_stride = park_record_bytes();
  A.park_cap = w.park_cap;
  A.events_pp = host_out ? w.events_pp : out->events_pp;
  A.X_pp = host_out ? w.X_pp : out->X_pp;
  if (grad && nd > 0) {
    RUN_TRY(cudaMemcpyAsync(w.dirs, gout->dirs, (size_t)nd * n * sizeof(double),
                            host_out ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    RUN_TRY(launch_dirs_dot_pi(w.dirs, nd, m->view, w.dpi, s));
    C.n_dirs = nd;
    C.dirs = w.dirs;
    C.dpi = w.dpi;
  }
  if (p->trace_event_start) RUN_TRY(record_trace_event(p->trace_event_start, s));
  if (replay) {
    // forward pass (all tallies, every particle's final X), then the
    // gradient pass over the same particles
    Acc A1 = A;
    A1.X_pp = w.xrep;
    RUN_TRY(launch_steady(p->precision, false, w.geos, w.offs, m->view, C, A1, p->threads_per_block,
                          p->blocks_per_sm, s));
    RUN_TRY(cudaMemsetAsync(w.work, 0, sizeof(unsigned long long), s));
    RUN_TRY(cudaMemsetAsync(w.park_n, 0, sizeof(unsigned long long), s));
    RUN_TRY(cudaMemsetAsync(w.park_rd, 0, sizeof(unsigned long long), s));
    Acc A2 = A;
    A2.X_pp = w.xrep;
    A2.events_pp = nullptr;
    RUN_TRY(launch_steady(p->precision, true, w.geos, w.offs, m->view, C, A2, p->threads_per_block,
                          p->blocks_per_sm, s));
    if (A.X_pp) RUN_TRY(cudaMemcpyAsync(A.X_pp, w.xrep, total * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    RUN_TRY(launch_steady(p->precision, grad, w.geos, w.offs, m->view, C, A, p->threads_per_block, p->blocks_per_sm,
                          s));
  }
  if (p->trace_event_stop) RUN_TRY(record_trace_event(p->trace_event_stop, s));
  SteadyOutDev O{};
  O.T = host_out ? w.T : out->T;
  O.q = host_out ? w.q : out->q;
  O.q_bin = host_out ? w.q_bin : out->q_bin;
  O.stats = host_out ? w.stats : out->stats;
  O.det = host_out ? w.det : out->det;
  O.kn = host_out ? w.kn : out->kappa_nscat;
  if (grad) {
    O.dk = host_out ? w.dk : gout->dkappa_dlogtau;
    O.dkp = host_out ? w.dkp : gout->dkappa_dp;
    O.dkdir = host_out ? w.dkdir : gout->dkappa_dir;
  }
  RUN_TRY(launch_finalize_steady(w.geos, m->view, C, A, O, grad, w.flags, s));
  mcbte_status result = MCBTE_OK;
  if (host_out) {
    auto d2h = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
      if (!dst || !src || bytes == 0) return cudaSuccess;
      return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
    };
    RUN_TRY(d2h(out->T, w.T, (size_t)G * nc * sizeof(double)));
    RUN_TRY(d2h(out->q, w.q, (size_t)G * nc * 3 * sizeof(double)));
    RUN_TRY(d2h(out->q_bin, w.q_bin, (size_t)G * n * sizeof(double)));
    RUN_TRY(d2h(out->stats, w.stats, (size_t)G * MCBTE_NSTATS * sizeof(double)));
    RUN_TRY(d2h(out->events_pp, w.events_pp, total * sizeof(uint32_t)));
    RUN_TRY(d2h(out->X_pp, w.X_pp, total * sizeof(double)));
    RUN_TRY(d2h(out->det, w.det, 4 * det_slots * sizeof(double)));
    RUN_TRY(d2h(out->kappa_nscat, w.kn, (size_t)G * (size_t)nscat * 2 * sizeof(double)));
    if (grad) {
      RUN_TRY(d2h(gout->dkappa_dlogtau, w.dk, (size_t)n * sizeof(double)));
      RUN_TRY(d2h(gout->dkappa_dp, w.dkp, 2 * sizeof(double)));
      if (nd > 0) RUN_TRY(d2h(gout->dkappa_dir, w.dkdir, 2 * (size_t)nd * sizeof(double)));
    }
    release();
    own = false;
    RUN_TRY(cudaStreamSynchronize(s));
    for (int g = 0; g < G; ++g) {
      const double code = out->stats[(size_t)g * MCBTE_NSTATS + MCBTE_STAT_STATUS];
      if (code == (double)MCBTE_ERR_TIMEOUT) result = fail(MCBTE_ERR_TIMEOUT, "run: time budget exceeded");
      else if (code == (double)MCBTE_WARN_TRUNCATED && result == MCBTE_OK)
        result = fail(MCBTE_WARN_TRUNCATED, "run: some particles reached max_events");
    }
  } else {
    release();
  }
#undef RUN_TRY
  return result;
}

}  // namespace

extern "C" {

mcbte_status mcbte_steady_workspace_size(const mcbte_material* m, const mcbte_geometry* const* geoms, int n_geoms,
                                         const mcbte_steady_params* p, int want_grad, int n_dirs, size_t* bytes) {
  uint64_t total = 0;
  mcbte_status st = check_steady(m, geoms, n_geoms, p, &total);
  if (st != MCBTE_OK) return st;
  if (!bytes) return fail(MCBTE_ERR_INVALID_ARG, "workspace_size: null bytes");
  SteadyWs w = layout_steady(nullptr, n_geoms, m->n, p->n_cells, total, want_grad != 0,
                             want_grad != 0 && p->precision == MCBTE_FP32_TRACE && !grad_fused(p), n_dirs, false,
                             false, false, false,
                             false, false, steady_det_slots(p, m->n), p->nscat_curve ? p->n_scat_max : 0,
                             park_capacity(p, total));
  *bytes = w.bytes;
  return MCBTE_OK;
}

mcbte_status mcbte_run_steady(const mcbte_material* m, const mcbte_geometry* const* geoms, int n_geoms,
                              const mcbte_steady_params* p, const mcbte_steady_out* out, void* workspace,
                              size_t workspace_bytes, mcbte_stream stream) {
  return steady_impl(m, geoms, n_geoms, p, out, nullptr, workspace, workspace_bytes, (cudaStream_t)stream);
}

mcbte_status mcbte_grad(const mcbte_material* m, const mcbte_geometry* g, const mcbte_steady_params* p,
                        const mcbte_steady_out* fwd, const mcbte_grad_out* grad, void* workspace,
                        size_t workspace_bytes, mcbte_stream stream) {
  if (!grad) return fail(MCBTE_ERR_INVALID_ARG, "grad: null grad output");
  const mcbte_geometry* gs[1] = {g};
  return steady_impl(m, gs, 1, p, fwd, grad, workspace, workspace_bytes, (cudaStream_t)stream);
}

}  // extern "C"

// ------------------------------------------------------------------ transient runs
namespace {

struct TransientWs {
  GeoRun* geos;
  uint64_t* offs;
  char* zero_begin;
  double* dsc;
  unsigned long long* cnt;
  unsigned long long* work;
  int* flags;
  unsigned long long* t0;
  char* zero_end;
  double* t_meas_ps;
  double* snap;     // only when outputs are on the host
  double* stats;
  uint32_t* events_pp;
  uint4* tstate;    // FP32 time windows: particle state between windows
  DetRegion* regs;  // detector regions
  size_t bytes;
};

// FP32 transient time windows: measurement times per window.  Automatic
// choice: the largest window whose [times][cells][4] x 8-byte slice of the
// snapshot tally fits a third of the L2, so the snapshot atomics of a window
// hit in L2 instead of read-modify-writing HBM.
uint64_t transient_detectors(const mcbte_transient_params* p) {
  if (p->n_regions == 0) return (uint64_t)p->grid[0] * p->grid[1] * p->grid[2];
  uint64_t nd = 0;
  for (int k = 0; k < p->n_regions; ++k)
    nd += (uint64_t)p->region_grid[3 * k] * p->region_grid[3 * k + 1] * p->region_grid[3 * k + 2];
  return nd;
}

int transient_window_times(const mcbte_transient_params* p) {
  if (p->precision != MCBTE_FP32_TRACE) return p->n_times;
  int wt = p->window_times;
  if (wt <= 0) {
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess ||
        l2 <= 0)
      l2 = 96 << 20;
    const size_t slice = (size_t)transient_detectors(p) * 4 * sizeof(long long);
    const size_t fit = ((size_t)l2 / 3) / slice;
    wt = fit < 1 ? 1 : (fit > (size_t)p->n_times ? p->n_times : (int)fit);
  }
  return wt < p->n_times ? wt : p->n_times;
}

TransientWs layout_transient(char* base, size_t snap_len, int n_times, bool host_out, bool want_ev, uint64_t total,
                             bool windows) {
  Carve c;
  c.base = base;
  TransientWs w{};
  w.geos = c.take<GeoRun>(1);
  w.offs = c.take<uint64_t>(2);
  c.off = (c.off + 255) & ~(size_t)255;
  w.zero_begin = base ? base + c.off : nullptr;
  w.dsc = c.take<double>(8 * (size_t)kSumCopies);
  w.cnt = c.take<unsigned long long>(4 * (size_t)kSumCopies);
  w.work = c.take<unsigned long long>(1);
  w.flags = c.take<int>(2);
  w.t0 = c.take<unsigned long long>(1);
  c.off = (c.off + 255) & ~(size_t)255;
  w.zero_end = base ? base + c.off : nullptr;
  w.t_meas_ps = c.take<double>(n_times);
  w.tstate = windows ? c.take<uint4>(3 * total) : nullptr;
  w.regs = c.take<DetRegion>(MCBTE_MAX_REGIONS);
  if (host_out) {
    w.snap = c.take<double>(snap_len);
    w.stats = c.take<double>(MCBTE_NSTATS);
    w.events_pp = want_ev ? c.take<uint32_t>(total) : nullptr;
  }
  w.bytes = c.off + 256;
  return w;
}

mcbte_status check_transient(const mcbte_material* m, const mcbte_geometry* g, const mcbte_transient_params* p) {
  if (!m || !g || !p) return fail(MCBTE_ERR_INVALID_ARG, "run_transient: null argument");
  if (p->n_particles < 1 || p->n_particles >= (1ull << 32))
    return fail(MCBTE_ERR_INVALID_ARG, "run_transient: n_particles in [1, 2^32)");
  if (p->precision != MCBTE_FP64_PLAIN && p->precision != MCBTE_FP32_TRACE)
    return fail(MCBTE_ERR_INVALID_ARG, "run_transient: precision");
  if (!finite_pos(p->t_max)) return fail(MCBTE_ERR_INVALID_ARG, "run_transient: t_max must be > 0");
  if (p->n_times < 1 || !p->t_meas) return fail(MCBTE_ERR_INVALID_ARG, "run_transient: t_meas required");
  if (p->n_times > MCBTE_MAX_TIMES) return fail(MCBTE_ERR_INVALID_ARG, "run_transient: n_times above MCBTE_MAX_TIMES");
  for (int k = 0; k < p->n_times; ++k) {
    if (!(p->t_meas[k] > 0.0 && p->t_meas[k] <= p->t_max)) return fail(MCBTE_ERR_INVALID_ARG, "run_transient: t_meas in (0, t_max]");
    if (k > 0 && !(p->t_meas[k] > p->t_meas[k - 1])) return fail(MCBTE_ERR_INVALID_ARG, "run_transient: t_meas ascending");
  }
  for (int a = 0; a < 3; ++a)
    if (p->grid[a] < 1 || p->grid[a] > 4096) return fail(MCBTE_ERR_INVALID_ARG, "run_transient: grid in [1, 4096]");
  {
    const mcbte_status rs = check_regions(p->n_regions, p->regions, p->region_grid, "run_transient");
    if (rs != MCBTE_OK) return rs;
  }
  if (p->threads_per_block != 0 && p->threads_per_block != 256 && p->threads_per_block != 512 &&
      p->threads_per_block != 768 && p->threads_per_block != 1024)
    return fail(MCBTE_ERR_INVALID_ARG, "run_transient: threads_per_block must be 0, 256, 512, 768 or 1024");
  const mcbte_geometry_desc& d = g->host;
  if (has_gradient(d)) return fail(MCBTE_ERR_INVALID_ARG, "run_transient: body (gradient) sources are steady only");
  if (uses_spec_bin(d) && !m->view.spec_thr)
    return fail(MCBTE_ERR_INVALID_ARG, "run_transient: a per-bin specularity needs the material's spec_bin");
  if (!d.gauss && !has_isothermal_source(d)) return fail(MCBTE_ERR_INVALID_ARG, "run_transient: no source");
  return MCBTE_OK;
}

}  // namespace

extern "C" {

mcbte_status mcbte_transient_workspace_size(const mcbte_material* m, const mcbte_geometry* g,
                                            const mcbte_transient_params* p, size_t* bytes) {
  mcbte_status st = check_transient(m, g, p);
  if (st != MCBTE_OK) return st;
  if (!bytes) return fail(MCBTE_ERR_INVALID_ARG, "workspace_size: null bytes");
  *bytes = layout_transient(nullptr, 0, p->n_times, false, false, p->n_particles,
                            transient_window_times(p) < p->n_times).bytes;
  return MCBTE_OK;
}

mcbte_status mcbte_run_transient(const mcbte_material* m, const mcbte_geometry* g, const mcbte_transient_params* p,
                                 const mcbte_transient_out* out, void* workspace, size_t workspace_bytes,
                                 mcbte_stream stream) {
  mcbte_status st = check_transient(m, g, p);
  if (st != MCBTE_OK) return st;
  if (!out || !out->tally || !out->stats) return fail(MCBTE_ERR_INVALID_ARG, "run_transient: tally and stats required");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ncell = (size_t)transient_detectors(p);
  const size_t snap_len = (size_t)p->n_times * ncell * 4;
  const bool host_out = out->on_host != 0;
  const int wt = transient_window_times(p);
  const int n_win = (p->n_times + wt - 1) / wt;
  TransientWs w = layout_transient(nullptr, snap_len, p->n_times, host_out, out->events_pp, p->n_particles, n_win > 1);
  char* base = static_cast<char*>(workspace);
  bool own = false;
  if (!base) {
    CUDA_TRY(cudaMallocAsync((void**)&base, w.bytes, s));
    own = true;
  } else if (workspace_bytes < w.bytes) {
    return fail(MCBTE_ERR_WORKSPACE, "run_transient: workspace too small");
  }
  char* aligned = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(base) + 255) & ~(uintptr_t)255);
  w = layout_transient(aligned, snap_len, p->n_times, host_out, out->events_pp, p->n_particles, n_win > 1);
  auto release = [&]() {
    if (own) cudaFreeAsync(base, s);
  };
#define RUN_TRY(call)              \
  do {                             \
    cudaError_t e_ = (call);       \
    if (e_ != cudaSuccess) {       \
      release();                   \
      return cuda_fail(e_, #call); \
    }                              \
  } while (0)
  double* snap = host_out ? w.snap : out->tally;
  RUN_TRY(cudaMemsetAsync(w.zero_begin, 0, (size_t)(w.zero_end - w.zero_begin), s));
  RUN_TRY(cudaMemsetAsync(snap, 0, snap_len * sizeof(double), s));
  std::vector<double> tm(p->n_times);
  for (int k = 0; k < p->n_times; ++k) tm[k] = p->t_meas[k] * 1e12;
  RUN_TRY(param_upload(w.t_meas_ps, tm.data(), tm.size() * sizeof(double), s));
  SetupArgs a;
  std::memset(&a, 0, sizeof(a));
  a.desc[0] = g->dev;
  a.n[0] = p->n_particles;
  RUN_TRY(launch_setup(a, 1, m->view, 1, p->t_max, 2, w.geos, w.offs, w.t0, s));
  RunCfg C{};
  C.k0 = (uint32_t)p->seed;
  C.k1 = (uint32_t)(p->seed >> 32);
  C.n_scat_max = 0;
  C.max_events = (p->max_events == 0 || p->max_events > 0xFFFFFFFFull) ? 0xFFFFFFFFu : (uint32_t)p->max_events;
  C.n_geoms = 1;
  C.total = p->n_particles;
  C.take_chunk = 256u;
  C.t0 = w.t0;
  C.budget_ns = (uint64_t)((p->time_budget_s > 0 ? p->time_budget_s : 120.0) * 1e9);
  C.t_max_ps = p->t_max * 1e12;
  C.ext = uses_ext(m, g->host) ? 1 : 0;
  C.n_times = p->n_times;
  C.t_meas_ps = w.t_meas_ps;
  for (int k = 0; k < 3; ++k) C.grid[k] = p->grid[k];
  // detector regions, derived on the host with the CPU reference's arithmetic;
  // bin averages over the whole box walk the box grid as one region
  C.time_average = p->time_average ? 1 : 0;
  const bool whole_region = p->time_average && p->n_regions == 0;
  C.n_regs = whole_region ? 1 : p->n_regions;
  C.n_det = (uint32_t)ncell;
  C.regs = w.regs;
  if (C.n_regs > 0) {
    const std::vector<DetRegion> rg =
        build_regions(C.n_regs, p->regions, p->region_grid, whole_region, p->grid, g->host.L);
    RUN_TRY(param_upload(w.regs, rg.data(), rg.size() * sizeof(DetRegion), s));
  }
  Acc A{};
  A.dsc = w.dsc;
  A.cnt = w.cnt;
  A.work = w.work;
  A.flags = w.flags;
  A.snap = snap;
  A.events_pp = host_out ? w.events_pp : out->events_pp;
  A.tstate = w.tstate;
  if (p->trace_event_start) RUN_TRY(record_trace_event(p->trace_event_start, s));
  // one launch per time window (a single one unless the FP32 tally exceeds the L2 budget)
  for (int k = 0; k < n_win; ++k) {
    C.win_first = k == 0;
    C.win_last = k == n_win - 1;
    C.win_end = (k + 1) * wt < p->n_times ? (k + 1) * wt : p->n_times;
    if (k > 0) RUN_TRY(cudaMemsetAsync(w.work, 0, sizeof(unsigned long long), s));
    RUN_TRY(launch_transient(p->precision, w.geos, m->view, C, A, p->threads_per_block, p->blocks_per_sm, s));
  }
  if (p->trace_event_stop) RUN_TRY(record_trace_event(p->trace_event_stop, s));
  double* stats = host_out ? w.stats : out->stats;
  RUN_TRY(launch_finalize_transient(w.geos, m->view, C, A, snap, stats, ncell, p->precision == MCBTE_FP32_TRACE, s));
  mcbte_status result = MCBTE_OK;
  if (host_out) {
    RUN_TRY(cudaMemcpyAsync(out->tally, snap, snap_len * sizeof(double), cudaMemcpyDeviceToHost, s));
    RUN_TRY(cudaMemcpyAsync(out->stats, stats, MCBTE_NSTATS * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (out->events_pp)
      RUN_TRY(cudaMemcpyAsync(out->events_pp, w.events_pp, p->n_particles * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    release();
    own = false;
    RUN_TRY(cudaStreamSynchronize(s));
    const double code = out->stats[MCBTE_STAT_STATUS];
    if (code == (double)MCBTE_ERR_TIMEOUT) result = fail(MCBTE_ERR_TIMEOUT, "run: time budget exceeded");
    else if (code == (double)MCBTE_WARN_TRUNCATED) result = fail(MCBTE_WARN_TRUNCATED, "run: some particles reached max_events");
  } else {
    release();
  }
#undef RUN_TRY
  return result;
}

}  // extern "C"

// ------------------------------------------------------------------ steady run without device allocation
// For callers that cannot call cudaMalloc: code running where the CUDA
// allocator is off limits (inside another library's allocation-free region,
// a real-time or pre-allocated memory budget, a host process that must not
// grow device memory after start-up).  The run's scratch lives in a fixed
// device array that every GPU loading this library holds until the process
// exits; outputs are still the caller's device buffers.
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;   // 8 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};

}  // namespace

extern "C" {

mcbte_status mcbte_run_steady_noalloc(const mcbte_material* m, const mcbte_geometry* const* geoms, int n_geoms,
                                      const mcbte_steady_params* p, const mcbte_steady_out* out,
                                      mcbte_stream stream) {
  if (!out) return fail(MCBTE_ERR_INVALID_ARG, "run_steady_noalloc: null outputs");
  if (out->on_host) return fail(MCBTE_ERR_INVALID_ARG, "run_steady_noalloc: outputs must be device memory");
  uint64_t total = 0;
  mcbte_status st = check_steady(m, geoms, n_geoms, p, &total);
  if (st != MCBTE_OK) return st;
  // (the tail kernel's park buffer is used only when it fits as well)
  const SteadyWs w = layout_steady(nullptr, n_geoms, m->n, p->n_cells, total, false, false, 0, false, false, false,
                                   false, false, false, steady_det_slots(p, m->n),
                                   p->nscat_curve ? p->n_scat_max : 0);
  if (w.bytes > kNoAllocScratchBytes)
    return fail(MCBTE_ERR_WORKSPACE, "run_steady_noalloc: this run needs " + std::to_string(w.bytes) +
                                         " bytes of scratch, above the fixed " +
                                         std::to_string(kNoAllocScratchBytes) + " bytes");
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(MCBTE_ERR_INVALID_ARG, "run_steady_noalloc: device ordinal");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      // the array's name is a host-side stand-in; its device address comes
      // from the runtime, once per device, with that device current
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "run_steady_noalloc: cudaGetSymbolAddress");
      g_noalloc_addr[dev] = ptr;
    }
    scratch = g_noalloc_addr[dev];
  }
  return steady_impl(m, geoms, n_geoms, p, out, nullptr, scratch, kNoAllocScratchBytes, (cudaStream_t)stream);
}

}  // extern "C"
