// Material table build (FP64, on the GPU).
//
// Per bin: C_i = D_i dE/dT(omega_i) d_omega_i (Eq. BE_derivative read as the
// derivative of the Bose-Einstein mode energy, Eq. Nbin), or C_i given
// (format 2); emission weights C v (Eqs. iso_flux, grad_flux_sim), C
// (Eq. Nbin) and relaxation weights C / tau (Eq. n_scatt); unit conversion
// to nm / ps.  Then one thread per table builds Walker's alias table with
// Vose's two work lists (filled in increasing bin order, popped from the
// back), so the table is a deterministic function of the weights.
#include "launch.h"

namespace mcbte {

namespace {

__device__ __forceinline__ double dEdT(double omega, double T) {
  const double kHbar = 1.054571817e-34;
  const double kBoltz = 1.380649e-23;
  const double x = (kHbar * omega) / (kBoltz * T);
  const double h = 0.5 * x;
  const double s = sinh(h);
  return kBoltz * (h * h) / (s * s);
}

__global__ void k_bins(MatBuild b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b.n) return;
  double C;
  if (b.C_in) C = b.C_in[i];
  else C = (b.D[i] * dEdT(b.omega[i], b.T_lin)) * b.domega[i];
  b.C[i] = C;
  b.w_emit[i] = C * b.v[i];
  b.w_init[i] = C;
  b.w_relax[i] = C / b.tau[i];
  const double v_nm = b.v[i] * 1e-3;
  const double tau_ps = b.tau[i] * 1e12;
  const double lam = v_nm * tau_ps;
  const double inv_v = 1.0 / v_nm;
  // two-phonon mean free path (Sec. 3.3); +inf where the bin has none
  double lam2 = __longlong_as_double(0x7ff0000000000000ll);
  if (b.tau_imp && isfinite(b.tau_imp[i])) lam2 = v_nm * (b.tau_imp[i] * 1e12);
  b.v_nm[i] = v_nm;
  b.lam[i] = lam;
  b.inv_v[i] = inv_v;
  b.lam2[i] = lam2;
  if (b.spec_bin) b.spec_thr[i] = spec_threshold(b.spec_bin[i]);
  b.binf[i] = make_float4((float)v_nm, (float)inv_v, (float)lam, (float)lam2);
}

// Largest table whose build runs in shared memory: 24 bytes per bin (the
// weights or work probabilities, the two work lists and the aliases; the
// sums block stages three weight columns).
constexpr int kAliasSmemBins = 9216;

// blockIdx.x = 0..2 builds alias table k (weights C v, C, C / tau);
// blockIdx.x = 3 forms the sums and the relaxation pmf.  The sums and
// Vose's lists are sequential (thread 0, bin order, so the table is a fixed
// function of the weights); the per-bin arithmetic around them is spread
// over the block.  With `smem` the work arrays live in shared memory, else
// in the global scratch.
__global__ void k_alias(MatBuild b, int smem) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ double s_tot;
  const int n = b.n;
  const int k = blockIdx.x;
  const int t = threadIdx.x;
  if (k == 3) {
    // the columns are staged in shared memory first, so the sequential sums
    // read at shared-memory latency
    const double *c0 = b.C, *c1 = b.w_emit, *c2 = b.w_relax;
    if (smem) {
      double* st = reinterpret_cast<double*>(sm);
      for (int i = t; i < n; i += blockDim.x) {
        st[i] = b.C[i];
        st[n + i] = b.w_emit[i];
        st[2 * (size_t)n + i] = b.w_relax[i];
      }
      __syncthreads();
      c0 = st;
      c1 = st + n;
      c2 = st + 2 * (size_t)n;
    }
    if (t == 0) {
      double ct = 0.0, cv = 0.0, cr = 0.0;
      for (int i = 0; i < n; ++i) {
        ct += c0[i];
        cv += c1[i];
        cr += c2[i];
      }
      b.sums[0] = ct;
      b.sums[1] = cv;
      b.sums[2] = cr;
      s_tot = cr;
    }
    __syncthreads();
    const double cr = s_tot;
    for (int i = t; i < n; i += blockDim.x) b.pi[i] = b.w_relax[i] / cr;
    return;
  }
  const double* w = (k == 0) ? b.w_emit : (k == 1 ? b.w_init : b.w_relax);
  double* p;
  int *small, *large, *alias;
  if (smem) {
    p = reinterpret_cast<double*>(sm);
    small = reinterpret_cast<int*>(p + n);
    large = small + n;
    alias = large + n;
  } else {
    p = b.scratch_p + (size_t)k * n;
    small = b.scratch_small + (size_t)k * n;
    large = b.scratch_large + (size_t)k * n;
    alias = b.alias + (size_t)k * n;
  }
  for (int i = t; i < n; i += blockDim.x) p[i] = w[i];
  __syncthreads();
  if (t == 0) {
    double W = 0.0;
    for (int i = 0; i < n; ++i) W += p[i];
    s_tot = W;
  }
  __syncthreads();
  const double W = s_tot;
  for (int i = t; i < n; i += blockDim.x) {
    p[i] = (p[i] * (double)n) / W;
    alias[i] = i;
  }
  __syncthreads();
  if (t == 0) {
    int ns = 0, nl = 0;
    for (int i = 0; i < n; ++i) {
      if (p[i] < 1.0) small[ns++] = i; else large[nl++] = i;
    }
    // a bin popped from the small list keeps its p as its probability and
    // takes the large bin as its alias (never itself); every other bin
    // keeps probability 1
    while (ns > 0 && nl > 0) {
      const int l = small[--ns];
      const int g = large[--nl];
      alias[l] = g;
      p[g] = (p[g] + p[l]) - 1.0;
      if (p[g] < 1.0) small[ns++] = g; else large[nl++] = g;
    }
  }
  __syncthreads();
  double* prob = b.prob + (size_t)k * n;
  int32_t* alias_out = b.alias + (size_t)k * n;
  uint64_t* thr = b.thr + (size_t)k * n;
  uint4* rec = b.rec + (size_t)k * n;
  for (int i = t; i < n; i += blockDim.x) {
    const int a = alias[i];
    const double q = (a != i) ? p[i] : 1.0;
    prob[i] = q;
    alias_out[i] = a;
    const uint64_t th = (q >= 1.0) ? UINT64_MAX : (uint64_t)(q * 18446744073709551616.0);
    thr[i] = th;
    rec[i] = make_uint4((uint32_t)th, (uint32_t)(th >> 32), (uint32_t)a, 0u);
  }
}

}  // namespace

cudaError_t launch_material_build(const MatBuild& b, cudaStream_t s) {
  k_bins<<<(b.n + 255) / 256, 256, 0, s>>>(b);
  const int smem = b.n <= kAliasSmemBins ? 1 : 0;
  const size_t bytes = smem ? (size_t)b.n * 24 : 0;
  if (smem) {
    const cudaError_t e = cudaFuncSetAttribute(k_alias, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
  }
  k_alias<<<4, 256, bytes, s>>>(b, smem);
  return cudaGetLastError();
}

}  // namespace mcbte
