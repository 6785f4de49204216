// Host-side launch interface between the C-ABI layer and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "tracer.cuh"

namespace mcbte {

// Per-geometry inputs of the setup kernel, passed by value (4 KB): the
// descriptor, the particles of this call, the index of the first one, and
// the particles of the whole run that normalise E_eff = E_tot / N.
struct SetupArgs {
  const mcbte_geometry_desc* desc[kMaxGeoms];
  uint64_t n[kMaxGeoms];
  uint64_t pid0[kMaxGeoms];
  uint64_t n_norm[kMaxGeoms];
};

// Shared-memory plan of the persistent FP32 tracer.
struct SmemPlan {
  int relax_in_smem;   // alias records ~ C/tau in shared memory
  int binf_in_smem;    // per-bin {v, 1/v, Lambda} in shared memory
  int qbin_in_smem;    // frequency-resolved flux privatised per block
  int cells_in_smem;   // cell tallies privatised per block
  int tail_slots;      // the tail's per-thread draw slots (first in the layout)
  int grad_in_smem;    // the gradient accumulator privatised per block
  int snap_in_smem;    // a pore-hit snapshot per thread (measure-valued d/dp; after the tail slots)
  size_t bytes;
};

SmemPlan plan_smem_f32(int n_bins, int n_geoms, int n_cells, int per_bin, size_t budget, int tail_threads = 0,
                       int grad_acc = 0, int snap_threads = 0);

cudaError_t launch_setup(const SetupArgs& a, int n_geoms, const MatView& M, int transient, double t_max_s,
                         int tally_axis, GeoRun* geos, uint64_t* offs, unsigned long long* t0, cudaStream_t s);

cudaError_t launch_steady(int precision, bool grad, const GeoRun* geos, const uint64_t* offs, const MatView& M,
                          const RunCfg& C, const Acc& A, int threads, int blocks_per_sm, cudaStream_t s);

struct SteadyOutDev {
  double* T;
  double* q;
  double* q_bin;
  double* stats;
  double* dk;        // grad: [n_bins]
  double* dkp;       // grad: [2]
  double* dkdir;     // grad: [n_dirs][2]
  double* det;       // detector regions: [n_det][4], or null
  double* kn;        // N_scat_max curve: [G][n_scat_max][2], or null
};

cudaError_t launch_steady_f32(bool grad, bool cells, const GeoRun* geos, const uint64_t* offs, const MatView& M,
                              const RunCfg& C, const Acc& A, int threads, int bps, cudaStream_t s);
// the same with the main kernel that parks its tail and the tail kernel
cudaError_t launch_steady_f32_tail(bool grad, bool cells, const GeoRun* geos, const uint64_t* offs, const MatView& M,
                                   const RunCfg& C, const Acc& A, int threads, int bps, cudaStream_t s);
cudaError_t launch_transient_f32(const GeoRun* geos, const MatView& M, const RunCfg& C, const Acc& A, int threads,
                                 int bps, cudaStream_t s);

cudaError_t launch_finalize_steady(const GeoRun* geos, const MatView& M, const RunCfg& C, const Acc& A,
                                   const SteadyOutDev& O, bool grad, const int* flags, cudaStream_t s);

cudaError_t launch_dirs_dot_pi(const double* dirs, int n_dirs, const MatView& M, double* dpi, cudaStream_t s);

cudaError_t launch_transient(int precision, const GeoRun* geos, const MatView& M, const RunCfg& C, const Acc& A,
                             int threads, int blocks_per_sm, cudaStream_t s);

cudaError_t launch_finalize_transient(const GeoRun* geos, const MatView& M, const RunCfg& C, const Acc& A,
                                      double* tally, double* stats, size_t n_cells_total, bool fixed,
                                      cudaStream_t s);

// Material table build (FP64): per-bin kernel + one thread per alias table.
struct MatBuild {
  int n;
  const double *omega, *v, *tau, *C_in, *D, *domega;
  const double* tau_imp;   // optional two-phonon relaxation times (s), or null
  const double* spec_bin;  // optional per-bin specularity, or null
  uint64_t* spec_thr;      // [n] its thresholds (when given)
  double T_lin;
  double *C, *w_emit, *w_init, *w_relax, *v_nm, *inv_v, *lam, *pi, *sums;
  double* lam2;            // [n] v tau_imp (nm), +inf without a two-phonon clock
  double* prob;        // [3][n]
  uint64_t* thr;       // [3][n]
  int32_t* alias;      // [3][n]
  uint4* rec;          // [3][n]
  float4* binf;        // [n]
  double* scratch_p;   // [3][n]
  int* scratch_small;  // [3][n]
  int* scratch_large;  // [3][n]
};

cudaError_t launch_material_build(const MatBuild& b, cudaStream_t s);

int sm_count();
// bytes of one parked particle of the FP32 steady tracer's tail (both passes)
size_t park_record_bytes();

}  // namespace mcbte
