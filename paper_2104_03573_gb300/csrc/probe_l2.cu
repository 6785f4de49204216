// Measurement utility: the GPU's rate of 64-bit integer reductions into an
// L2-resident array, in the access pattern of the FP32 transient snapshots
// (four adds into one cell's 32-byte record, cells spread over the window's
// tally slice).  The bench times it to bound snapshot-dominated transient
// runs; the method itself does not use it.
#include "launch.h"

namespace mcbte {
namespace {

// splitmix64 finaliser (Steele, Lea, Flood, OOPSLA 2014): spreads the group
// index over the array's records
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__global__ void k_l2_reduction_probe(unsigned long long* slots, uint64_t n_rec, uint64_t n_groups) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_groups; g += stride) {
    unsigned long long* r = slots + (mix64(g) % n_rec) * 4;
    atomicAdd(r + 0, 1ull);
    atomicAdd(r + 1, 1ull);
    atomicAdd(r + 2, 1ull);
    atomicAdd(r + 3, 1ull);
  }
}

}  // namespace

cudaError_t launch_l2_reduction_probe(unsigned long long* slots, uint64_t n_rec, uint64_t n_groups, cudaStream_t s) {
  k_l2_reduction_probe<<<sm_count() * 8, 256, 0, s>>>(slots, n_rec, n_groups);
  return cudaGetLastError();
}

}  // namespace mcbte
