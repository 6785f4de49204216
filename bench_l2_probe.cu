// Measurement utility of bench.py, built beside it (not part of the MCBTE
// library): the GPU's rate of 64-bit integer reductions into an L2-resident
// array, in the access pattern of the FP32 transient snapshots (four adds
// into one cell's 32-byte record, cells spread over a time window's tally
// slice).  The bench times it to bound snapshot-dominated transient runs.
#include <cstdint>
#include <cuda_runtime.h>

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

// n_groups groups of four adds of 1 into the 4-word records of `slots`
// (device memory, n_slots words, a positive multiple of 4) on `stream`
// (a cudaStream_t, or null).  Returns 0, 1 for bad sizes (checked before any
// CUDA call), 2 for a CUDA error.
extern "C" int bench_l2_reduction_probe(long long* slots, uint64_t n_slots, uint64_t n_groups, void* stream) {
  if (!slots || n_slots < 4 || (n_slots & 3u) != 0) return 1;
  if (n_groups == 0) return 0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 2;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 2;
  k_l2_reduction_probe<<<sms * 8, 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<unsigned long long*>(slots),
                                                                   n_slots / 4, n_groups);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
