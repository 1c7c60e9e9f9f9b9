// Device-side sizes for a solve captured into a CUDA graph (fs_graph_* in
// flashsplat.h).  A captured solve reads nothing back to the host: the depth
// chunks are cut from the visible count the projection left on the device,
// the binning, the tile sort and the ranges read their counts from device
// memory, and the grids are sized for the capacities of the capture's plan.
// A replay whose sizes outgrow that plan is reported, not run past it.
#include "fs_common.cuh"
#include "fs_internal.h"

namespace fs {

namespace {

// Chunk ci of k visible slots in `chunks` front-to-back chunks ends at
// k >> (chunks - 1 - ci) (the last at k): sizes 1/32, 1/32, 1/16 ... 1/2.
__global__ void chunk_bounds_kernel(const uint32_t* __restrict__ key_range, int chunks,
                                    int64_t* __restrict__ bnd) {
  if (threadIdx.x != 0) return;
  const int64_t k = key_range[0] <= key_range[1] ? static_cast<int64_t>(key_range[2]) : 0;
  bnd[0] = 0;
  for (int ci = 0; ci < chunks; ++ci) bnd[ci + 1] = ci == chunks - 1 ? k : (k >> (chunks - 1 - ci));
}

__global__ void chunk_last_kernel(const int64_t* __restrict__ bnd, int chunks,
                                  const uint32_t* __restrict__ sorted_val,
                                  uint32_t* __restrict__ bound) {
  const int ci = threadIdx.x;
  if (ci + 1 >= chunks) return;
  const int64_t p0 = bnd[ci], p1 = bnd[ci + 1];
  bound[ci] = p1 > p0 ? sorted_val[p1 - 1] : 0xFFFFFFFFu;
}

__global__ void __launch_bounds__(256) copy_count_kernel(const uint32_t* __restrict__ src,
                                                         uint32_t* __restrict__ dst,
                                                         const uint32_t* __restrict__ n_dev,
                                                         int64_t cap) {
  const int64_t n = min(cap, static_cast<int64_t>(*n_dev));
  for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dst[k] = src[k];
}

__global__ void graph_check_kernel(const uint32_t* __restrict__ total, uint32_t capacity,
                                   const uint32_t* __restrict__ key_range, int key_bits,
                                   const int64_t* __restrict__ rng, int64_t rng_cap,
                                   unsigned long long* __restrict__ counters) {
  if (threadIdx.x != 0) return;
  if (total && *total > capacity) atomicAdd(&counters[kGraphOverflow], 1ull);
  if (rng && rng[1] - rng[0] > rng_cap) atomicAdd(&counters[kGraphOverflow], 1ull);
  if (key_range && key_range[0] <= key_range[1]) {
    // the sort maps visible keys to 0 .. span - 1 and the others to span
    const uint64_t span = static_cast<uint64_t>(key_range[1] - key_range[0]) + 1u;
    if (key_bits < 32 && span >= (1ull << key_bits)) atomicAdd(&counters[kGraphKeyRange], 1ull);
  }
}

}  // namespace

cudaError_t launch_chunk_bounds(const uint32_t* key_range, int chunks, int64_t* bnd,
                                cudaStream_t stream) {
  chunk_bounds_kernel<<<1, 32, 0, stream>>>(key_range, chunks, bnd);
  return cudaGetLastError();
}

cudaError_t launch_chunk_last(const int64_t* bnd, int chunks, const uint32_t* sorted_val,
                              uint32_t* bound, cudaStream_t stream) {
  if (chunks < 2) return cudaSuccess;
  chunk_last_kernel<<<1, 32, 0, stream>>>(bnd, chunks, sorted_val, bound);
  return cudaGetLastError();
}

cudaError_t launch_copy_count(const uint32_t* src, uint32_t* dst, const uint32_t* n_dev,
                              int64_t cap, cudaStream_t stream) {
  if (cap <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((cap + 255) / 256, 4096);
  copy_count_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(src, dst, n_dev, cap);
  return cudaGetLastError();
}

cudaError_t launch_graph_check(const uint32_t* total, uint32_t capacity,
                               const uint32_t* key_range, int key_bits, const int64_t* rng,
                               int64_t rng_cap, unsigned long long* counters,
                               cudaStream_t stream) {
  graph_check_kernel<<<1, 32, 0, stream>>>(total, capacity, key_range, key_bits, rng, rng_cap,
                                           counters);
  return cudaGetLastError();
}

}  // namespace fs
