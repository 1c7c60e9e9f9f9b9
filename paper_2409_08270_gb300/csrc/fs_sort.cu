// Device exclusive scan and stable LSD radix sort of (uint32 key, uint32 value)
// pairs, used for the depth order and the tile binning of Sec. 3.1.
//
// Both work on tiles of 4096 elements per 256-thread block.  The radix sort
// is the classic three-step pass (per-block digit histogram, scan of the
// histogram in digit-major order, stable scatter).  No step waits on another
// block.
#include "fs_internal.h"

namespace fs {

namespace {

constexpr int kThreads = 256;
constexpr int kRounds = 16;
constexpr int kTileElems = kThreads * kRounds;
constexpr int kWarps = kThreads / 32;
constexpr int kRadix = 256;

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Exclusive scan of one value per thread across the block; returns the
// thread's exclusive prefix and writes the block total to *total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* s_warp,
                                                          uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  uint32_t warp_pre = 0, all = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const uint32_t c = s_warp[w];
    if (w < warp) warp_pre += c;
    all += c;
  }
  __syncthreads();
  *total = all;
  return warp_pre + inc - x;
}

__device__ __forceinline__ uint32_t load_in(const uint32_t* in, const uint32_t* gather, int64_t j) {
  return gather ? in[gather[j]] : in[j];
}

__global__ void __launch_bounds__(kThreads) scan_reduce_kernel(const uint32_t* __restrict__ in,
                                                               const uint32_t* __restrict__ gather,
                                                               int64_t n,
                                                               uint32_t* __restrict__ block_sums) {
  __shared__ uint32_t s_warp[kWarps];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTileElems;
  uint32_t acc = 0;
#pragma unroll 4
  for (int r = 0; r < kRounds; ++r) {
    const int64_t j = base + r * kThreads + threadIdx.x;
    if (j < n) acc += load_in(in, gather, j);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kWarps; ++w) t += s_warp[w];
    block_sums[blockIdx.x] = t;
  }
}

// Single block: exclusive scan of the block sums in place, total to *total.
__global__ void __launch_bounds__(kThreads) scan_blocks_kernel(uint32_t* __restrict__ sums,
                                                               int64_t nb,
                                                               uint32_t* __restrict__ total) {
  __shared__ uint32_t s_warp[kWarps];
  uint32_t carry = 0;
  for (int64_t base = 0; base < nb; base += kThreads) {
    const int64_t j = base + threadIdx.x;
    const uint32_t x = j < nb ? sums[j] : 0u;
    uint32_t t;
    const uint32_t ex = block_exclusive_scan(x, s_warp, &t);
    if (j < nb) sums[j] = carry + ex;
    carry += t;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(kThreads) scan_down_kernel(const uint32_t* __restrict__ in,
                                                             const uint32_t* __restrict__ gather,
                                                             int64_t n,
                                                             const uint32_t* __restrict__ block_pre,
                                                             uint32_t* __restrict__ out) {
  __shared__ uint32_t s_warp[kWarps];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTileElems;
  uint32_t carry = block_pre[blockIdx.x];
  for (int r = 0; r < kRounds; ++r) {
    const int64_t j = base + r * kThreads + threadIdx.x;
    const uint32_t x = j < n ? load_in(in, gather, j) : 0u;
    uint32_t t;
    const uint32_t ex = block_exclusive_scan(x, s_warp, &t);
    if (j < n) out[j] = carry + ex;
    carry += t;
  }
}

// Digits are taken from min(key - kmin, span): a key range [kmin, kmin + span)
// (and everything above it mapped to span) needs only the bits of span.
__device__ __forceinline__ uint32_t digit_of(uint32_t key, uint32_t kmin, uint32_t span,
                                             int shift) {
  return (min(key - kmin, span) >> shift) & 0xFFu;
}

__global__ void __launch_bounds__(kThreads) radix_hist_kernel(const uint32_t* __restrict__ keys,
                                                              int64_t n, int shift, int64_t nb,
                                                              uint32_t kmin, uint32_t span,
                                                              uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_h[kRadix];
  s_h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTileElems;
#pragma unroll 4
  for (int r = 0; r < kRounds; ++r) {
    const int64_t j = base + r * kThreads + threadIdx.x;
    if (j < n) atomicAdd(&s_h[digit_of(keys[j], kmin, span, shift)], 1u);
  }
  __syncthreads();
  hist[static_cast<int64_t>(threadIdx.x) * nb + blockIdx.x] = s_h[threadIdx.x];
}

// Stable scatter of one radix pass.  Each warp ranks its 512 elements (16
// coalesced columns of 32) by digit with a warp match per column and per-warp
// digit counters, so equal digits keep their input order; the block then
// turns (digit, warp) counts into local offsets, places its 4096 elements
// digit-sorted in shared memory and writes each digit's run to its global
// offset with consecutive threads on consecutive addresses.
__global__ void __launch_bounds__(kThreads) radix_scatter_kernel(
    const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t n, int shift,
    int64_t nb, uint32_t kmin, uint32_t span, const uint32_t* __restrict__ hist_pre,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out) {
  __shared__ uint32_t s_key[kTileElems];
  __shared__ uint32_t s_val[kTileElems];
  __shared__ uint32_t s_wcnt[kWarps][kRadix];  // per-warp digit counts, then warp prefixes
  __shared__ uint32_t s_loc[kRadix];           // local start of each digit's run
  __shared__ uint32_t s_glob[kRadix];          // global start of this block's run per digit
  __shared__ uint32_t s_warp[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTileElems;
  const int n_here = static_cast<int>(min(static_cast<int64_t>(kTileElems), n - base));
  const int wbase = warp * (kTileElems / kWarps);  // 512 elements per warp
#pragma unroll
  for (int k = 0; k < kRadix / 32; ++k) s_wcnt[warp][lane + 32 * k] = 0;
  __syncwarp();

  const uint32_t lt = lanemask_lt();
  uint32_t key[kRounds], rank[kRounds];
#pragma unroll
  for (int i = 0; i < kRounds; ++i) {
    const int j = wbase + i * 32 + lane;
    const bool ok = j < n_here;
    key[i] = ok ? keys[base + j] : 0u;
    const uint32_t d = ok ? digit_of(key[i], kmin, span, shift) : 0x100u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = ok ? s_wcnt[warp][d] : 0u;
    rank[i] = before + __popc(peers & lt);
    __syncwarp();
    if (ok && (peers & lt) == 0) s_wcnt[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit (thread t): warp prefixes, then the block-wide digit offsets
  uint32_t running = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const uint32_t c = s_wcnt[w][threadIdx.x];
    s_wcnt[w][threadIdx.x] = running;
    running += c;
  }
  uint32_t tot;
  s_loc[threadIdx.x] = block_exclusive_scan(running, s_warp, &tot);
  s_glob[threadIdx.x] = hist_pre[static_cast<int64_t>(threadIdx.x) * nb + blockIdx.x];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kRounds; ++i) {
    const int j = wbase + i * 32 + lane;
    if (j < n_here) {
      const uint32_t d = digit_of(key[i], kmin, span, shift);
      const uint32_t pos = s_loc[d] + s_wcnt[warp][d] + rank[i];
      s_key[pos] = key[i];
      s_val[pos] = vals[base + j];
    }
  }
  __syncthreads();
  // coalesced write-out of the digit runs
  for (int j = threadIdx.x; j < n_here; j += kThreads) {
    const uint32_t k = s_key[j];
    const uint32_t d = digit_of(k, kmin, span, shift);
    const uint32_t dst = s_glob[d] + (static_cast<uint32_t>(j) - s_loc[d]);
    keys_out[dst] = k;
    vals_out[dst] = s_val[j];
  }
}

inline int64_t tiles_of(int64_t n) { return (n + kTileElems - 1) / kTileElems; }

}  // namespace

size_t scan_temp_bytes(int64_t n) {
  return static_cast<size_t>(tiles_of(n) + 1) * sizeof(uint32_t);
}

cudaError_t exclusive_scan(const uint32_t* in, const uint32_t* gather, uint32_t* out, int64_t n,
                           uint32_t* total, void* temp, cudaStream_t stream) {
  if (n <= 0) {
    if (total) return cudaMemsetAsync(total, 0, sizeof(uint32_t), stream);
    return cudaSuccess;
  }
  const int64_t nb = tiles_of(n);
  uint32_t* sums = static_cast<uint32_t*>(temp);
  scan_reduce_kernel<<<static_cast<unsigned>(nb), kThreads, 0, stream>>>(in, gather, n, sums);
  scan_blocks_kernel<<<1, kThreads, 0, stream>>>(sums, nb, total);
  scan_down_kernel<<<static_cast<unsigned>(nb), kThreads, 0, stream>>>(in, gather, n, sums, out);
  return cudaGetLastError();
}

size_t radix_temp_bytes(int64_t n) {
  const int64_t nb = tiles_of(n);
  const int64_t hist = nb * kRadix;
  return static_cast<size_t>(hist) * sizeof(uint32_t) + scan_temp_bytes(hist) + 256;
}

cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                             uint32_t* vals_alt, int64_t n, int bits, void* temp, bool* in_alt,
                             cudaStream_t stream, uint32_t kmin, uint32_t span) {
  *in_alt = false;
  if (n <= 1 || bits <= 0) return cudaSuccess;
  const int64_t nb = tiles_of(n);
  uint32_t* hist = static_cast<uint32_t*>(temp);
  void* scan_tmp = reinterpret_cast<char*>(temp) +
                   ((static_cast<size_t>(nb) * kRadix * sizeof(uint32_t) + 255) / 256) * 256;
  uint32_t *src_k = keys, *src_v = vals, *dst_k = keys_alt, *dst_v = vals_alt;
  for (int shift = 0; shift < bits; shift += 8) {
    radix_hist_kernel<<<static_cast<unsigned>(nb), kThreads, 0, stream>>>(src_k, n, shift, nb,
                                                                          kmin, span, hist);
    cudaError_t e = exclusive_scan(hist, nullptr, hist, nb * kRadix, nullptr, scan_tmp, stream);
    if (e != cudaSuccess) return e;
    radix_scatter_kernel<<<static_cast<unsigned>(nb), kThreads, 0, stream>>>(
        src_k, src_v, n, shift, nb, kmin, span, hist, dst_k, dst_v);
    uint32_t* tk = src_k;
    uint32_t* tv = src_v;
    src_k = dst_k;
    src_v = dst_v;
    dst_k = tk;
    dst_v = tv;
    *in_alt = !*in_alt;
  }
  return cudaGetLastError();
}

}  // namespace fs
