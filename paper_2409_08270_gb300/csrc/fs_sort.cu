// Device exclusive scan and stable LSD radix sort of (uint32 key, uint32 value)
// pairs, used for the depth order and the tile binning of Sec. 3.1.
//
// Both work on tiles of 4096 elements per 256-thread block.  The radix sort
// is the classic three-step pass (per-block digit histogram, scan of the
// histogram in digit-major order, stable scatter).  No step waits on another
// block.
#include <atomic>

#include "fs_internal.h"

namespace fs {

namespace {

constexpr int kThreads = 256;
constexpr int kRounds = 16;
constexpr int kTileElems = kThreads * kRounds;
constexpr int kWarps = kThreads / 32;

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
  uint32_t x[kRounds];
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int64_t j = base + r * kThreads + threadIdx.x;
    x[r] = j < n ? load_in(in, gather, j) : 0u;
  }
  uint32_t acc = 0;
#pragma unroll
  for (int r = 0; r < kRounds; ++r) acc += x[r];
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
  // all loads in flight before the first block barrier
  uint32_t x[kRounds];
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int64_t j = base + r * kThreads + threadIdx.x;
    x[r] = j < n ? load_in(in, gather, j) : 0u;
  }
  uint32_t carry = block_pre[blockIdx.x];
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int64_t j = base + r * kThreads + threadIdx.x;
    uint32_t t;
    const uint32_t ex = block_exclusive_scan(x[r], s_warp, &t);
    if (j < n) out[j] = carry + ex;
    carry += t;
  }
}

// Digits are taken from min(key - kmin, span): a key range [kmin, kmin + span)
// (and everything above it mapped to span) needs only the bits of span.
// A pass takes DB bits (8 or 9: a 17-bit tile key sorts in two passes).
template <int DB>
__device__ __forceinline__ uint32_t digit_of(uint32_t key, uint32_t kmin, uint32_t span,
                                             int shift) {
  return (min(key - kmin, span) >> shift) & ((1u << DB) - 1u);
}

// Sizes read on the device (a launch captured once and replayed): the element
// count *n_dev (at most the n the grid was sized for) and the key range
// range_dev[0..1] (min, max of the keys that sort first; min > max: none).
// NULL pointers keep the launch's own values.
__device__ __forceinline__ void device_sizes(const uint32_t* n_dev, const uint32_t* range_dev,
                                             int64_t* n, uint32_t* kmin, uint32_t* span) {
  if (n_dev) *n = min(*n, static_cast<int64_t>(*n_dev));
  if (range_dev) {
    const uint32_t lo = range_dev[0], hi = range_dev[1];
    *kmin = lo <= hi ? lo : 0u;
    *span = lo <= hi ? hi - lo + 1u : 0u;
  }
}

template <int DB>
__global__ void __launch_bounds__(kThreads) radix_hist_kernel(const uint32_t* __restrict__ keys,
                                                              int64_t n, int shift, int64_t nb,
                                                              uint32_t kmin, uint32_t span,
                                                              uint32_t* __restrict__ hist,
                                                              const uint32_t* __restrict__ n_dev,
                                                              const uint32_t* __restrict__ range_dev) {
  constexpr int kRad = 1 << DB;
  device_sizes(n_dev, range_dev, &n, &kmin, &span);
  __shared__ uint32_t s_h[kRad];
  for (int d = threadIdx.x; d < kRad; d += kThreads) s_h[d] = 0;
  __syncthreads();
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTileElems;
  // all of the thread's loads in flight before the first count
  uint32_t key[kRounds];
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int64_t j = base + r * kThreads + threadIdx.x;
    key[r] = j < n ? keys[j] : 0u;
  }
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int64_t j = base + r * kThreads + threadIdx.x;
    if (j < n) atomicAdd(&s_h[digit_of<DB>(key[r], kmin, span, shift)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRad; d += kThreads)
    hist[static_cast<int64_t>(d) * nb + blockIdx.x] = s_h[d];
}

// Shared memory of one scatter block (dynamic: the 9-bit form needs 52 KB).
template <int DB>
struct ScatterSmem {
  uint32_t key[kTileElems];
  uint32_t val[kTileElems];
  uint32_t wcnt[kWarps][1 << DB];  // per-warp digit counts, then warp prefixes
  uint32_t loc[1 << DB];           // local start of each digit's run
  uint32_t glob[1 << DB];          // global start of this block's run per digit
  uint32_t warp_sums[kWarps];
};

// Stable scatter of one radix pass.  Each warp ranks its 512 elements (16
// coalesced columns of 32) by digit with a warp match per column and per-warp
// digit counters, so equal digits keep their input order; the block then
// turns (digit, warp) counts into local offsets, places its 4096 elements
// digit-sorted in shared memory and writes each digit's run to its global
// offset with consecutive threads on consecutive addresses.
template <int DB>
__global__ void __launch_bounds__(kThreads) radix_scatter_kernel(
    const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t n, int shift,
    int64_t nb, uint32_t kmin, uint32_t span, const uint32_t* __restrict__ hist_pre,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
    const uint32_t* __restrict__ n_dev, const uint32_t* __restrict__ range_dev) {
  constexpr int kRad = 1 << DB;
  device_sizes(n_dev, range_dev, &n, &kmin, &span);
  constexpr int kPer = kRad / kThreads;  // digits per thread in the block-wide steps
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScatterSmem<DB>& S = *reinterpret_cast<ScatterSmem<DB>*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTileElems;
  const int n_here =
      static_cast<int>(max(static_cast<int64_t>(0), min(static_cast<int64_t>(kTileElems), n - base)));
  const int wbase = warp * (kTileElems / kWarps);  // 512 elements per warp
#pragma unroll
  for (int k = 0; k < kRad / 32; ++k) S.wcnt[warp][lane + 32 * k] = 0;
  __syncwarp();

  const uint32_t lt = lanemask_lt();
  uint32_t key[kRounds], rank[kRounds];
  // all of the warp's key loads in flight at once (the ranking below has
  // warp barriers, which no load is moved across)
#pragma unroll
  for (int i = 0; i < kRounds; ++i) {
    const int j = wbase + i * 32 + lane;
    key[i] = j < n_here ? keys[base + j] : 0u;
  }
#pragma unroll
  for (int i = 0; i < kRounds; ++i) {
    const int j = wbase + i * 32 + lane;
    const bool ok = j < n_here;
    const uint32_t d = ok ? digit_of<DB>(key[i], kmin, span, shift) : static_cast<uint32_t>(kRad);
    // lanes holding the same digit: one ballot per digit bit
    uint32_t peers = __ballot_sync(0xffffffffu, ok);
    if (!ok) peers = ~peers;
#pragma unroll
    for (int b = 0; b < DB; ++b) {
      const bool bit = (d >> b) & 1u;
      const uint32_t bb = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? bb : ~bb;
    }
    const uint32_t before = ok ? S.wcnt[warp][d] : 0u;
    rank[i] = before + __popc(peers & lt);
    __syncwarp();
    if (ok && (peers & lt) == 0) S.wcnt[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit (thread t holds digits t * kPer .. t * kPer + kPer - 1): warp
  // prefixes, then the block-wide digit offsets
  uint32_t running[kPer], own = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int d = threadIdx.x * kPer + q;
    running[q] = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = S.wcnt[w][d];
      S.wcnt[w][d] = running[q];
      running[q] += c;
    }
    own += running[q];
  }
  uint32_t tot;
  uint32_t ex = block_exclusive_scan(own, S.warp_sums, &tot);
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int d = threadIdx.x * kPer + q;
    S.loc[d] = ex;
    ex += running[q];
    S.glob[d] = hist_pre[static_cast<int64_t>(d) * nb + blockIdx.x];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kRounds; ++i) {
    const int j = wbase + i * 32 + lane;
    if (j < n_here) {
      const uint32_t d = digit_of<DB>(key[i], kmin, span, shift);
      const uint32_t pos = S.loc[d] + S.wcnt[warp][d] + rank[i];
      S.key[pos] = key[i];
      S.val[pos] = vals[base + j];
    }
  }
  __syncthreads();
  // coalesced write-out of the digit runs
#pragma unroll
  for (int i = 0; i < kRounds; ++i) {
    const int j = i * kThreads + threadIdx.x;
    if (j < n_here) {
      const uint32_t k = S.key[j];
      const uint32_t d = digit_of<DB>(k, kmin, span, shift);
      const uint32_t dst = S.glob[d] + (static_cast<uint32_t>(j) - S.loc[d]);
      keys_out[dst] = k;
      vals_out[dst] = S.val[j];
    }
  }
}

template <int DB>
cudaError_t radix_pass(const uint32_t* src_k, const uint32_t* src_v, uint32_t* dst_k,
                       uint32_t* dst_v, int64_t n, int shift, int64_t nb, uint32_t kmin,
                       uint32_t span, uint32_t* hist, void* scan_tmp, cudaStream_t stream,
                       const uint32_t* n_dev, const uint32_t* range_dev);

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
  const int64_t hist = nb * 512;  // the widest digit
  return static_cast<size_t>(hist) * sizeof(uint32_t) + scan_temp_bytes(hist) + 256;
}

namespace {

template <int DB>
cudaError_t radix_pass(const uint32_t* src_k, const uint32_t* src_v, uint32_t* dst_k,
                       uint32_t* dst_v, int64_t n, int shift, int64_t nb, uint32_t kmin,
                       uint32_t span, uint32_t* hist, void* scan_tmp, cudaStream_t stream,
                       const uint32_t* n_dev, const uint32_t* range_dev) {
  constexpr int kRad = 1 << DB;
  const size_t smem = sizeof(ScatterSmem<DB>);
  // dynamic shared memory above 48 KB needs the opt-in, once per device
  static std::atomic<uint64_t> attr_set{0};
  int dev = 0;
  cudaError_t e0 = cudaGetDevice(&dev);
  if (e0 != cudaSuccess) return e0;
  const uint64_t bit = 1ull << (dev & 63);
  if (!(attr_set.load() & bit)) {
    cudaError_t e = cudaFuncSetAttribute(radix_scatter_kernel<DB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    attr_set.fetch_or(bit);
  }
  radix_hist_kernel<DB><<<static_cast<unsigned>(nb), kThreads, 0, stream>>>(
      src_k, n, shift, nb, kmin, span, hist, n_dev, range_dev);
  cudaError_t e = exclusive_scan(hist, nullptr, hist, nb * kRad, nullptr, scan_tmp, stream);
  if (e != cudaSuccess) return e;
  radix_scatter_kernel<DB><<<static_cast<unsigned>(nb), kThreads, smem, stream>>>(
      src_k, src_v, n, shift, nb, kmin, span, hist, dst_k, dst_v, n_dev, range_dev);
  return cudaGetLastError();
}

}  // namespace

int radix_passes(int bits) {
  if (bits <= 0) return 0;
  return (bits + 8) / 9 < (bits + 7) / 8 ? (bits + 8) / 9 : (bits + 7) / 8;
}

cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                             uint32_t* vals_alt, int64_t n, int bits, void* temp, bool* in_alt,
                             cudaStream_t stream, uint32_t kmin, uint32_t span,
                             const uint32_t* n_dev, const uint32_t* range_dev) {
  *in_alt = false;
  if (n <= 1 || bits <= 0) return cudaSuccess;
  const int64_t nb = tiles_of(n);
  uint32_t* hist = static_cast<uint32_t*>(temp);
  void* scan_tmp = reinterpret_cast<char*>(temp) +
                   ((static_cast<size_t>(nb) * 512 * sizeof(uint32_t) + 255) / 256) * 256;
  // digit widths: 8 bits, or 9 where that saves a whole pass (17 -> 9 + 8)
  const int passes = radix_passes(bits);
  int wide = bits - 8 * passes;  // passes that take 9 bits
  if (wide < 0) wide = 0;
  uint32_t *src_k = keys, *src_v = vals, *dst_k = keys_alt, *dst_v = vals_alt;
  int shift = 0;
  for (int p = 0; p < passes; ++p) {
    const bool nine = p < wide;
    cudaError_t e = nine ? radix_pass<9>(src_k, src_v, dst_k, dst_v, n, shift, nb, kmin, span,
                                         hist, scan_tmp, stream, n_dev, range_dev)
                         : radix_pass<8>(src_k, src_v, dst_k, dst_v, n, shift, nb, kmin, span,
                                         hist, scan_tmp, stream, n_dev, range_dev);
    if (e != cudaSuccess) return e;
    shift += nine ? 9 : 8;
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
