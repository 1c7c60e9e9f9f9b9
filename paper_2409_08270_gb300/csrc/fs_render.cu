// Novel-view mask rendering (Sec. 3.4; Supp. Sec. 8.2): the segmentation's
// objects are rendered one at a time into views that may have no mask.
//
// A view batch is projected and depth-sorted once.  For object e the sorted
// slots are compacted to the visible members of {G_i}_e (order kept), binned
// into tiles in one list, and composited per pixel (Eq. 1 over the subset):
// rho^e = sum alpha T and the alpha-weighted depth sum.  The same pass folds
// the object into the mask: where rho^e > tau and its depth D^e = sum alpha T
// z / rho^e is below the best depth so far, the pixel takes label e.  Objects
// run in increasing e, so equal depths keep the smaller e.
#include <cuda_fp16.h>

#include "fs_common.cuh"
#include "fs_internal.h"

namespace fs {

namespace {

// flag[k] = 1 iff sorted slot k is visible and its Gaussian has bit `bit`.
__global__ void __launch_bounds__(256) member_flag_kernel(
    int64_t k_total, int64_t n, const uint32_t* __restrict__ sorted_val,
    const uint32_t* __restrict__ cnt, const uint64_t* __restrict__ member, uint64_t bit,
    uint32_t* __restrict__ flag) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= k_total) return;
  const uint32_t slot = sorted_val[k];
  const int64_t i = static_cast<int64_t>(slot) % n;
  flag[k] = (cnt[slot] != 0u && (member[i] & bit) != 0ull) ? 1u : 0u;
}

// out[offs[k]] = sorted_val[k] where flag[k]: the flagged slots, in order.
__global__ void __launch_bounds__(256) member_scatter_kernel(
    int64_t k_total, const uint32_t* __restrict__ flag, const uint32_t* __restrict__ offs,
    const uint32_t* __restrict__ sorted_val, uint32_t* __restrict__ out) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < k_total && flag[k]) out[offs[k]] = sorted_val[k];
}

constexpr int kRenderThreads = kTilePixels;  // one thread per pixel of a 16x16 tile

// One block per (tile, view); the tile's list is walked in depth order in
// batches of 256 records staged in shared memory.  Plain FP32 compositing
// with the solve's rules: alpha = min(0.99, o 2^-|W (p - m)|^2), skipped
// below 1/255, and the pixel stops before a Gaussian that takes T below
// 1e-4.  best[] holds, per pixel of the batch, the smallest depth of a
// passing object so far (written on the first object).
template <typename OutT>
__global__ void __launch_bounds__(kRenderThreads) render_kernel(
    const ViewParams* __restrict__ views, const RenderOut* __restrict__ outs,
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ list_val,
    const ProjRecord* __restrict__ rec, const CompactRecord* __restrict__ rec16, int e,
    int first, float tau, float* __restrict__ best) {
  __shared__ float4 s_w[kRenderThreads];  // W (row-major 2x2)
  __shared__ float4 s_m[kRenderThreads];  // mean as float pairs (mx, my, mx_lo, my_lo)
  __shared__ float4 s_o[kRenderThreads];  // (-log2 o, clamp, depth, -)
  const int v = blockIdx.y;
  const ViewParams& vp = views[v];
  const int tiles_x = vp.tiles_x;
  const int tile = blockIdx.x;
  if (tile >= tiles_x * vp.tiles_y) return;  // whole block
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int px = tx * kTile + (threadIdx.x & (kTile - 1));
  const int py = ty * kTile + threadIdx.x / kTile;
  const bool inside = px < vp.width && py < vp.height;
  const uint2 rg = ranges[vp.tile_base + tile];
  const float pxc = static_cast<float>(px) + 0.5f, pyc = static_cast<float>(py) + 0.5f;
  float T = 1.f, rho = 0.f, zsum = 0.f;
  bool done = !inside;
  for (uint32_t base = rg.x; base < rg.y; base += kRenderThreads) {
    if (__syncthreads_and(done ? 1 : 0)) break;  // every pixel of the tile stopped
    const uint32_t k = base + threadIdx.x;
    if (k < rg.y) {
      const uint32_t g = list_val[k];
      if (rec16) {
        const CompactRecord r = rec16[g];
        const float2 wa = __half22float2(*reinterpret_cast<const __half2*>(&r.w01));
        const float2 wb = __half22float2(*reinterpret_cast<const __half2*>(&r.w23));
        s_w[threadIdx.x] = make_float4(wa.x, wa.y, wb.x, wb.y);
        s_m[threadIdx.x] = make_float4(r.mx, r.my, 0.f, 0.f);
        s_o[threadIdx.x] = make_float4(r.nlo, r.o > kAlphaMax ? 1.f : 0.f, r.depth, 0.f);
      } else {
        const ProjRecord r = rec[g];
        s_w[threadIdx.x] = r.w_hi;
        s_m[threadIdx.x] = r.m;
        s_o[threadIdx.x] = make_float4(r.misc.z, r.misc.x > kAlphaMax ? 1.f : 0.f, r.misc.w, 0.f);
      }
    }
    __syncthreads();
    const int count = static_cast<int>(min(rg.y - base, static_cast<uint32_t>(kRenderThreads)));
    for (int j = 0; j < count && !done; ++j) {
      const float4 w = s_w[j], m = s_m[j], o = s_o[j];
      const float dx = (pxc - m.x) - m.z, dy = (pyc - m.y) - m.w;
      const float w0 = fmaf(w.x, dx, w.y * dy), w1 = fmaf(w.z, dx, w.w * dy);
      float alpha = ex2_approx(-fmaf(w0, w0, fmaf(w1, w1, o.x)));
      if (o.y != 0.f) alpha = fminf(alpha, kAlphaMax);
      if (alpha < kAlphaMin) continue;
      const float t_next = T * (1.f - alpha);
      if (t_next < kTMin) {
        done = true;
        break;
      }
      const float c = alpha * T;
      rho += c;
      zsum = fmaf(c, o.z, zsum);
      T = t_next;
    }
    __syncthreads();  // the batch is read by every thread before the next one lands
  }
  if (!inside) return;
  const int64_t npix = static_cast<int64_t>(vp.width) * vp.height;
  const int64_t p = static_cast<int64_t>(py) * vp.width + px;
  const RenderOut ro = outs[v];
  const float depth = rho > 0.f ? zsum / rho : 0.f;
  if (ro.rho) ro.rho[static_cast<int64_t>(e - 1) * npix + p] = rho;
  if (ro.depth) ro.depth[static_cast<int64_t>(e - 1) * npix + p] = depth;
  float* const bp = best + vp.state_off + p;
  OutT* const mp = static_cast<OutT*>(ro.mask) + p;
  float b = first ? __int_as_float(0x7f800000) : *bp;
  OutT lab = first ? static_cast<OutT>(0) : *mp;
  if (rho > tau && depth < b) {
    b = depth;
    lab = static_cast<OutT>(e);
  }
  *bp = b;
  *mp = lab;
}

}  // namespace

cudaError_t launch_member_select(int64_t k_total, int64_t n, const uint32_t* sorted_val,
                                 const uint32_t* cnt, const uint64_t* member, uint64_t bit,
                                 uint32_t* flag, cudaStream_t stream) {
  if (k_total == 0) return cudaSuccess;
  member_flag_kernel<<<static_cast<unsigned>((k_total + 255) / 256), 256, 0, stream>>>(
      k_total, n, sorted_val, cnt, member, bit, flag);
  return cudaGetLastError();
}

cudaError_t launch_member_scatter(int64_t k_total, const uint32_t* flag, const uint32_t* offs,
                                  const uint32_t* sorted_val, uint32_t* out,
                                  cudaStream_t stream) {
  if (k_total == 0) return cudaSuccess;
  member_scatter_kernel<<<static_cast<unsigned>((k_total + 255) / 256), 256, 0, stream>>>(
      k_total, flag, offs, sorted_val, out);
  return cudaGetLastError();
}

cudaError_t launch_render(const ViewParams* views, const RenderOut* outs, int n_views,
                          int max_tiles_per_view, const uint2* ranges, const uint32_t* list_val,
                          const ProjRecord* rec, const CompactRecord* rec16, int e, bool first,
                          float tau, float* best, int out_dtype, cudaStream_t stream) {
  if (n_views == 0 || max_tiles_per_view == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(max_tiles_per_view), static_cast<unsigned>(n_views));
  if (out_dtype == 4)
    render_kernel<uint8_t><<<grid, kRenderThreads, 0, stream>>>(
        views, outs, ranges, list_val, rec, rec16, e, first ? 1 : 0, tau, best);
  else
    render_kernel<int32_t><<<grid, kRenderThreads, 0, stream>>>(
        views, outs, ranges, list_val, rec, rec16, e, first ? 1 : 0, tau, best);
  return cudaGetLastError();
}

}  // namespace fs
