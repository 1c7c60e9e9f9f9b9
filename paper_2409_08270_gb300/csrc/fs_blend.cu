// Front-to-back alpha blending of every mask pixel and accumulation of
// alpha_i T_i into the contribution table (Sec. 3.1 Eq. 1, Sec. 3.2 Eq. 6,
// Sec. 3.3 Eq. 7, Sec. 4.2: each Gaussian's alpha_i T_i at a pixel goes into
// the table column of that pixel's label, added atomically).
//
// One warp per 8x8 sub-tile of a 16x16 tile; each lane walks two adjacent
// pixels; no block barriers.  A block holds the four independent warps of one
// tile and the kernel is held to 48 registers, so that 40 warps share an SM
// (registers and shared memory both allow 10 blocks) instead of the 32 that
// one-warp blocks allow.
//  * The warp reads its tile's depth-sorted list (one depth chunk of it) 32
//    entries at a time.  Each lane forms its entry's offset b = W o + c at the
//    sub-tile centre o (float pairs) and keeps the entry only when the
//    alpha >= 1/255 region can reach the sub-tile; kept entries are compacted
//    into shared memory in list order.
//  * Per pixel, per kept Gaussian, without branches and with packed FP32
//    pairs for the lane's two pixels: w = W p + b,
//    alpha = min(0.99, o 2^-|w|^2); alpha < 1/255 is skipped; the pixel stops
//    before a Gaussian that would take T below 1e-4; else it adds alpha*T.
//    The decisions are 1.0/0.0 factors, so a stopped pixel simply carries
//    T = 0.  T is kept per pixel across depth chunks (0 = stopped); a
//    sub-tile whose pixels have all stopped is done, and a tile with four
//    done sub-tiles is saturated (no later chunk lists it).
//  * No per-pixel atomics: the lane adds its two contributions when they
//    share a label and writes one value per Gaussian into a shared row whose
//    positions are ordered by label; lane j then sums Gaussian j's row per
//    label and issues one global atomic add per non-zero (Gaussian, label).
//    A lane whose two pixels straddle a label boundary adds its second
//    pixel's contribution with its own atomic.
#include <cuda_fp16.h>

#include "fs_common.cuh"
#include "fs_internal.h"

namespace fs {

namespace {

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename TableT>
__device__ __forceinline__ void table_add(TableT* p, float v) {
  atomicAdd(p, static_cast<TableT>(v));
}

// 1.0f if a >= b else 0.0f
__device__ __forceinline__ float step_ge(float a, float b) {
  float r;
  asm("set.ge.f32.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}

// One compositing step (Eq. 1) of the lane's two pixels, (x0, y) and
// (x0 + 1, y), branch-free and with packed FP32 pairs.  T == 0 marks a pixel
// that has stopped: its later steps give alpha' T = 0 and keep T = 0.
//   alpha = min(0.99, o 2^-|w|^2),  alpha' = alpha if alpha >= 1/255 else 0
//   T' = T (1 - alpha');  the pixel stops (T' < 1e-4) without adding,
//   else it adds alpha' T and continues with T'.
// `live` counts, per pixel, the steps taken while running on (not stopping).
__device__ __forceinline__ float2 composite2(const float4& W, const float4& bo, float2 X, float y,
                                             float2& T, float2& live) {
  const float t0 = fmaf(W.y, y, bo.x), t1 = fmaf(W.w, y, bo.y);
  const float2 w0 = __ffma2_rn(make_float2(W.x, W.x), X, make_float2(t0, t0));
  const float2 w1 = __ffma2_rn(make_float2(W.z, W.z), X, make_float2(t1, t1));
  const float2 q = __ffma2_rn(w0, w0, __fmul2_rn(w1, w1));
  float2 a = __fmul2_rn(make_float2(bo.z, bo.z), make_float2(ex2_approx(-q.x), ex2_approx(-q.y)));
  a.x = fminf(kAlphaMax, a.x);
  a.y = fminf(kAlphaMax, a.y);
  a = __fmul2_rn(a, make_float2(step_ge(a.x, kAlphaMin), step_ge(a.y, kAlphaMin)));
  const float2 tt = __ffma2_rn(make_float2(-T.x, -T.y), a, T);
  const float2 go = make_float2(step_ge(tt.x, kTMin), step_ge(tt.y, kTMin));
  const float2 c = __fmul2_rn(__fmul2_rn(a, T), go);
  T = __fmul2_rn(tt, go);
  live = __fadd2_rn(live, go);
  return c;
}

__device__ __forceinline__ void set_bit(uint64_t* bits, int i) {
  atomicOr(reinterpret_cast<unsigned long long*>(bits + (i >> 6)), 1ull << (i & 63));
}

// Per-pixel state of a batch before its first depth chunk: T = 1 for pixels
// with a label in [0, E), 0 ("stopped") for the others.  Sub-tiles (and tiles)
// without a labelled pixel start saturated.  Counts the pixels with bad
// labels.  One 256-thread block per 16x16 tile: 64 threads (two warps) per
// 8x8 sub-tile.
template <typename LabelT>
__global__ void __launch_bounds__(256) state_init_kernel(
    const ViewParams* __restrict__ views, int E, float* __restrict__ state,
    uint64_t* __restrict__ sat, uint64_t* __restrict__ subsat,
    unsigned long long* __restrict__ counters) {
  __shared__ uint32_t s_bad[8], s_any[8];
  const int v = blockIdx.y;
  const int tiles_x = views[v].tiles_x;
  const int tile = blockIdx.x;
  if (tile >= tiles_x * views[v].tiles_y) return;  // whole block
  const int W = views[v].width, H = views[v].height;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int sub = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int px = tx * kTile + (sub & 1) * 8 + (t & 7);
  const int py = ty * kTile + (sub >> 1) * 8 + (t >> 3);
  const bool inside = px < W && py < H;
  bool valid = false;
  if (inside) {
    const int64_t p = static_cast<int64_t>(py) * W + px;
    const int label = static_cast<int>(static_cast<const LabelT*>(views[v].mask)[p]);
    valid = label >= 0 && label < E;
    state[views[v].state_off + p] = valid ? 1.f : 0.f;
  }
  const uint32_t bad = __ballot_sync(0xffffffffu, inside && !valid);
  const uint32_t any = __ballot_sync(0xffffffffu, valid);
  if ((threadIdx.x & 31) == 0) {
    s_bad[threadIdx.x >> 5] = __popc(bad);
    s_any[threadIdx.x >> 5] = any;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t n_bad = 0, empty = 0;  // empty: bit s = sub-tile s has no labelled pixel
    for (int s = 0; s < 4; ++s) {
      n_bad += s_bad[2 * s] + s_bad[2 * s + 1];
      if ((s_any[2 * s] | s_any[2 * s + 1]) == 0u) empty |= 1u << s;
    }
    if (n_bad) atomicAdd(&counters[kBadLabels], static_cast<unsigned long long>(n_bad));
    if (empty) {
      const int g = views[v].tile_base + tile;
      const int gs = 4 * g;  // the tile's four sub-tile bits: one nibble of a word
      atomicOr(reinterpret_cast<unsigned long long*>(subsat + (gs >> 6)),
               static_cast<unsigned long long>(empty) << (gs & 63));
      if (empty == 0xFu) set_bit(sat, g);
    }
  }
}

// ---------------------------------------------------------------------------
// blend: one warp per 8x8 sub-tile, 2 adjacent pixels per lane, 4 warps a block
// ---------------------------------------------------------------------------
constexpr int kStage = 32;  // list entries examined per round (one per lane)

struct SubSmem {
  float4 w[kStage];       // whitening matrix of each staged Gaussian
  float4 bo[kStage];      // (b0, b1, opacity, -)
  int32_t gid[kStage];    // scene index of each staged Gaussian
  float buf[kStage][33];  // [Gaussian][lane position in label order]: main-label sums
  int32_t poslab[32];     // label of each lane position (INT_MAX: none)
};

template <typename LabelT, typename TableT>
__global__ void __launch_bounds__(128, 10) blend_kernel(
    const ViewParams* __restrict__ views, const uint2* __restrict__ ranges,
    const uint32_t* __restrict__ list_val, const ProjRecord* __restrict__ rec,
    const CompactRecord* __restrict__ rec16, const float4* __restrict__ pos_op, int64_t n, int E,
    TableT* __restrict__ table, float* __restrict__ state, uint64_t* __restrict__ sat,
    uint64_t* __restrict__ subsat, uint8_t* __restrict__ sat_chunk, int chunk,
    unsigned long long* __restrict__ counters) {
  __shared__ SubSmem S_warp[4];
  SubSmem& S = S_warp[threadIdx.x >> 5];
  const int v = blockIdx.y;
  const int tiles_x = views[v].tiles_x;
  const int bsub = 4 * blockIdx.x + (threadIdx.x >> 5);  // sub-tile of the view
  const int tile = bsub >> 2, sub = bsub & 3;
  if (tile >= tiles_x * views[v].tiles_y) return;  // whole warp
  const int gtile = views[v].tile_base + tile;
  const uint2 rg = ranges[gtile];
  if (rg.y <= rg.x) return;  // no list entry for this tile in this chunk
  const int gsub = 4 * gtile + sub;
  if ((subsat[gsub >> 6] >> (gsub & 63)) & 1ull) return;  // every pixel already stopped
  const int W = views[v].width, H = views[v].height;
  const int lane = threadIdx.x & 31;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int sx = sub & 1, sy = sub >> 1;
  const int lx = 2 * (lane & 3), ly = lane >> 2;
  const int px0 = tx * kTile + sx * 8 + lx, py = ty * kTile + sy * 8 + ly;

  // ---- the lane's two pixels: labels and transmittance --------------------
  const LabelT* mask = static_cast<const LabelT*>(views[v].mask);
  int lab0 = -1, lab1 = -1;
  const int64_t p0 = static_cast<int64_t>(py) * W + px0;
  if (py < H && px0 < W) lab0 = static_cast<int>(mask[p0]);
  if (py < H && px0 + 1 < W) lab1 = static_cast<int>(mask[p0 + 1]);
  const bool valid0 = lab0 >= 0 && lab0 < E, valid1 = lab1 >= 0 && lab1 < E;
  float* const st = state + views[v].state_off;
  float2 T = make_float2(valid0 ? st[p0] : 0.f, valid1 ? st[p0 + 1] : 0.f);
  const float2 T_start = T;
  float2 live = make_float2(0.f, 0.f);
  // the lane's main label, and whether its second pixel has another one
  const int main_lab = valid0 ? lab0 : (valid1 ? lab1 : -1);
  const bool minor = valid0 && valid1 && lab1 != lab0;
  const float w0 = valid0 ? 1.f : 0.f;
  const float w1 = (valid1 && !minor) ? 1.f : 0.f;
  // lane positions ordered by main label (labelless lanes last): lanes with a
  // smaller label, then lanes of the same label before this one -- one ballot
  // per distinct label of the warp (usually one or two)
  const int mkey = main_lab >= 0 ? main_lab : 0x7FFFFFFF;
  const uint32_t lt_lanes = lanemask_lt();
  int pos = 0;
  for (uint32_t rem = 0xffffffffu; rem;) {
    const int lead = __ffs(rem) - 1;
    const int k = __shfl_sync(0xffffffffu, mkey, lead);
    const uint32_t grp = __ballot_sync(0xffffffffu, mkey == k);
    rem &= ~grp;
    if (k < mkey) pos += __popc(grp);
    if (k == mkey) pos += __popc(grp & lt_lanes);
  }
  S.poslab[pos] = mkey;
  const uint32_t minor_lanes = __ballot_sync(0xffffffffu, minor);
  __syncwarp();
  const int plab = S.poslab[lane];
  const int plab_prev = __shfl_up_sync(0xffffffffu, plab, 1);
  const uint32_t segmask = __ballot_sync(0xffffffffu, lane == 0 || plab != plab_prev);

  // pixel centres relative to the sub-tile centre, in [-3.5, 3.5]
  const float2 X = make_float2(static_cast<float>(lx) - 3.5f, static_cast<float>(lx) - 2.5f);
  const float yy = static_cast<float>(ly) - 3.5f;
  const float ox = static_cast<float>(tx * kTile + sx * 8 + 4);
  const float oy = static_cast<float>(ty * kTile + sy * 8 + 4);
  const uint32_t gbase = static_cast<uint32_t>(static_cast<int64_t>(v) * n);
  const uint32_t lt = lanemask_lt();
  uint32_t n_staged = 0;

  // list entries one round ahead
  uint32_t g_next = rg.x + lane < rg.y ? list_val[rg.x + lane] : 0u;
  for (uint32_t base = rg.x; base < rg.y; base += kStage) {
    if (!__any_sync(0xffffffffu, T.x > 0.f || T.y > 0.f)) break;
    const int nin = static_cast<int>(min(static_cast<uint32_t>(kStage), rg.y - base));
    const uint32_t g_here = g_next;
    if (base + kStage + lane < rg.y) g_next = list_val[base + kStage + lane];
    // stage the Gaussians whose alpha >= 1/255 region can reach this sub-tile
    bool keep = false;
    float4 wk;
    float b0f = 0.f, b1f = 0.f, ok_ = 0.f;
    uint32_t g = 0;
    float qc = 0.f;
    if (lane < nin && rec16) {
      // reduced-precision record: b = W16 (o - m) in FP32
      g = g_here;
      const CompactRecord r = rec16[g];
      const float2 wa = __half22float2(*reinterpret_cast<const __half2*>(&r.w01));
      const float2 wb = __half22float2(*reinterpret_cast<const __half2*>(&r.w23));
      wk = make_float4(wa.x, wa.y, wb.x, wb.y);
      const float dx = ox - r.mx, dy = oy - r.my;
      b0f = fmaf(wk.x, dx, wk.y * dy);
      b1f = fmaf(wk.z, dx, wk.w * dy);
      ok_ = r.o;
      qc = r.q_cut;
    } else if (lane < nin) {
      // b = W (o - m) for the sub-tile centre o: o - m_hi is exact whenever
      // the mean lies within a factor of two of o (and off by far less than
      // a pixel's 1e-7 otherwise); W = W_hi + W_lo
      g = g_here;
      const ProjRecord r = rec[g];
      const float dx = (ox - r.m.x) - r.m.z, dy = (oy - r.m.y) - r.m.w;
      wk = r.w_hi;
      b0f = fmaf(wk.x, dx, fmaf(wk.y, dy, fmaf(r.w_lo.x, dx, r.w_lo.y * dy)));
      b1f = fmaf(wk.z, dx, fmaf(wk.w, dy, fmaf(r.w_lo.z, dx, r.w_lo.w * dy)));
      ok_ = r.misc.x;
      qc = r.misc.y;
    }
    if (lane < nin) {
      // over the sub-tile's pixel centres w ranges inside the box
      // b +- 3.5 (|W_k0| + |W_k1|); keep if that box meets |w|^2 <= q_cut
      const float h0 = 3.5f * (fabsf(wk.x) + fabsf(wk.y));
      const float h1 = 3.5f * (fabsf(wk.z) + fabsf(wk.w));
      const float d0 = fmaxf(0.f, fabsf(b0f) - h0), d1 = fmaxf(0.f, fabsf(b1f) - h1);
      keep = fmaf(d0, d0, d1 * d1) <= qc;
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      const int k = __popc(bal & lt);
      S.w[k] = wk;
      S.bo[k] = make_float4(b0f, b1f, ok_, 0.f);
      S.gid[k] = static_cast<int32_t>(g - gbase);
    }
    const int ns = __popc(bal);
    n_staged += static_cast<uint32_t>(ns);
    __syncwarp();
    if (minor_lanes) {
      // a lane whose second pixel has another label adds that pixel's
      // contribution itself (label boundaries only)
      for (int jj = 0; jj < ns; ++jj) {
        const float2 c = composite2(S.w[jj], S.bo[jj], X, yy, T, live);
        S.buf[jj][pos] = fmaf(c.x, w0, c.y * w1);
        if (minor && c.y != 0.f) table_add(&table[static_cast<int64_t>(S.gid[jj]) * E + lab1], c.y);
      }
    } else {
      for (int jj = 0; jj < ns; ++jj) {
        const float2 c = composite2(S.w[jj], S.bo[jj], X, yy, T, live);
        S.buf[jj][pos] = fmaf(c.x, w0, c.y * w1);
      }
    }
    __syncwarp();
    if (lane < ns) {
      // lane j owns staged Gaussian j: one atomic per label it reached here
      const int j = lane;
      const int64_t rowbase = static_cast<int64_t>(S.gid[j]) * E;
      uint32_t m = segmask;
      while (m) {
        const int s0 = __ffs(m) - 1;
        m &= m - 1;
        const int s1 = m ? __ffs(m) - 1 : 32;
        const int lab = S.poslab[s0];
        if (lab == 0x7FFFFFFF) continue;
        float sum = 0.f;
        for (int l = s0; l < s1; ++l) sum += S.buf[j][l];
        if (sum != 0.f) table_add(&table[rowbase + lab], sum);
      }
    }
    __syncwarp();
  }

  if (valid0) st[p0] = T.x;
  if (valid1) st[p0 + 1] = T.y;
  // steps evaluated up to termination: those that ran on, plus the stop
  uint32_t n_eval = static_cast<uint32_t>(live.x) + static_cast<uint32_t>(live.y) +
                    ((T_start.x > 0.f && T.x == 0.f) ? 1u : 0u) +
                    ((T_start.y > 0.f && T.y == 0.f) ? 1u : 0u);
  if (__all_sync(0xffffffffu, T.x == 0.f && T.y == 0.f) && lane == 0) {
    const unsigned long long bit = 1ull << (gsub & 63);
    const unsigned long long nib = 0xFull << (gsub & 63 & ~3);
    const unsigned long long old =
        atomicOr(reinterpret_cast<unsigned long long*>(subsat + (gsub >> 6)), bit);
    if (((old | bit) & nib) == nib) {
      set_bit(sat, gtile);
      // the tile's lists are complete up to this chunk only
      if (sat_chunk) sat_chunk[gtile] = static_cast<uint8_t>(chunk);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n_eval += __shfl_xor_sync(0xffffffffu, n_eval, o);
  if (lane == 0) {
    if (n_eval) atomicAdd(&counters[kPairs], static_cast<unsigned long long>(n_eval));
    if (n_staged) atomicAdd(&counters[kStaged], static_cast<unsigned long long>(n_staged));
  }
}

template <typename LabelT, typename TableT>
cudaError_t launch_typed(const ViewParams* views, int n_views, int max_tiles, const uint2* ranges,
                         const uint32_t* list_val, const ProjRecord* rec,
                         const CompactRecord* rec16, const float4* pos_op, int64_t n, int E,
                         void* table, float* state, uint64_t* sat, uint64_t* subsat,
                         uint8_t* sat_chunk, int chunk, unsigned long long* counters,
                         cudaStream_t stream) {
  dim3 grid(static_cast<unsigned>(max_tiles), static_cast<unsigned>(n_views));
  blend_kernel<LabelT, TableT><<<grid, 128, 0, stream>>>(views, ranges, list_val, rec, rec16,
                                                        pos_op, n, E,
                                                        static_cast<TableT*>(table), state, sat,
                                                        subsat, sat_chunk, chunk, counters);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_state_init(const ViewParams* views, int n_views, int max_tiles_per_view, int E,
                              int mask_dtype, float* state, uint64_t* sat, uint64_t* subsat,
                              unsigned long long* counters, cudaStream_t stream) {
  if (n_views == 0 || max_tiles_per_view == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(max_tiles_per_view), static_cast<unsigned>(n_views));
  if (mask_dtype == 4)
    state_init_kernel<uint8_t><<<grid, 256, 0, stream>>>(views, E, state, sat, subsat, counters);
  else
    state_init_kernel<int32_t><<<grid, 256, 0, stream>>>(views, E, state, sat, subsat, counters);
  return cudaGetLastError();
}

cudaError_t launch_blend(const ViewParams* views, int n_views, int max_tiles_per_view,
                         const uint2* ranges, const uint32_t* list_val, const ProjRecord* rec,
                         const CompactRecord* rec16, const float4* pos_op, int64_t n, int E,
                         int mask_dtype, void* table, int table_dtype, float* state,
                         uint64_t* sat, uint64_t* subsat, uint8_t* sat_chunk, int chunk,
                         unsigned long long* counters, cudaStream_t stream) {
  if (n_views == 0 || max_tiles_per_view == 0) return cudaSuccess;
  const int mt = max_tiles_per_view;
  if (mask_dtype == 4) {
    if (table_dtype == 0)
      return launch_typed<uint8_t, float>(views, n_views, mt, ranges, list_val, rec, rec16, pos_op,
                                          n, E, table, state, sat, subsat, sat_chunk, chunk,
                                          counters, stream);
    return launch_typed<uint8_t, double>(views, n_views, mt, ranges, list_val, rec, rec16, pos_op,
                                         n, E, table, state, sat, subsat, sat_chunk, chunk,
                                         counters, stream);
  }
  if (table_dtype == 0)
    return launch_typed<int32_t, float>(views, n_views, mt, ranges, list_val, rec, rec16, pos_op,
                                        n, E, table, state, sat, subsat, sat_chunk, chunk,
                                        counters, stream);
  return launch_typed<int32_t, double>(views, n_views, mt, ranges, list_val, rec, rec16, pos_op,
                                       n, E, table, state, sat, subsat, sat_chunk, chunk,
                                       counters, stream);
}

}  // namespace fs
