// Re-check of near-tie decisions at float-pair ("double-float") precision.
//
// The blend composites in FP32, so every table entry carries a relative error
// of about 1e-5 and the biased argmax (Sec. 3.2, Supp. Sec. 6 Listing 1) can
// come out differently from an exact evaluation for a Gaussian whose decision
// margin is that close to zero.  Such Gaussians (margin below a threshold)
// are re-evaluated here: every pixel of every view that one of them can reach
// is composited again front to back (Eq. 1: alpha, T, the 1/255 and 1e-4
// decisions) in float-pair arithmetic, about 1e-11 relative, up to its last
// re-checked Gaussian; their contributions alpha_i T_i go into an FP64 table
// of their own (Eq. 6/7) which then replaces their rows.  Float pairs keep
// the work on the FP32 pipe (GB300's FP64 rate is a small fraction of it).
//
// The per-tile depth-ordered lists come either from the main pass (its depth
// chunks, kept in memory) or from a dedicated binning of just the tiles the
// re-checked Gaussians reach.  A tile that saturated in the main pass has no
// list entries in later chunks; when a re-checked Gaussian sits in such a
// chunk ("deep" tile), every pixel of the tile is walked to its stop, and a
// pixel still compositing at the end of the kept lists (the FP32 and the
// exact stop decisions differ there) is reported so the caller redoes the
// batch with the dedicated binning.
//
// alpha = o 2^-|W (p - m)|^2 from the float-pair whitening record of the
// projection; 2^-q follows Tang's table-driven method (ACM TOMS 15(2), 1989):
// a 64-entry table of 2^(-j/64) (computed in FP64) times a degree-4 Taylor
// polynomial of e^-x on the remaining [0, ln2/64).
#include <cuda_fp16.h>
#include <math.h>

#include "fs_binning.cuh"
#include "fs_common.cuh"
#include "fs_internal.h"

namespace fs {

namespace {

__global__ void flag_margin_kernel(int64_t n, const float* __restrict__ margin, float tau,
                                   uint32_t* __restrict__ flag) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float m = margin[i];
  flag[i] = (m < tau) ? 1u : 0u;  // +inf (unseen) and NaN are never flagged
}

__global__ void scatter_flagged_kernel(int64_t n, const uint32_t* __restrict__ flag,
                                       const uint32_t* __restrict__ offs,
                                       uint32_t* __restrict__ F, int32_t* __restrict__ map) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (flag[i]) {
    F[offs[i]] = static_cast<uint32_t>(i);
    map[i] = static_cast<int32_t>(offs[i]);
  } else {
    map[i] = -1;
  }
}

// Position of slot a before-or-equal slot b in the batch's depth order:
// (depth key, view, low word of the depth, slot).
__device__ __forceinline__ bool order_le(uint32_t a, uint32_t b, int64_t n,
                                         const uint32_t* __restrict__ dkey,
                                         const uint32_t* __restrict__ dlo) {
  if (dkey[a] != dkey[b]) return dkey[a] < dkey[b];
  const uint32_t va = a / static_cast<uint32_t>(n), vb = b / static_cast<uint32_t>(n);
  if (va != vb) return va < vb;
  if (dlo[a] != dlo[b]) return dlo[a] < dlo[b];
  return a <= b;
}

// Clears, in the skip bit array, every tile that a re-checked Gaussian's
// footprint reaches in a view of the batch (the array starts all ones), and
// counts the visible (view, re-checked Gaussian) pairs in *visible.  With
// kept chunk lists (bound != NULL), a tile that saturated in an earlier chunk
// than the re-checked Gaussian's own gets its `deep` bit set.
__global__ void mark_tiles_kernel(int64_t n_flagged, int n_views, int64_t n,
                                  const uint32_t* __restrict__ F,
                                  const ViewParams* __restrict__ views,
                                  const uint32_t* __restrict__ cnt,
                                  const Footprint* __restrict__ foot,
                                  unsigned long long* __restrict__ skip,
                                  uint32_t* __restrict__ visible,
                                  const uint32_t* __restrict__ bound, int chunks,
                                  const uint32_t* __restrict__ dkey,
                                  const uint32_t* __restrict__ dlo,
                                  const uint8_t* __restrict__ sat_chunk,
                                  unsigned long long* __restrict__ deep) {
  const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= n_flagged * n_views) return;
  const int v = static_cast<int>(idx / n_flagged);
  const int64_t slot = static_cast<int64_t>(v) * n + F[idx % n_flagged];
  if (!cnt[slot]) return;
  atomicAdd(visible, 1u);
  int my_chunk = 0;
  if (bound) {
    my_chunk = chunks - 1;
    for (int ci = 0; ci < chunks - 1; ++ci)
      if (bound[ci] != 0xFFFFFFFFu &&  // an empty chunk holds nothing
          order_le(static_cast<uint32_t>(slot), bound[ci], n, dkey, dlo)) {
        my_chunk = ci;
        break;
      }
  }
  const Footprint f = foot[slot];
  const ViewParams& vp = views[v];
  int ty0, ty1;
  footprint_rows(f, &ty0, &ty1);
  for (int ty = ty0; ty <= ty1; ++ty) {
    int tx0, tx1;
    if (!row_span(f, ty, vp.width, &tx0, &tx1) || !clip_cols(vp, slot, &tx0, &tx1)) continue;
    const int a = vp.tile_base + ty * vp.tiles_x + tx0;
    const int b = vp.tile_base + ty * vp.tiles_x + tx1;
    for (int w = a >> 6; w <= (b >> 6); ++w) {
      unsigned long long m = ~0ull;
      if (w == (a >> 6)) m &= ~0ull << (a & 63);
      if (w == (b >> 6)) m &= ~0ull >> (63 - (b & 63));
      atomicAnd(&skip[w], ~m);
    }
    if (bound) {
      for (int t = a; t <= b; ++t)
        if (sat_chunk[t] < my_chunk) atomicOr(&deep[t >> 6], 1ull << (t & 63));
    }
  }
}

// flag[slot] = 1 iff the slot's footprint reaches a tile left unskipped.
__global__ void candidates_kernel(int64_t k_total, int64_t n, const ViewParams* __restrict__ views,
                                  const uint32_t* __restrict__ cnt,
                                  const Footprint* __restrict__ foot,
                                  const uint64_t* __restrict__ skip, uint32_t* __restrict__ flag) {
  const int64_t slot = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (slot >= k_total) return;
  uint32_t hit = 0;
  if (cnt[slot]) {
    const int v = static_cast<int>(slot / n);
    const ViewParams& vp = views[v];
    const Footprint f = foot[slot];
    int ty0, ty1;
    footprint_rows(f, &ty0, &ty1);
    for (int ty = ty0; ty <= ty1 && !hit; ++ty) {
      int tx0, tx1;
      if (!row_span(f, ty, vp.width, &tx0, &tx1) || !clip_cols(vp, slot, &tx0, &tx1)) continue;
      const int base = vp.tile_base + ty * vp.tiles_x;
      if (count_free(skip, base + tx0, base + tx1)) hit = 1;
    }
  }
  flag[slot] = hit;
}

__global__ void compact_kernel(int64_t k_total, const uint32_t* __restrict__ flag,
                               const uint32_t* __restrict__ offs,
                               const uint32_t* __restrict__ key_src,
                               uint32_t* __restrict__ out_key, uint32_t* __restrict__ out_val) {
  const int64_t slot = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (slot >= k_total || !flag[slot]) return;
  const uint32_t o = offs[slot];
  out_key[o] = key_src[slot];
  out_val[o] = static_cast<uint32_t>(slot);
}

constexpr int kRB = 64;  // list entries staged per round
constexpr int kDeepTest = 256;  // re-checked Gaussians a deep tile tests per pixel at most

// Float-pair constants of the compositing rule (Sec. 3.1 Eq. 1 conventions).
constexpr double kAlphaMinD = 1.0 / 255.0, kAlphaMaxD = 0.99, kTMinD = 1e-4;
constexpr double kLn2D = 0.69314718055994530942;
#define FS_F2C(d) f2{static_cast<float>(d), static_cast<float>((d) - static_cast<double>(static_cast<float>(d)))}

// 2^-q for q >= 0 as a float pair (about 1e-11 relative): q = k + j/64 + s,
// 2^-q = 2^-k * 2^(-j/64) * e^(-s ln 2) with a degree-4 Taylor polynomial of
// e^-x for x = s ln 2 in [0, ln2/64) (truncation below 1.3e-12).
__device__ __forceinline__ f2 f2_exp2_neg(f2 q, const float2* __restrict__ tab) {
  const float k = floorf(q.hi);
  const float r = q.hi - k;                        // exact
  const float jf = floorf(r * 64.f);
  const float s = r - jf * (1.f / 64.f);           // exact (Sterbenz)
  const f2 t = two_sum(s, q.lo);
  const f2 x = f2_mul(t, FS_F2C(kLn2D));
  const float xh = x.hi;
  const float p = xh * xh * fmaf(xh, fmaf(xh, 1.f / 24.f, -1.f / 6.f), 0.5f);
  f2 e = f2_add(f2_from(1.f), f2_neg(x));
  e = f2_add(e, f2_from(p));
  const float2 tj = tab[static_cast<int>(jf)];
  e = f2_mul(e, f2{tj.x, tj.y});
  const float sc = __int_as_float((127 - static_cast<int>(k)) << 23);  // 2^-k, k <= 126
  return {e.hi * sc, e.lo * sc};
}

// Staged list entry: W (float pairs), b = W (ctr - m) relative to the tile
// centre (float pairs), opacity, q_cut + slack, re-check row (-1: none).
struct Staged {
  f2 w[4];
  f2 b[2];
  float o, qc;
  int j;
};

__device__ __forceinline__ Staged stage_entry(const ProjRecord& r, float cx, float cy, int j) {
  Staged st;
  st.w[0] = {r.w_hi.x, r.w_lo.x};
  st.w[1] = {r.w_hi.y, r.w_lo.y};
  st.w[2] = {r.w_hi.z, r.w_lo.z};
  st.w[3] = {r.w_hi.w, r.w_lo.w};
  // b = W (ctr - m) with the difference of the centre and the float-pair mean
  const f2 dx = f2_sub(f2_from(cx), f2{r.m.x, r.m.z});
  const f2 dy = f2_sub(f2_from(cy), f2{r.m.y, r.m.w});
  st.b[0] = f2_add(f2_mul(st.w[0], dx), f2_mul(st.w[1], dy));
  st.b[1] = f2_add(f2_mul(st.w[2], dx), f2_mul(st.w[3], dy));
  st.o = r.misc.x;
  // near the cut the FP32 screen |W_hi l + b_hi|^2 is off by far less than 0.05
  st.qc = r.misc.y + 0.05f;
  st.j = j;
  return st;
}

// Reduced-precision record: W16 and the FP32 mean are exact float values, so
// b = W (ctr - m) is formed from the exact difference in float pairs.
__device__ __forceinline__ Staged stage_compact(const CompactRecord& r, float o, float cx,
                                                float cy, int j) {
  Staged st;
  const float2 wa = __half22float2(*reinterpret_cast<const __half2*>(&r.w01));
  const float2 wb = __half22float2(*reinterpret_cast<const __half2*>(&r.w23));
  st.w[0] = f2_from(wa.x);
  st.w[1] = f2_from(wa.y);
  st.w[2] = f2_from(wb.x);
  st.w[3] = f2_from(wb.y);
  const f2 dx = two_sum(cx, -r.mx), dy = two_sum(cy, -r.my);
  st.b[0] = f2_add(f2_mul(st.w[0], dx), f2_mul(st.w[1], dy));
  st.b[1] = f2_add(f2_mul(st.w[2], dx), f2_mul(st.w[3], dy));
  st.o = o;
  st.qc = fmaxf(log2f(255.f * o), 0.f) * 1.001f + 1e-3f + 0.05f;
  st.j = j;
  return st;
}

// FP32 screen: can the entry's alpha >= 1/255 region reach this pixel?
__device__ __forceinline__ bool reaches(const Staged& e, float lx, float ly) {
  const float q0 = fmaf(e.w[0].hi, lx, fmaf(e.w[1].hi, ly, e.b[0].hi));
  const float q1 = fmaf(e.w[2].hi, lx, fmaf(e.w[3].hi, ly, e.b[1].hi));
  return fmaf(q0, q0, q1 * q1) <= e.qc;
}

// One CTA per 16x16 tile of a view, one thread per pixel.  Pass 1 finds, per
// pixel, the last list position holding a re-checked Gaussian that can reach
// the pixel; pass 2 composites the pixel in float pairs up to that position
// (deep tiles: up to its stop).
template <typename LabelT>
__global__ void __launch_bounds__(kTilePixels, 6) recheck_blend_kernel(
    const ViewParams* __restrict__ views, RecheckLists L, const uint64_t* __restrict__ skip,
    const ProjRecord* __restrict__ rec, const CompactRecord* __restrict__ rec16,
    const float4* __restrict__ pos_op, int64_t n, int E, const int32_t* __restrict__ map,
    double* __restrict__ R, unsigned long long* __restrict__ counters) {
  __shared__ Staged s_e[kRB];
  __shared__ float2 s_tab[64];
  const ViewParams& vp = views[blockIdx.y];
  const int tile = blockIdx.x;
  if (tile >= vp.tiles_x * vp.tiles_y) return;
  const int gtile = vp.tile_base + tile;
  if ((skip[gtile >> 6] >> (gtile & 63)) & 1ull) return;
  const int n_chunks = L.sat_chunk ? min(L.chunks, static_cast<int>(L.sat_chunk[gtile]) + 1)
                                   : L.chunks;
  const bool truncated = n_chunks < L.chunks;
  const bool deep = L.deep && ((L.deep[gtile >> 6] >> (gtile & 63)) & 1ull);
  if (threadIdx.x < 64) {
    const double d = exp2(-static_cast<double>(threadIdx.x) / 64.0);
    const float hi = static_cast<float>(d);
    s_tab[threadIdx.x] = make_float2(hi, static_cast<float>(d - static_cast<double>(hi)));
  }
  const int x0 = (tile % vp.tiles_x) * kTile, y0 = (tile / vp.tiles_x) * kTile;
  const int x = x0 + (threadIdx.x & (kTile - 1));
  const int y = y0 + (threadIdx.x / kTile);
  int label = -1;
  if (x < vp.width && y < vp.height) {
    const int l = static_cast<int>(
        static_cast<const LabelT*>(vp.mask)[static_cast<int64_t>(y) * vp.width + x]);
    if (l >= 0 && l < E) label = l;
  }
  const float cx = static_cast<float>(x0) + 0.5f * kTile;
  const float cy = static_cast<float>(y0) + 0.5f * kTile;
  // pixel centre (x + 0.5, y + 0.5) relative to the tile centre: exact
  const float lx = static_cast<float>(x - x0) + 0.5f - 0.5f * kTile;
  const float ly = static_cast<float>(y - y0) + 0.5f - 0.5f * kTile;

  // pass 1: last re-checked entry (chunk << 32 | index) that may reach the pixel
  int64_t last = -1;
  for (int c = 0; c < n_chunks; ++c) {
    const uint2 rg = L.ranges[c][gtile];
    for (uint32_t b0 = rg.x; b0 < rg.y; b0 += kRB) {
      const int cnt = static_cast<int>(min(static_cast<uint32_t>(kRB), rg.y - b0));
      __syncthreads();
      if (threadIdx.x < cnt) {
        const uint32_t slot = L.val[c][b0 + threadIdx.x];
        const uint32_t gi = static_cast<uint32_t>(slot % static_cast<uint64_t>(n));
        const int j = map[gi];
        s_e[threadIdx.x].j = j;
        if (j >= 0)
          s_e[threadIdx.x] = rec16 ? stage_compact(rec16[slot], pos_op[gi].w, cx, cy, j)
                                   : stage_entry(rec[slot], cx, cy, j);
      }
      __syncthreads();
      if (label >= 0)
        for (int e = 0; e < cnt; ++e)
          if (s_e[e].j >= 0 && reaches(s_e[e], lx, ly))
            last = (static_cast<int64_t>(c) << 32) | (b0 + e);
    }
  }

  // deep tiles: a pixel is walked to its stop only where a re-checked
  // Gaussian visible in this view can reach it (the others hold nothing to
  // re-check); with many re-checked Gaussians every labelled pixel is
  bool deep_px = deep;
  if (deep && L.flagged && L.n_flagged <= kDeepTest) {
    bool reached = false;
    for (int k0 = 0; k0 < L.n_flagged; k0 += kRB) {
      const int cnt = min(kRB, L.n_flagged - k0);
      __syncthreads();
      if (threadIdx.x < cnt) {
        const uint32_t gi = L.flagged[k0 + threadIdx.x];
        const int64_t slot = static_cast<int64_t>(blockIdx.y) * n + gi;
        s_e[threadIdx.x].j = -1;
        if (L.cnt[slot])
          s_e[threadIdx.x] = rec16 ? stage_compact(rec16[slot], pos_op[gi].w, cx, cy, 0)
                                   : stage_entry(rec[slot], cx, cy, 0);
      }
      __syncthreads();
      for (int e = 0; e < cnt; ++e)
        if (s_e[e].j >= 0 && reaches(s_e[e], lx, ly)) reached = true;
    }
    deep_px = reached;
  }

  // pass 2: float-pair compositing
  const f2 a_min = FS_F2C(kAlphaMinD), a_max = FS_F2C(kAlphaMaxD), t_min = FS_F2C(kTMinD);
  f2 T = f2_from(1.f);
  bool live = label >= 0 && (deep_px || last >= 0);
  const bool to_stop = deep_px;
  unsigned long long evals = 0;
  bool done_all = false;
  for (int c = 0; c < n_chunks && !done_all; ++c) {
    const uint2 rg = L.ranges[c][gtile];
    for (uint32_t b0 = rg.x; b0 < rg.y; b0 += kRB) {
      if (__syncthreads_count(live) == 0) {
        done_all = true;
        break;
      }
      const int cnt = static_cast<int>(min(static_cast<uint32_t>(kRB), rg.y - b0));
      if (threadIdx.x < cnt) {
        const uint32_t slot = L.val[c][b0 + threadIdx.x];
        const uint32_t gi = static_cast<uint32_t>(slot % static_cast<uint64_t>(n));
        s_e[threadIdx.x] = rec16 ? stage_compact(rec16[slot], pos_op[gi].w, cx, cy, map[gi])
                                 : stage_entry(rec[slot], cx, cy, map[gi]);
      }
      __syncthreads();
      if (live) {
        const int64_t pos0 = (static_cast<int64_t>(c) << 32) | b0;
        int e_end = cnt;
        if (!to_stop) e_end = static_cast<int>(min(static_cast<int64_t>(cnt), last - pos0 + 1));
        for (int e = 0; e < e_end; ++e) {
          const Staged& en = s_e[e];
          if (!reaches(en, lx, ly)) continue;  // alpha < 1/255 in any precision
          ++evals;
          const f2 w0 = f2_add(f2_add(f2_mul_f(en.w[0], lx), f2_mul_f(en.w[1], ly)), en.b[0]);
          const f2 w1 = f2_add(f2_add(f2_mul_f(en.w[2], lx), f2_mul_f(en.w[3], ly)), en.b[1]);
          const f2 q = f2_add(f2_mul(w0, w0), f2_mul(w1, w1));
          f2 a = f2_mul_f(f2_exp2_neg(q, s_tab), en.o);
          if (f2_lt(a_max, a)) a = a_max;
          if (f2_lt(a, a_min)) continue;
          const f2 t = f2_mul(T, f2_sub(f2_from(1.f), a));
          if (f2_lt(t, t_min)) {
            live = false;
            break;
          }
          if (en.j >= 0) {
            const f2 ct = f2_mul(a, T);
            atomicAdd(&R[static_cast<int64_t>(en.j) * E + label],
                      static_cast<double>(ct.hi) + static_cast<double>(ct.lo));
          }
          T = t;
        }
        if (live && !to_stop && pos0 + cnt > last) live = false;
      }
    }
  }
  // still compositing where a saturated tile's kept lists end: the exact
  // walk needs entries the main pass never listed
  const bool incomplete = live && truncated && to_stop;
  const int n_inc = __syncthreads_count(incomplete);
  if (threadIdx.x == 0 && n_inc) atomicAdd(&counters[kRecheckIncomplete], 1ull);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(0xffffffffu, evals, o);
  if ((threadIdx.x & 31) == 0 && evals) atomicAdd(&counters[kRecheckPairs], evals);
}

__global__ void add_rows_kernel(int64_t count, const double* __restrict__ src,
                                double* __restrict__ dst) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < count) dst[i] += src[i];
}

inline unsigned blocks_for(int64_t n, int threads) {
  return static_cast<unsigned>((n + threads - 1) / threads);
}

}  // namespace

cudaError_t launch_flag_margin(int64_t n, const float* margin, float tau, uint32_t* flag,
                               cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  flag_margin_kernel<<<blocks_for(n, 256), 256, 0, stream>>>(n, margin, tau, flag);
  return cudaGetLastError();
}

cudaError_t launch_scatter_flagged(int64_t n, const uint32_t* flag, const uint32_t* offs,
                                   uint32_t* F, int32_t* map, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  scatter_flagged_kernel<<<blocks_for(n, 256), 256, 0, stream>>>(n, flag, offs, F, map);
  return cudaGetLastError();
}

cudaError_t launch_mark_tiles(int64_t n_flagged, int n_views, int64_t n, const uint32_t* F,
                              const ViewParams* views, const uint32_t* cnt, const Footprint* foot,
                              uint64_t* skip, uint32_t* visible, const uint32_t* bound,
                              int chunks, const uint32_t* dkey, const uint32_t* dlo,
                              const uint8_t* sat_chunk, uint64_t* deep, cudaStream_t stream) {
  const int64_t total = n_flagged * n_views;
  if (total == 0) return cudaSuccess;
  mark_tiles_kernel<<<blocks_for(total, 256), 256, 0, stream>>>(
      n_flagged, n_views, n, F, views, cnt, foot, reinterpret_cast<unsigned long long*>(skip),
      visible, bound, chunks, dkey, dlo, sat_chunk, reinterpret_cast<unsigned long long*>(deep));
  return cudaGetLastError();
}

cudaError_t launch_add_rows(int64_t count, const double* src, double* dst, cudaStream_t stream) {
  if (count == 0) return cudaSuccess;
  add_rows_kernel<<<blocks_for(count, 256), 256, 0, stream>>>(count, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_candidates(int64_t k_total, int64_t n, const ViewParams* views,
                              const uint32_t* cnt, const Footprint* foot, const uint64_t* skip,
                              uint32_t* flag, cudaStream_t stream) {
  if (k_total == 0) return cudaSuccess;
  candidates_kernel<<<blocks_for(k_total, 256), 256, 0, stream>>>(k_total, n, views, cnt, foot,
                                                                  skip, flag);
  return cudaGetLastError();
}

cudaError_t launch_compact(int64_t k_total, const uint32_t* flag, const uint32_t* offs,
                           const uint32_t* key_src, uint32_t* out_key, uint32_t* out_val,
                           cudaStream_t stream) {
  if (k_total == 0) return cudaSuccess;
  compact_kernel<<<blocks_for(k_total, 256), 256, 0, stream>>>(k_total, flag, offs, key_src,
                                                               out_key, out_val);
  return cudaGetLastError();
}

cudaError_t launch_recheck_blend(const ViewParams* views, int n_views, int max_tiles_per_view,
                                 const RecheckLists& lists, const uint64_t* skip,
                                 const ProjRecord* rec, const CompactRecord* rec16,
                                 const float4* pos_op, int64_t n, int E, int mask_dtype,
                                 const int32_t* map, double* R, unsigned long long* counters,
                                 cudaStream_t stream) {
  if (n_views == 0 || max_tiles_per_view == 0) return cudaSuccess;
  if (lists.chunks < 1 || lists.chunks > kMaxChunks) return cudaErrorInvalidValue;
  const dim3 grid(static_cast<unsigned>(max_tiles_per_view), static_cast<unsigned>(n_views));
  if (mask_dtype == 4)
    recheck_blend_kernel<uint8_t><<<grid, kTilePixels, 0, stream>>>(
        views, lists, skip, rec, rec16, pos_op, n, E, map, R, counters);
  else
    recheck_blend_kernel<int32_t><<<grid, kTilePixels, 0, stream>>>(
        views, lists, skip, rec, rec16, pos_op, n, E, map, R, counters);
  return cudaGetLastError();
}

}  // namespace fs
