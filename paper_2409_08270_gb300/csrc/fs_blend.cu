// Front-to-back alpha blending of every mask pixel and accumulation of
// alpha_i T_i into the contribution table (Sec. 3.1 Eq. 1, Sec. 3.2 Eq. 6,
// Sec. 3.3 Eq. 7, Sec. 4.2: each Gaussian's alpha_i T_i at a pixel goes into
// the table column of that pixel's label, added atomically).
//
// One 128-thread block per 16x16 tile; warp w composites the 8x8 sub-tile w,
// two adjacent pixels per lane.
//  * Staging (the whole block, 64 list entries of the tile's depth-sorted
//    list per step): each entry's projected record is read once; two
//    threads per entry test it against two sub-tiles each -- can its
//    alpha >= 1/255 region reach the sub-tile's pixel centres? -- and append
//    the Gaussian's whitening matrix W, its offset b = W (o - m) at the
//    sub-tile centre o and -log2(opacity) to the sub-tile's queue in shared
//    memory, in list order.  Queues hold Gaussians in pairs (g, h) side by
//    side, so the packed FP32 instructions (FFMA2, FMUL2, FADD2) evaluate
//    two Gaussians at once without rearranging registers.
//  * Compositing (each warp, rounds of 32 queued Gaussians), per lane, per
//    Gaussian pair, for its pixels P and Q = P + (1, 0):
//      q = |W p + b|^2 - log2 o,  alpha = 2^-q = o exp(-0.5 d^T Sigma^-1 d)
//    alpha >= 1/255 is decided by flushing alpha * 255 * 2^-126 to zero when
//    it falls below the smallest normal float (FTZ multiply); the clamp at
//    0.99 is applied only for pairs holding a Gaussian of opacity above
//    0.99.  T is carried as T * 2^126 / 255, so the flushed product times it
//    is alpha * T.  The stop before a Gaussian that would take T below 1e-4
//    is an exact 0/1 factor from a saturated FMA.  A stopped pixel carries
//    T = 0.
//  * Per Gaussian the lane writes its pixels' sum into a shared row ordered
//    by label (a lane whose two pixels carry different labels writes its
//    second pixel to a small second row); lane j then sums Gaussian j's rows
//    per label and issues one FP64 atomic add per non-zero (Gaussian, label).
#include <cuda_fp16.h>

#include "fs_common.cuh"
#include "fs_internal.h"

namespace fs {

namespace {

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename TableT>
__device__ __forceinline__ void table_add(TableT* p, float v) {
  atomicAdd(p, static_cast<TableT>(v));
}

// alpha * 255 * 2^-126 is subnormal exactly when alpha < 1/255 (FTZ flushes it)
constexpr float kSkipScale = 255.0f * 0x1p-126f;
// T is carried as T / kSkipScale, so (alpha kSkipScale) (T / kSkipScale) = alpha T
constexpr float kTScale = 0x1p126f / 255.0f;
// the scaled stop threshold 1e-4 / kSkipScale lies in [2^104, 2^105): ulp 2^81
constexpr float kStepScale = 0x1p-81f;

__device__ __forceinline__ void set_bit(uint64_t* bits, int i) {
  atomicOr(reinterpret_cast<unsigned long long*>(bits + (i >> 6)), 1ull << (i & 63));
}

// Per-pixel state of a batch before its first depth chunk: the scaled
// transmittance T * kTScale (the form the blend carries, so the state passes
// between depth chunks without rounding), with T = 1 for pixels with a label
// in [0, E) and 0 ("stopped") for the others.  Sub-tiles (and tiles)
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
    state[views[v].state_off + p] = valid ? kTScale : 0.f;
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
constexpr int kRound = 32;     // Gaussians composited per round (one per lane)
constexpr int kStep = 64;      // list entries staged per block step
constexpr int kStagers = kStep / 32;  // warps that stage them, one entry per thread
constexpr int kQCap = 96;      // per-warp queue: a partial round plus one step
constexpr int kMinorCap = 2;   // label-boundary lanes a warp sums in shared memory (more
                               // add their second pixel to the table directly; the cap keeps
                               // seven blocks' shared memory within an SM's)

// Per-warp shared memory.  The queue is a ring of kQCap Gaussians, two per
// float4 (g = first half of each component pair, h = second).
struct WarpSmem {
  float4 wx[kQCap / 2];              // (W00 g, W00 h, W10 g, W10 h): x coefficients of w = W p + b
  float4 wy[kQCap / 2];              // (W01 g, W01 h, W11 g, W11 h): y coefficients
  float4 bb[kQCap / 2];              // (b0 g, b0 h, b1 g, b1 h)
  float4 oo[kQCap / 2];              // (-log2 o_g, -log2 o_h, clamp g, clamp h)
  int32_t gid[kQCap];                // scene index of each queued Gaussian
  float buf[kRound][32];             // [Gaussian][lane position by main label], XOR-swizzled
  float buf2[kRound][kMinorCap];     // [Gaussian][boundary lane by its second label]
  int32_t poslab[32];                // label of each lane position (INT_MAX: none)
  int32_t minlab[kMinorCap];         // second label of each boundary-lane position
};

struct BlockSmem {
  WarpSmem w[4];
  uint32_t cnt[4][4];                // [warp][sub-tile]: entries kept in this step
  uint32_t tail[4];                  // queue tails (Gaussians ever queued)
  int32_t alive[4];                  // the sub-tile still has a compositing pixel
};

// Column of position p in row j of the partial-sum buffer: float4 groups are
// XOR-swizzled by the row so that row reads (one row per lane) and column
// writes (one column per lane) are both free of bank conflicts.
__device__ __forceinline__ int swz(int j, int p) { return p ^ ((j & 7) << 2); }

__device__ __forceinline__ float2 fmul2_ftz(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.ftz.f32x2 %0, %1, %2;"
      : "=l"(d)
      : "l"(*reinterpret_cast<unsigned long long*>(&a)),
        "l"(*reinterpret_cast<unsigned long long*>(&b)));
  return *reinterpret_cast<float2*>(&d);
}

// 1.0f if t >= thr (t - thr_below a positive multiple of ulp(thr)), else 0.0f:
// saturate((t - thr_below) / ulp(thr)), exact for the scaled transmittance.
__device__ __forceinline__ float step_sat(float t, float neg_thr_scaled) {
  float d;
  asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(t), "f"(kStepScale), "f"(neg_thr_scaled));
  return d;
}

// How a warp's pixels are labelled, which decides how a round's per-Gaussian
// sums are formed:
//   kOneLabel:  every labelled pixel carries one label; a lane writes the sum
//               of its two pixels (rounds of 32 Gaussians);
//   kTwoLabels: two labels La < Lb; a lane writes the sum of its pixels of La
//               to rows 0-15 and of Lb to rows 16-31 (rounds of 16 Gaussians);
//   kMany:      more labels; lane positions sorted by the first pixel's label,
//               second pixels of another label to a small second row (rounds
//               of 32 Gaussians).
enum LabelMode { kOneLabel = 0, kTwoLabels = 1, kMany = 2 };

// One round: the lane's two pixels P and Q = P + (1, 0) against queued
// Gaussian pairs pair0 .. pair0 + npairs - 1 (ring indices), in depth order.
// kTwoLabels: wA / wB weight P and Q for La / Lb.  kMany: a lane whose Q is
// labelled differently from P writes Q's term to the second row (slot
// mpos < kMinorCap) or, past its capacity, straight to the table.
template <int kMode, bool kCensus, typename TableT>
__device__ __forceinline__ void composite_round(
    WarpSmem& S, int pair0, int npairs, float2 X2, float2 Y2, float neg_thr, float wq,
    float2 wA, float2 wB, int pos, int mpos, bool minor, int lab1, int E,
    TableT* __restrict__ table, float2& Tu, unsigned long long& n_eval,
    unsigned long long& n_part) {
  const float2 nK = make_float2(-kTScale, -kTScale);
  const float2 skip = make_float2(kSkipScale, kSkipScale);
  const bool spill = minor && mpos >= kMinorCap;
  for (int k = 0; k < npairs; ++k) {
    int pr = pair0 + k;
    if (pr >= kQCap / 2) pr -= kQCap / 2;
    const float4 rx = S.wx[pr], ry = S.wy[pr], rb = S.bb[pr], ro = S.oo[pr];
    const float2 wx0 = make_float2(rx.x, rx.y), wx1 = make_float2(rx.z, rx.w);
    const float2 wy0 = make_float2(ry.x, ry.y), wy1 = make_float2(ry.z, ry.w);
    const float2 b0 = make_float2(rb.x, rb.y), b1 = make_float2(rb.z, rb.w);
    const float2 nlo = make_float2(ro.x, ro.y);
    // w at P for (g, h), then q = |w|^2 - log2 o at P and at Q = P + (1, 0)
    float2 u0 = __ffma2_rn(wx0, X2, __ffma2_rn(wy0, Y2, b0));
    float2 u1 = __ffma2_rn(wx1, X2, __ffma2_rn(wy1, Y2, b1));
    const float2 qP = __ffma2_rn(u0, u0, __ffma2_rn(u1, u1, nlo));
    u0 = __fadd2_rn(u0, wx0);
    u1 = __fadd2_rn(u1, wx1);
    const float2 qQ = __ffma2_rn(u0, u0, __ffma2_rn(u1, u1, nlo));
    float2 ag = make_float2(ex2_approx(-qP.x), ex2_approx(-qQ.x));  // Gaussian g at (P, Q)
    float2 ah = make_float2(ex2_approx(-qP.y), ex2_approx(-qQ.y));  // Gaussian h at (P, Q)
    if (ro.z != 0.f || ro.w != 0.f) {
      ag.x = fminf(ag.x, kAlphaMax);
      ag.y = fminf(ag.y, kAlphaMax);
      ah.x = fminf(ah.x, kAlphaMax);
      ah.y = fminf(ah.y, kAlphaMax);
    }
    ag = fmul2_ftz(ag, skip);  // 0 where alpha < 1/255
    ah = fmul2_ftz(ah, skip);
    if (kCensus) {
      n_eval += (Tu.x != 0.f) + (Tu.y != 0.f);
      n_part += (Tu.x != 0.f && ag.x != 0.f) + (Tu.y != 0.f && ag.y != 0.f);
    }
    float2 cg = __fmul2_rn(ag, Tu);              // alpha_g T
    const float2 T1 = __ffma2_rn(cg, nK, Tu);    // T (1 - alpha_g), scaled
    if (kCensus) {
      n_eval += (T1.x != 0.f) + (T1.y != 0.f);
      n_part += (T1.x != 0.f && ah.x != 0.f) + (T1.y != 0.f && ah.y != 0.f);
    }
    float2 ch = __fmul2_rn(ah, T1);
    const float2 T2 = __ffma2_rn(ch, nK, T1);
    // the pixel stops before a Gaussian that takes T below 1e-4; once T2
    // passes the threshold so did T1 (alpha >= 0)
    const float2 gg = make_float2(step_sat(T1.x, neg_thr), step_sat(T1.y, neg_thr));
    const float2 gh = make_float2(step_sat(T2.x, neg_thr), step_sat(T2.y, neg_thr));
    cg = __fmul2_rn(cg, gg);
    ch = __fmul2_rn(ch, gh);
    Tu = __fmul2_rn(T2, gh);
    if (kCensus) {
      // a pixel that stops at g does not evaluate h: undo its count
      n_eval -= (T1.x != 0.f && gg.x == 0.f) + (T1.y != 0.f && gg.y == 0.f);
      n_part -= (T1.x != 0.f && gg.x == 0.f && ah.x != 0.f) +
                (T1.y != 0.f && gg.y == 0.f && ah.y != 0.f);
    }
    if (kMode == kTwoLabels) {
      // rows 2k, 2k + 1 for La; 16 + 2k, 17 + 2k for Lb; columns by lane
      S.buf[2 * k][swz(2 * k, pos)] = fmaf(cg.y, wA.y, cg.x * wA.x);
      S.buf[2 * k + 1][swz(2 * k + 1, pos)] = fmaf(ch.y, wA.y, ch.x * wA.x);
      S.buf[16 + 2 * k][swz(16 + 2 * k, pos)] = fmaf(cg.y, wB.y, cg.x * wB.x);
      S.buf[17 + 2 * k][swz(17 + 2 * k, pos)] = fmaf(ch.y, wB.y, ch.x * wB.x);
    } else {
      S.buf[2 * k][swz(2 * k, pos)] = fmaf(cg.y, wq, cg.x);
      S.buf[2 * k + 1][swz(2 * k + 1, pos)] = fmaf(ch.y, wq, ch.x);
    }
    if (kMode == kMany) {
      if (minor && !spill) {
        S.buf2[2 * k][mpos] = cg.y;
        S.buf2[2 * k + 1][mpos] = ch.y;
      }
      int q0 = 2 * pr;
      if (spill && cg.y != 0.f)
        table_add(&table[static_cast<int64_t>(S.gid[q0]) * E + lab1], cg.y);
      if (spill && ch.y != 0.f)
        table_add(&table[static_cast<int64_t>(S.gid[q0 + 1]) * E + lab1], ch.y);
    }
  }
}

// Row j of the buffer holds one label's terms of one Gaussian (scene index
// gi) over the 32 lanes: their sum into the table.
template <typename TableT>
__device__ __forceinline__ void reduce_plane(const WarpSmem& S, int j, int64_t gi, int E, int lab,
                                             TableT* __restrict__ table) {
  const float4* row = reinterpret_cast<const float4*>(S.buf[j]);
  const int sw = j & 7;
  float sum = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 x = row[q ^ sw];
    sum += (x.x + x.y) + (x.z + x.w);
  }
  if (sum != 0.f) table_add(&table[gi * E + lab], sum);
}

// Lane j < nq: Gaussian j of the round (scene index gi) -- its sums per label
// into the table.
template <typename TableT>
__device__ __forceinline__ void reduce_row(const WarpSmem& S, int j, int64_t gi, int E,
                                           bool one_label, int lab_first, uint32_t segmask,
                                           int n_minor, TableT* __restrict__ table) {
  const int64_t rowbase = gi * E;
  // the boundary lanes' second pixels: folded into the main sum of the same
  // label when they all share one label (the usual case)
  float extra = 0.f;
  int extra_lab = -1;
  if (n_minor > 0) {
    const int l0 = S.minlab[0];
    bool one = true;
    for (int r = 1; r < n_minor; ++r) one = one && S.minlab[r] == l0;
    if (one) {
      for (int r = 0; r < n_minor; ++r) extra += S.buf2[j][r];
      extra_lab = l0;
    } else {
      float acc = 0.f;
      int lab = l0;
      for (int r = 0; r < n_minor; ++r) {
        if (S.minlab[r] != lab) {
          if (acc != 0.f) table_add(&table[rowbase + lab], acc);
          acc = 0.f;
          lab = S.minlab[r];
        }
        acc += S.buf2[j][r];
      }
      if (acc != 0.f) table_add(&table[rowbase + lab], acc);
    }
  }
  const float4* row = reinterpret_cast<const float4*>(S.buf[j]);
  const int sw = j & 7;
  if (one_label) {
    float sum = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 x = row[q ^ sw];
      sum += (x.x + x.y) + (x.z + x.w);
    }
    if (lab_first == extra_lab) {
      sum += extra;
      extra = 0.f;
    }
    if (sum != 0.f && lab_first != 0x7FFFFFFF) table_add(&table[rowbase + lab_first], sum);
  } else {
    // segments of equal label over the positions (segmask: their starts)
    float acc = 0.f;
    int lab = lab_first;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 x = row[q ^ sw];
      const uint32_t starts = (segmask >> (4 * q)) & (q == 0 ? 0xEu : 0xFu);
      if (starts == 0u) {
        acc += (x.x + x.y) + (x.z + x.w);
      } else {
        const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if ((starts >> i) & 1u) {
            if (lab == extra_lab) {
              acc += extra;
              extra = 0.f;
            }
            if (acc != 0.f && lab != 0x7FFFFFFF) table_add(&table[rowbase + lab], acc);
            acc = 0.f;
            lab = S.poslab[4 * q + i];
          }
          acc += xs[i];
        }
      }
    }
    if (lab == extra_lab) {
      acc += extra;
      extra = 0.f;
    }
    if (acc != 0.f && lab != 0x7FFFFFFF) table_add(&table[rowbase + lab], acc);
  }
  if (extra != 0.f) table_add(&table[rowbase + extra_lab], extra);
}

// Rank of each lane among the lanes with the same or a smaller key (keys of
// INT_MAX last): one ballot per distinct key.
__device__ __forceinline__ int rank_by_key(int key, uint32_t lt) {
  int r = 0;
  for (uint32_t rem = 0xffffffffu; rem;) {
    const int lead = __ffs(rem) - 1;
    const int k = __shfl_sync(0xffffffffu, key, lead);
    const uint32_t grp = __ballot_sync(0xffffffffu, key == k);
    rem &= ~grp;
    if (k < key) r += __popc(grp);
    if (k == key) r += __popc(grp & lt);
  }
  return r;
}

template <typename LabelT, typename TableT, bool kCensus>
__global__ void __launch_bounds__(128, 7) blend_kernel(
    const ViewParams* __restrict__ views, const uint2* __restrict__ ranges,
    const uint32_t* __restrict__ list_val, const ProjRecord* __restrict__ rec,
    const CompactRecord* __restrict__ rec16, int64_t n, int E, TableT* __restrict__ table,
    float* __restrict__ state, uint64_t* __restrict__ sat, uint64_t* __restrict__ subsat,
    uint8_t* __restrict__ sat_chunk, int chunk, unsigned long long* __restrict__ counters) {
  __shared__ BlockSmem B;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpSmem& S = B.w[warp];
  const int v = blockIdx.y;
  const int tiles_x = views[v].tiles_x;
  const int tile = blockIdx.x;
  if (tile >= tiles_x * views[v].tiles_y) return;  // whole block
  const int gtile = views[v].tile_base + tile;
  const uint2 rg = ranges[gtile];
  if (rg.y <= rg.x) return;  // no list entry for this tile in this chunk
  const uint32_t done4 = static_cast<uint32_t>(subsat[gtile >> 4] >> (4 * (gtile & 15))) & 0xFu;
  if (done4 == 0xFu) return;  // every pixel of the tile already stopped
  const int sub = warp;
  const int gsub = 4 * gtile + sub;
  const int W = views[v].width, H = views[v].height;
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
  float2 Tu = make_float2(valid0 ? st[p0] : 0.f, valid1 ? st[p0 + 1] : 0.f);
  // the labels of the warp's pixels: the smallest two, and how many there are
  const uint32_t lt = lanemask_lt();
  int la = 0x7FFFFFFF, lb = 0x7FFFFFFF, n_labels = 0;
  {
    int k0 = valid0 ? lab0 : 0x7FFFFFFF, k1 = valid1 ? lab1 : 0x7FFFFFFF;
    for (; n_labels < 3; ++n_labels) {
      const int m = __reduce_min_sync(0xffffffffu, min(k0, k1));
      if (m == 0x7FFFFFFF) break;
      if (n_labels == 0) la = m;
      if (n_labels == 1) lb = m;
      if (k0 == m) k0 = 0x7FFFFFFF;
      if (k1 == m) k1 = 0x7FFFFFFF;
    }
  }
  const int mode = n_labels <= 1 ? kOneLabel : (n_labels == 2 ? kTwoLabels : kMany);
  const float2 wA = make_float2(valid0 && lab0 == la ? 1.f : 0.f, valid1 && lab1 == la ? 1.f : 0.f);
  const float2 wB = make_float2(valid0 && lab0 == lb ? 1.f : 0.f, valid1 && lab1 == lb ? 1.f : 0.f);
  const int round_size = mode == kTwoLabels ? kRound / 2 : kRound;
  // kMany: the lane's main label (its first labelled pixel's), and whether
  // its second pixel has another one (a label-boundary lane)
  const int main_lab = valid0 ? lab0 : (valid1 ? lab1 : -1);
  const bool minor = mode == kMany && valid0 && valid1 && lab1 != lab0;
  const float wq = minor ? 0.f : 1.f;  // weight of the second pixel in the main-label sum
  // kMany: lane positions ordered by main label (labelless lanes last), and
  // the boundary lanes ordered by their second label; otherwise the lane
  int pos = lane, mpos = 0;
  uint32_t minor_lanes = 0u;
  if (mode == kMany) {
    const int mkey = main_lab >= 0 ? main_lab : 0x7FFFFFFF;
    pos = rank_by_key(mkey, lt);
    minor_lanes = __ballot_sync(0xffffffffu, minor);
    mpos = minor_lanes ? rank_by_key(minor ? lab1 : 0x7FFFFFFF, lt) : 0;
    S.poslab[pos] = mkey;
    if (minor && mpos < kMinorCap) S.minlab[mpos] = lab1;
  }
  bool alive = !((done4 >> sub) & 1u);
  if (lane == 0) {
    B.tail[sub] = 0;
    B.alive[sub] = alive ? 1 : 0;
  }
  __syncthreads();  // every warp reads the others' tails and flags
  uint32_t segmask = 1u;
  int lab_first = la;
  if (mode == kMany) {
    const int plab = S.poslab[lane];
    const int plab_prev = __shfl_up_sync(0xffffffffu, plab, 1);
    segmask = __ballot_sync(0xffffffffu, lane == 0 || plab != plab_prev);
    lab_first = S.poslab[0];
  }
  const int n_minor = min(__popc(minor_lanes), kMinorCap);

  // pixel centres relative to the sub-tile centre, in [-3.5, 3.5]
  const float2 X2 = make_float2(static_cast<float>(lx) - 3.5f, static_cast<float>(lx) - 3.5f);
  const float2 Y2 = make_float2(static_cast<float>(ly) - 3.5f, static_cast<float>(ly) - 3.5f);
  const uint32_t gbase = static_cast<uint32_t>(static_cast<int64_t>(v) * n);
  // -(1e-4 / kSkipScale rounded down to the float below) / ulp
  const float thr = 1e-4f * kTScale;
  const float neg_thr = -__uint_as_float(__float_as_uint(thr) - 1u) * kStepScale;
  // staging: the first kStagers warps take one list entry per thread and step
  const bool stager = threadIdx.x < kStep;
  const float tcx = static_cast<float>(tx * kTile + 8), tcy = static_cast<float>(ty * kTile + 8);
  uint32_t head = 0, n_staged = 0;
  unsigned long long n_eval = 0, n_part = 0;
  unsigned long long n_rounds = 0, n_steps = 0, n_mixed = 0;

  // the stager's list entry of the next step, loaded a step ahead so that
  // the record gather does not wait behind it
  uint32_t g_next = (stager && rg.x + threadIdx.x < rg.y) ? list_val[rg.x + threadIdx.x] : 0u;
  for (uint32_t base = rg.x;; base += kStep) {
    const bool more = base < rg.y;
    const uint32_t g_here = g_next;
    if (stager && base + kStep + threadIdx.x < rg.y) g_next = list_val[base + kStep + threadIdx.x];
    // ---- stage (the stager warps): entry base + threadIdx.x against all four
    // sub-tiles; bit s of keep: the entry goes to sub-tile s's queue
    uint32_t keep = 0u;
    float4 wk = make_float4(0.f, 0.f, 0.f, 0.f);
    float bt0 = 0.f, bt1 = 0.f, nlo = 0.f, clampf = 0.f;
    int32_t gi = 0;
    if (stager && more && base + threadIdx.x < rg.y) {
      const uint32_t g = g_here;
      gi = static_cast<int32_t>(g - gbase);
      float o, qc;
      if (rec16) {
        // reduced-precision record: b = W16 (c - m) in FP32
        const CompactRecord r = rec16[g];
        const float2 wa = __half22float2(*reinterpret_cast<const __half2*>(&r.w01));
        const float2 wb = __half22float2(*reinterpret_cast<const __half2*>(&r.w23));
        wk = make_float4(wa.x, wa.y, wb.x, wb.y);
        const float dx = tcx - r.mx, dy = tcy - r.my;
        bt0 = fmaf(wk.x, dx, wk.y * dy);
        bt1 = fmaf(wk.z, dx, wk.w * dy);
        o = r.o;
        qc = r.q_cut;
        nlo = r.nlo;
      } else {
        // b = W (c - m) at the tile centre c: c - m_hi is exact whenever the
        // mean lies within a factor of two of c (and off by far less than a
        // pixel's 1e-7 otherwise); W = W_hi + W_lo
        const ProjRecord r = rec[g];
        const float dx = (tcx - r.m.x) - r.m.z, dy = (tcy - r.m.y) - r.m.w;
        wk = r.w_hi;
        bt0 = fmaf(wk.x, dx, fmaf(wk.y, dy, fmaf(r.w_lo.x, dx, r.w_lo.y * dy)));
        bt1 = fmaf(wk.z, dx, fmaf(wk.w, dy, fmaf(r.w_lo.z, dx, r.w_lo.w * dy)));
        o = r.misc.x;
        qc = r.misc.y;
        nlo = r.misc.z;
      }
      clampf = o > kAlphaMax ? 1.f : 0.f;
      // over a sub-tile's pixel centres w = W (p - o) + b ranges inside the
      // box b +- 3.5 (|W_k0| + |W_k1|) around b at the sub-tile centre o =
      // c + (-+4, -+4); keep if that box meets |w|^2 <= q_cut
      const float h0 = 3.5f * (fabsf(wk.x) + fabsf(wk.y));
      const float h1 = 3.5f * (fabsf(wk.z) + fabsf(wk.w));
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const float ex = (s & 1) ? 4.f : -4.f, ey = (s & 2) ? 4.f : -4.f;
        const float c0 = fmaf(wk.x, ex, fmaf(wk.y, ey, bt0));
        const float c1 = fmaf(wk.z, ex, fmaf(wk.w, ey, bt1));
        const float d0 = fmaxf(0.f, fabsf(c0) - h0), d1 = fmaxf(0.f, fabsf(c1) - h1);
        if (fmaf(d0, d0, d1 * d1) <= qc && B.alive[s] != 0) keep |= 1u << s;
      }
    }
    uint32_t bal[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) bal[s] = __ballot_sync(0xffffffffu, (keep >> s) & 1u);
    if (stager && lane < 4)
      B.cnt[warp][lane] = __popc(lane == 0 ? bal[0] : lane == 1 ? bal[1] : lane == 2 ? bal[2] : bal[3]);
    // the block is done once no sub-tile is compositing
    if (!__syncthreads_or(alive ? 1 : 0)) break;
    if (kCensus) ++n_steps;
    // the queue tails after this step (entries of warp 0, then of warp 1)
    const uint32_t my_tail = B.tail[sub];
    uint32_t new_tail = my_tail;
#pragma unroll
    for (int w = 0; w < kStagers; ++w) new_tail += B.cnt[w][sub];
    // ---- append the kept entries to the sub-tiles' queues, in list order
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (!((keep >> s) & 1u)) continue;
      uint32_t before = B.tail[s];  // entries queued ahead: earlier steps', earlier stagers'
#pragma unroll
      for (int w = 0; w < kStagers; ++w)
        if (w < warp) before += B.cnt[w][s];
      const uint32_t qi = (before + __popc(bal[s] & lt)) % kQCap;
      WarpSmem& T = B.w[s];
      const int pr = static_cast<int>(qi >> 1), c = static_cast<int>(qi & 1u);
      const float ex = (s & 1) ? 4.f : -4.f, ey = (s & 2) ? 4.f : -4.f;
      float* fx = reinterpret_cast<float*>(&T.wx[pr]);
      float* fy = reinterpret_cast<float*>(&T.wy[pr]);
      float* fb = reinterpret_cast<float*>(&T.bb[pr]);
      float* fo = reinterpret_cast<float*>(&T.oo[pr]);
      fx[c] = wk.x;
      fx[2 + c] = wk.z;
      fy[c] = wk.y;
      fy[2 + c] = wk.w;
      fb[c] = fmaf(wk.x, ex, fmaf(wk.y, ey, bt0));
      fb[2 + c] = fmaf(wk.z, ex, fmaf(wk.w, ey, bt1));
      fo[c] = nlo;
      fo[2 + c] = clampf;
      T.gid[qi] = gi;
    }
    __syncthreads();
    if (lane == 0) B.tail[sub] = new_tail;
    // ---- composite whole rounds (and, at the end of the list, the rest)
    const bool last = base + kStep >= rg.y;
    if (!alive) head = new_tail;
    while (alive && (new_tail - head >= static_cast<uint32_t>(round_size) ||
                     (last && new_tail > head))) {
      const int nq = static_cast<int>(min(new_tail - head, static_cast<uint32_t>(round_size)));
      if (nq & 1) {
        // an odd count gets an empty partner: q = +inf, alpha 0
        const uint32_t qi = (head + nq) % kQCap;
        if (lane == 0) {
          float* fx = reinterpret_cast<float*>(&S.wx[qi >> 1]);
          float* fy = reinterpret_cast<float*>(&S.wy[qi >> 1]);
          float* fb = reinterpret_cast<float*>(&S.bb[qi >> 1]);
          float* fo = reinterpret_cast<float*>(&S.oo[qi >> 1]);
          fx[1] = fx[3] = fy[1] = fy[3] = fb[1] = fb[3] = fo[3] = 0.f;
          fo[1] = __int_as_float(0x7f800000);
        }
        __syncwarp();
      }
      const int pair0 = static_cast<int>((head % kQCap) >> 1);
      const int npairs = (nq + 1) >> 1;
      if (mode == kOneLabel)
        composite_round<kOneLabel, kCensus>(S, pair0, npairs, X2, Y2, neg_thr, wq, wA, wB, pos,
                                            mpos, minor, lab1, E, table, Tu, n_eval, n_part);
      else if (mode == kTwoLabels)
        composite_round<kTwoLabels, kCensus>(S, pair0, npairs, X2, Y2, neg_thr, wq, wA, wB, pos,
                                             mpos, minor, lab1, E, table, Tu, n_eval, n_part);
      else
        composite_round<kMany, kCensus>(S, pair0, npairs, X2, Y2, neg_thr, wq, wA, wB, pos, mpos,
                                        minor, lab1, E, table, Tu, n_eval, n_part);
      __syncwarp();
      if (mode == kTwoLabels) {
        // lanes 0-15: La of round Gaussian lane; lanes 16-31: Lb of lane - 16
        const int gj = lane & 15;
        if (gj < nq)
          reduce_plane(S, lane, static_cast<int64_t>(S.gid[(head + gj) % kQCap]), E,
                       lane < 16 ? la : lb, table);
      } else if (lane < nq) {
        reduce_row(S, lane, static_cast<int64_t>(S.gid[(head + lane) % kQCap]), E,
                   mode == kOneLabel, lab_first, segmask, n_minor, table);
      }
      n_staged += static_cast<uint32_t>(nq);
      head += static_cast<uint32_t>(nq);
      if (kCensus) {
        ++n_rounds;
        if (mode != kOneLabel) ++n_mixed;
      }
      __syncwarp();
      if (!__any_sync(0xffffffffu, Tu.x != 0.f || Tu.y != 0.f)) {
        alive = false;
        head = new_tail;
        if (lane == 0) B.alive[sub] = 0;
      }
    }
    if (last) break;
  }

  if (valid0) st[p0] = Tu.x;
  if (valid1) st[p0 + 1] = Tu.y;
  if (__all_sync(0xffffffffu, Tu.x == 0.f && Tu.y == 0.f) && lane == 0 &&
      !((done4 >> sub) & 1u)) {
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
  if (kCensus) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      n_eval += __shfl_xor_sync(0xffffffffu, n_eval, o);
      n_part += __shfl_xor_sync(0xffffffffu, n_part, o);
    }
    if (lane == 0) {
      if (n_eval) atomicAdd(&counters[kPairs], n_eval);
      if (n_part) atomicAdd(&counters[kCensusPairs], n_part);
      if (n_rounds) atomicAdd(&counters[kRounds], n_rounds);
      if (n_mixed) atomicAdd(&counters[kRoundsMixed], n_mixed);
      if (warp == 0 && n_steps) atomicAdd(&counters[kSteps], n_steps);
    }
  }
  if (lane == 0 && n_staged) atomicAdd(&counters[kStaged], static_cast<unsigned long long>(n_staged));
}

template <typename LabelT, typename TableT>
cudaError_t launch_typed(const ViewParams* views, int n_views, int max_tiles, const uint2* ranges,
                         const uint32_t* list_val, const ProjRecord* rec,
                         const CompactRecord* rec16, int64_t n, int E, void* table, float* state,
                         uint64_t* sat, uint64_t* subsat, uint8_t* sat_chunk, int chunk,
                         unsigned long long* counters, bool census, cudaStream_t stream) {
  dim3 grid(static_cast<unsigned>(max_tiles), static_cast<unsigned>(n_views));
  if (census)
    blend_kernel<LabelT, TableT, true><<<grid, 128, 0, stream>>>(
        views, ranges, list_val, rec, rec16, n, E, static_cast<TableT*>(table), state, sat,
        subsat, sat_chunk, chunk, counters);
  else
    blend_kernel<LabelT, TableT, false><<<grid, 128, 0, stream>>>(
        views, ranges, list_val, rec, rec16, n, E, static_cast<TableT*>(table), state, sat,
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
                         const CompactRecord* rec16, int64_t n, int E, int mask_dtype,
                         void* table, int table_dtype, float* state, uint64_t* sat,
                         uint64_t* subsat, uint8_t* sat_chunk, int chunk,
                         unsigned long long* counters, bool census, cudaStream_t stream) {
  if (n_views == 0 || max_tiles_per_view == 0) return cudaSuccess;
  const int mt = max_tiles_per_view;
  if (mask_dtype == 4) {
    if (table_dtype == 0)
      return launch_typed<uint8_t, float>(views, n_views, mt, ranges, list_val, rec, rec16, n, E,
                                          table, state, sat, subsat, sat_chunk, chunk, counters,
                                          census, stream);
    return launch_typed<uint8_t, double>(views, n_views, mt, ranges, list_val, rec, rec16, n, E,
                                         table, state, sat, subsat, sat_chunk, chunk, counters,
                                         census, stream);
  }
  if (table_dtype == 0)
    return launch_typed<int32_t, float>(views, n_views, mt, ranges, list_val, rec, rec16, n, E,
                                        table, state, sat, subsat, sat_chunk, chunk, counters,
                                        census, stream);
  return launch_typed<int32_t, double>(views, n_views, mt, ranges, list_val, rec, rec16, n, E,
                                       table, state, sat, subsat, sat_chunk, chunk, counters,
                                       census, stream);
}

}  // namespace fs
