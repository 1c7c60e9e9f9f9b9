// Shared device-side definitions of the FlashSplat CUDA path (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fs {

constexpr int kTile = 16;                 // 16x16 pixel tiles (Sec. 3.1)
constexpr int kTilePixels = kTile * kTile;

// Thresholds of the compositing rule (Sec. 3.1 Eq. 1 with the rasteriser's
// conventions): alpha below 1/255 is skipped, alpha is clamped to 0.99, and a
// pixel stops before a Gaussian that would take T below 1e-4.
constexpr float kAlphaMin = (float)(1.0 / 255.0);
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kLowPass = 0.3f;          // px^2 added to the 2D covariance diagonal
// 0.5 * log2(e): alpha = o * 2^(-|W d|^2) with W = sqrt(kHalfLog2e) Lambda^-1/2 V^T
constexpr double kHalfLog2e = 0.72134752044448170368;
constexpr float kHalfLog2eHi = static_cast<float>(kHalfLog2e);
constexpr float kHalfLog2eLo = static_cast<float>(kHalfLog2e - static_cast<double>(kHalfLog2eHi));

// Slot ids are view * n + Gaussian index.  The view of a slot by a multiply:
// with m = floor((2^32 - 1) / n), umulhi(g, m) is floor(g / n) or one less.
struct SlotView {
  uint32_t n, m;
  __host__ __device__ __forceinline__ explicit SlotView(int64_t n_)
      : n(static_cast<uint32_t>(n_)), m(0xFFFFFFFFu / static_cast<uint32_t>(n_)) {}
  __device__ __forceinline__ uint32_t operator()(uint32_t g) const {
    uint32_t q = __umulhi(g, m);
    if (g - q * n >= n) ++q;
    return q;
  }
};

// Per-view parameters, prepared on the host.  Double precision quantities are
// carried as float pairs (hi + lo) so the projection needs no FP64 pipe.
struct ViewParams {
  float R_hi[9], R_lo[9];      // world->camera rotation, row-major
  float t_hi[3], t_lo[3];
  float fx_hi, fx_lo, fy_hi, fy_lo, cx_hi, cx_lo, cy_hi, cy_lo;
  float near_hi, near_lo;      // near plane 0.2 as a float pair
  float limx_hi, limx_lo;      // 1.3 * tan(half field of view), x
  float limy_hi, limy_lo;      // 1.3 * tan(half field of view), y
  int32_t width, height;
  int32_t tiles_x, tiles_y;
  int32_t tile_base;           // first tile id of this view in the batch
  int32_t pad0;
  int64_t state_off;           // first pixel of this view in the batch's pixel state
  const void* mask;            // device pointer to the view's labels
  // 3-sigma tile coverage: per (view, Gaussian) slot, indexed like the
  // footprints, the tile columns the Gaussian may reach (first | last << 16);
  // written by the projection.  NULL: exact coverage.
  uint32_t* cols;
  // Per view, the 2-D prefix sums of its unsaturated tiles for the binning's
  // slot test: (tiles_y + 1) x (tiles_x + 1) counts, entry r * (tiles_x + 1)
  // + c = unsaturated tiles in rows < r and columns < c, rebuilt before each
  // binning.  NULL: the test walks the saturation bits row by row.
  uint32_t* free_tab;
};

// Projected record of one (view, Gaussian): 4 x float4 = 64 B.
//   w_hi, w_lo = whitening matrix W (row-major 2x2) as float pairs, with
//                |W d|^2 = 0.5 log2(e) d^T Sigma2D^-1 d
//   m          = (mx_hi, my_hi, mx_lo, my_lo): the projected mean as float pairs
//   misc       = (opacity, q_cut, -log2 o, depth), q_cut ~ log2(255 o): alpha =
//                o 2^-|w|^2 reaches 1/255 at |w|^2 = log2(255 o) (stored
//                slightly widened); depth = view-space depth of the mean
//                (FP32), read by the mask renderer
// For a sub-tile whose centre is o the blend forms b = W (o - m) in FP32 (o - m
// is exact or nearly so) and evaluates w = W_hi (p - o) + b for the pixel
// centre p, |p - o| <= 5 px.
struct alignas(16) ProjRecord {
  float4 w_hi;
  float4 w_lo;
  float4 m;
  float4 misc;
};

// Reduced-precision record of one (view, Gaussian): 32 B, one DRAM sector.
// The mean stays FP32; the whitening matrix W is stored as four FP16 values
// (correctly rounded from the float pairs), so alpha = o 2^-|W16 (p - m)|^2.
// The opacity o (the scene's own value) and the cut q_cut ~ log2(255 o) ride
// along so the blend needs no second gather.  |W d|^2 stays a sum of squares
// whatever the rounding, unlike an FP16 conic, which can lose positive
// definiteness for elongated footprints.
struct alignas(16) CompactRecord {
  float mx, my;
  uint32_t w01, w23;  // (W00, W01), (W10, W11) as FP16 pairs, low half first
  float o, q_cut;
  float nlo;          // -log2 o
  float depth;        // view-space depth of the mean (FP32)
};

// Footprint of one (view, Gaussian) for the tile binning: the alpha >= 1/255
// ellipse {d : d^T Sigma2D^-1 d <= r2} around the projected mean, r2 slightly
// inflated, in FP32 (the binning is conservative: it also adds a pixel of
// margin).  With S = Sigma2D, the ellipse's x-range at height dy is
//   x(dy) = mx + a dy +- sqrt(b2 (syr - dy^2)),  a = Sxy/Syy, b2 = det S / Syy^2,
//   syr = Syy r2  (|dy| <= hy = sqrt(syr)),
// and its rightmost point lies at dy* = Sxy sqrt(r2 / Sxx).
struct alignas(16) Footprint {
  float mx, my;            // projected mean (pixels)
  float hy, syr;           // half height of the ellipse, and its square
  float dys;               // dy of the rightmost point
  float a, b2;             // slope and width factor of x(dy)
  uint32_t rows;           // first | last tile row << 16
};

// ---------------------------------------------------------------------------
// Float-pair ("double-float") arithmetic: error-free transformations of
// Knuth (TwoSum), Dekker/FMA (TwoProduct) and the compensated dot product of
// Ogita, Rump and Oishi (2005).  Values are hi + lo with |lo| <= ulp(hi)/2.
// ---------------------------------------------------------------------------
struct f2 {
  float hi, lo;
};

__device__ __forceinline__ f2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ f2 fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

__device__ __forceinline__ f2 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  return {p, e};
}

// Sum of float pairs (Dekker's addition): error below ~2^-44 (|a| + |b|),
// i.e. about 1e-11 relative to the result even when a and b cancel to three
// orders of magnitude -- far more than any quantity here needs.
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  const f2 s = two_sum(a.hi, b.hi);
  const float e = __fadd_rn(__fadd_rn(s.lo, a.lo), b.lo);
  return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ f2 f2_mul_f(f2 a, float b) {
  f2 p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

// a / b for float pairs: one correction step of the float quotient.
__device__ __forceinline__ f2 f2_div(f2 a, f2 b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  // r = a - q1 * b, exactly up to the lo terms
  const f2 p = two_prod(q1, b.hi);
  float r = __fsub_rn(a.hi, p.hi);
  r = __fsub_rn(r, p.lo);
  r = __fadd_rn(r, a.lo);
  r = __fmaf_rn(-q1, b.lo, r);
  const float q2 = __fdiv_rn(r, b.hi);
  return fast_two_sum(q1, q2);
}

// sum_k a_k * x_k + c for float-pair a_k, c and float x_k (compensated dot product).
__device__ __forceinline__ f2 f2_dot3_add(const float* a_hi, const float* a_lo, float x0, float x1,
                                          float x2, float c_hi, float c_lo) {
  f2 p0 = two_prod(a_hi[0], x0);
  f2 p1 = two_prod(a_hi[1], x1);
  f2 p2 = two_prod(a_hi[2], x2);
  float err = __fmaf_rn(a_lo[0], x0, p0.lo);
  err = __fadd_rn(err, __fmaf_rn(a_lo[1], x1, p1.lo));
  err = __fadd_rn(err, __fmaf_rn(a_lo[2], x2, p2.lo));
  f2 s = two_sum(p0.hi, p1.hi);
  err = __fadd_rn(err, s.lo);
  s = two_sum(s.hi, p2.hi);
  err = __fadd_rn(err, s.lo);
  s = two_sum(s.hi, c_hi);
  err = __fadd_rn(err, s.lo);
  err = __fadd_rn(err, c_lo);
  return fast_two_sum(s.hi, err);
}

__device__ __forceinline__ f2 f2_from(float x) { return {x, 0.f}; }
__device__ __forceinline__ f2 f2_neg(f2 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) { return f2_add(a, f2_neg(b)); }
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) { return f2_add(f2_mul(a, b), c); }
__device__ __forceinline__ f2 f2_scale(f2 a, float s) {  // exact for powers of two
  return {a.hi * s, a.lo * s};
}

// sqrt of a float pair: one Newton correction of the float square root.
__device__ __forceinline__ f2 f2_sqrt(f2 a) {
  if (!(a.hi > 0.f)) return {0.f, 0.f};
  const float s = __fsqrt_rn(a.hi);
  const f2 p = two_prod(s, s);
  float r = __fsub_rn(a.hi, p.hi);
  r = __fsub_rn(r, p.lo);
  r = __fadd_rn(r, a.lo);
  const float c = __fdiv_rn(r, __fadd_rn(s, s));
  return fast_two_sum(s, c);
}

// Two float pairs side by side, for the packed FP32 instructions (FADD2,
// FMUL2, FFMA2): each lane runs exactly the operation sequence of the scalar
// f2 functions above, so results are bit-identical to them, in about half the
// issued instructions.  x - y is formed as fma(y, -1, x), which rounds like
// the subtraction itself.
struct f2x2 {
  float2 hi, lo;
};

__device__ __forceinline__ f2x2 f2x2_pack(f2 x, f2 y) {
  return {make_float2(x.hi, y.hi), make_float2(x.lo, y.lo)};
}
__device__ __forceinline__ f2 f2x2_first(const f2x2& v) { return {v.hi.x, v.lo.x}; }
__device__ __forceinline__ f2 f2x2_second(const f2x2& v) { return {v.hi.y, v.lo.y}; }

__device__ __forceinline__ float2 add2(float2 x, float2 y) { return __fadd2_rn(x, y); }
__device__ __forceinline__ float2 sub2(float2 x, float2 y) {
  return __ffma2_rn(y, make_float2(-1.f, -1.f), x);
}
__device__ __forceinline__ float2 neg2(float2 x) { return make_float2(-x.x, -x.y); }

__device__ __forceinline__ f2x2 f2x2_add(const f2x2& a, const f2x2& b) {
  // two_sum of the hi parts
  const float2 s = add2(a.hi, b.hi);
  const float2 bb = sub2(s, a.hi);
  const float2 e0 = add2(sub2(a.hi, sub2(s, bb)), sub2(b.hi, bb));
  const float2 e = add2(add2(e0, a.lo), b.lo);
  // fast_two_sum(s, e)
  const float2 r = add2(s, e);
  return {r, sub2(e, sub2(r, s))};
}

__device__ __forceinline__ f2x2 f2x2_neg(const f2x2& a) { return {neg2(a.hi), neg2(a.lo)}; }
__device__ __forceinline__ f2x2 f2x2_sub(const f2x2& a, const f2x2& b) {
  return f2x2_add(a, f2x2_neg(b));
}

__device__ __forceinline__ f2x2 f2x2_mul(const f2x2& a, const f2x2& b) {
  // two_prod of the hi parts, then the cross terms
  const float2 p = __fmul2_rn(a.hi, b.hi);
  float2 e = __ffma2_rn(a.hi, b.hi, neg2(p));
  e = __ffma2_rn(a.hi, b.lo, __ffma2_rn(a.lo, b.hi, e));
  const float2 r = add2(p, e);
  return {r, sub2(e, sub2(r, p))};
}

__device__ __forceinline__ f2x2 f2x2_fma(const f2x2& a, const f2x2& b, const f2x2& c) {
  return f2x2_add(f2x2_mul(a, b), c);
}

// f2_dot3_add for two rows at once: lane r computes
// sum_k a_r,k * x_k + c_r with the scalar function's operation sequence.
__device__ __forceinline__ f2x2 f2x2_dot3_add(const float* a0_hi, const float* a0_lo,
                                              const float* a1_hi, const float* a1_lo, float x0,
                                              float x1, float x2, float2 c_hi, float2 c_lo) {
  const float2 X0 = make_float2(x0, x0), X1 = make_float2(x1, x1), X2 = make_float2(x2, x2);
  const float2 h0 = make_float2(a0_hi[0], a1_hi[0]), h1 = make_float2(a0_hi[1], a1_hi[1]);
  const float2 h2 = make_float2(a0_hi[2], a1_hi[2]);
  const float2 l0 = make_float2(a0_lo[0], a1_lo[0]), l1 = make_float2(a0_lo[1], a1_lo[1]);
  const float2 l2 = make_float2(a0_lo[2], a1_lo[2]);
  const float2 p0 = __fmul2_rn(h0, X0), p1 = __fmul2_rn(h1, X1), p2 = __fmul2_rn(h2, X2);
  const float2 q0 = __ffma2_rn(h0, X0, neg2(p0)), q1 = __ffma2_rn(h1, X1, neg2(p1));
  const float2 q2 = __ffma2_rn(h2, X2, neg2(p2));
  float2 err = __ffma2_rn(l0, X0, q0);
  err = add2(err, __ffma2_rn(l1, X1, q1));
  err = add2(err, __ffma2_rn(l2, X2, q2));
  // two_sum(p0, p1), two_sum(s, p2), two_sum(s, c_hi), each error into err
  float2 s = add2(p0, p1);
  float2 bb = sub2(s, p0);
  err = add2(err, add2(sub2(p0, sub2(s, bb)), sub2(p1, bb)));
  float2 s2 = add2(s, p2);
  bb = sub2(s2, s);
  err = add2(err, add2(sub2(s, sub2(s2, bb)), sub2(p2, bb)));
  float2 s3 = add2(s2, c_hi);
  bb = sub2(s3, s2);
  err = add2(err, add2(sub2(s2, sub2(s3, bb)), sub2(c_hi, bb)));
  err = add2(err, c_lo);
  const float2 r = add2(s3, err);
  return {r, sub2(err, sub2(r, s3))};
}

__device__ __forceinline__ bool f2_lt(f2 a, f2 b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

// Order-preserving map of a positive float to uint32 (depth keys).
__device__ __forceinline__ uint32_t depth_key(float z) { return __float_as_uint(z); }

// Order-preserving map of any float to uint32 (low word of a float-pair depth).
__device__ __forceinline__ uint32_t float_order_key(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// 2^x by the hardware approximation (relative error ~2^-22, flushes
// subnormal results to zero): alpha = o 2^-|w|^2 in the compositing kernels.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

}  // namespace fs
