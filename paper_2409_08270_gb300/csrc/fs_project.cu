// Scene preparation, EWA projection and tile binning (Sec. 3.1).
//
// Projection of Gaussian i into view v, in float-pair arithmetic (about 48
// significant bits, no FP64 pipe):
//   t = R m + t_c                              (compensated dot product)
//   m2D = (fx tx/tz + cx, fy ty/tz + cy)
//   J = perspective Jacobian at t, tx/tz and ty/tz clamped to 1.3 tan(fov/2)
//   Sigma2D = (J W) Sigma3D (J W)^T + 0.3 I,   W = camera rotation
//   Sigma2D = lambda1 e e^T + lambda2 e' e'^T  (lambda2 = det / lambda1)
// The record stores the whitening matrix W_ws = sqrt(0.5 log2 e)
// diag(lambda1, lambda2)^-1/2 [e e']^T and the mean m2D as float pairs (hi,
// lo), so alpha = o 2^-|W_ws (p - m2D)|^2.  Carrying the eigenvectors
// to ~1e-14 keeps thin ("needle") Gaussians correctly oriented: an FP32
// orientation error of 1e-7 rad moves alpha at the tip of a 4500:1 Gaussian
// by ~1e-4.  Sigma3D = R(q) diag(s^2) R(q)^T is formed once per scene in FP64
// and kept as float pairs.
//
// Binning: a tile is listed for a Gaussian when its pixel centres, widened
// by one pixel, can meet the alpha >= 1/255 ellipse {d^T Sigma2D^-1 d <= r2},
// r2 = 2 ln(255 o) (slightly inflated).  For every tile row the x-extent of
// the ellipse over that row's band is exact (the boundary's extreme points),
// so far fewer tiles are listed than with the bounding box.
#include <cuda_fp16.h>

#include "fs_binning.cuh"
#include "fs_common.cuh"
#include "fs_internal.h"

namespace fs {

// ---------------------------------------------------------------------------
// scene preparation: covariance in FP64 (once), packed attributes, validation
// ---------------------------------------------------------------------------

__device__ __forceinline__ float load_attr(const void* p, int64_t idx, int dtype) {
  if (dtype == 0) return static_cast<const float*>(p)[idx];
  const uint16_t bits = static_cast<const uint16_t*>(p)[idx];
  if (dtype == 2) return __uint_as_float(static_cast<uint32_t>(bits) << 16);  // bf16
  return __half2float(__ushort_as_half(bits));                                 // fp16
}

__device__ __forceinline__ void split_d(double x, float* hi, float* lo) {
  const float h = static_cast<float>(x);
  *hi = h;
  *lo = static_cast<float>(x - static_cast<double>(h));
}

__global__ void scene_prep_kernel(int64_t n, const float* __restrict__ mean, const void* quat,
                                  int quat_dtype, const void* scale, int scale_dtype,
                                  const void* opacity, int opacity_dtype, float4* __restrict__ pos_op,
                                  float4* __restrict__ cov, unsigned int* __restrict__ err) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float mx = mean[3 * i], my = mean[3 * i + 1], mz = mean[3 * i + 2];
  const float o = load_attr(opacity, i, opacity_dtype);
  const float q0 = load_attr(quat, 4 * i, quat_dtype), q1 = load_attr(quat, 4 * i + 1, quat_dtype);
  const float q2 = load_attr(quat, 4 * i + 2, quat_dtype), q3 = load_attr(quat, 4 * i + 3, quat_dtype);
  const float s0 = load_attr(scale, 3 * i, scale_dtype), s1 = load_attr(scale, 3 * i + 1, scale_dtype);
  const float s2 = load_attr(scale, 3 * i + 2, scale_dtype);
  bool bad = !(isfinite(mx) && isfinite(my) && isfinite(mz) && isfinite(o) && isfinite(q0) &&
               isfinite(q1) && isfinite(q2) && isfinite(q3) && isfinite(s0) && isfinite(s1) &&
               isfinite(s2));
  const double nn = (double)q0 * q0 + (double)q1 * q1 + (double)q2 * q2 + (double)q3 * q3;
  if (!(nn > 0.0)) bad = true;
  if (bad) {
    atomicOr(err, 1u);
    pos_op[i] = make_float4(0.f, 0.f, -1e30f, 0.f);
    cov[3 * i] = cov[3 * i + 1] = cov[3 * i + 2] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  // Sigma3D = Rq diag(s^2) Rq^T in FP64 (once per scene)
  const double inv = 1.0 / sqrt(nn);
  const double w = q0 * inv, x = q1 * inv, y = q2 * inv, z = q3 * inv;
  double Rq[3][3];
  Rq[0][0] = 1.0 - 2.0 * (y * y + z * z);
  Rq[0][1] = 2.0 * (x * y - w * z);
  Rq[0][2] = 2.0 * (x * z + w * y);
  Rq[1][0] = 2.0 * (x * y + w * z);
  Rq[1][1] = 1.0 - 2.0 * (x * x + z * z);
  Rq[1][2] = 2.0 * (y * z - w * x);
  Rq[2][0] = 2.0 * (x * z - w * y);
  Rq[2][1] = 2.0 * (y * z + w * x);
  Rq[2][2] = 1.0 - 2.0 * (x * x + y * y);
  const double sq[3] = {(double)s0 * s0, (double)s1 * s1, (double)s2 * s2};
  const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
  float h[6], lo[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double acc = 0.0;
    for (int l = 0; l < 3; ++l) acc += Rq[ia[k]][l] * sq[l] * Rq[ib[k]][l];
    split_d(acc, &h[k], &lo[k]);
  }
  pos_op[i] = make_float4(mx, my, mz, o);
  // (s00, s01, s02, s11, s12, s22) as (hi, lo) pairs
  cov[3 * i] = make_float4(h[0], lo[0], h[1], lo[1]);
  cov[3 * i + 1] = make_float4(h[2], lo[2], h[3], lo[3]);
  cov[3 * i + 2] = make_float4(h[4], lo[4], h[5], lo[5]);
}

// ---------------------------------------------------------------------------
// projection
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool f2_greater(f2 a, float b_hi, float b_lo) {
  return a.hi > b_hi || (a.hi == b_hi && a.lo > b_lo);
}

__device__ __forceinline__ f2 f2_clamp(f2 x, float lim_hi, float lim_lo) {
  const f2 lim = {lim_hi, lim_lo}, nlim = {-lim_hi, -lim_lo};
  if (f2_lt(x, nlim)) return nlim;
  if (f2_lt(lim, x)) return lim;
  return x;
}

// x rounded to FP16 (round to nearest, ties to even), x a float pair: the
// float rounding of hi is corrected when hi sits exactly halfway between two
// FP16 values and lo says on which side x lies.
__device__ __forceinline__ uint16_t f2_to_half_rn(f2 x) {
  const __half h = __float2half_rn(x.hi);
  const float hf = __half2float(h);
  if (x.lo == 0.f || hf == x.hi) return __half_as_ushort(h);
  // the FP16 neighbour on the other side of hi
  const uint16_t hb = __half_as_ushort(h);
  const bool up_in_magnitude = (fabsf(x.hi) > fabsf(hf));
  const uint16_t ob = static_cast<uint16_t>(up_in_magnitude ? hb + 1 : hb - 1);
  const float of = __half2float(__ushort_as_half(ob));
  if (0.5f * (hf + of) != x.hi) return hb;  // not a tie: hi's rounding is x's
  // tie on hi alone: x lies towards lo's side
  const bool towards_other = (x.lo > 0.f) == (of > hf);
  return towards_other ? ob : hb;
}

// One thread per Gaussian; it projects the Gaussian into every view of the
// batch so the scene is read once per batch.  rec16 != NULL: the record is
// written in the reduced-precision form instead (rec is not written).  The
// paired float-pair quantities (the two rows of the Jacobian-rotation product,
// the two rows of T Sigma3D, the x and y halves of the pinhole map, the rows
// of W) run in packed FP32 (f2x2), bit-identical to the scalar form.  Three
// blocks per SM (80 registers) spill less than four.
template <bool kFast>
__global__ void __launch_bounds__(256, kFast ? 4 : 3) project_kernel(
    int64_t n, int n_views, const ViewParams* __restrict__ views_g,
    const float4* __restrict__ pos_op, const float4* __restrict__ cov3,
    ProjRecord* __restrict__ rec, CompactRecord* __restrict__ rec16, Footprint* __restrict__ foot,
    uint32_t* __restrict__ cnt, uint32_t* __restrict__ key, uint32_t* __restrict__ val,
    uint32_t* __restrict__ depth_lo, uint32_t* __restrict__ key_range) {
  __shared__ ViewParams views[kMaxViewsPerBatch];
  for (int k = threadIdx.x; k < n_views * (int)(sizeof(ViewParams) / 4); k += blockDim.x)
    reinterpret_cast<uint32_t*>(views)[k] = reinterpret_cast<const uint32_t*>(views_g)[k];
  __syncthreads();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  uint32_t kmin = 0xFFFFFFFFu, kmax = 0u;  // visible depth keys of this thread
  uint32_t n_vis = 0;                       // and their number
  if (i < n) {
  const float4 po = pos_op[i];
  const float4 ca = cov3[3 * i], cb = cov3[3 * i + 1], cc = cov3[3 * i + 2];
  const f2 S00 = {ca.x, ca.y}, S01 = {ca.z, ca.w}, S02 = {cb.x, cb.y};
  const f2 S11 = {cb.z, cb.w}, S12 = {cc.x, cc.y}, S22 = {cc.z, cc.w};
  const f2 S[3][3] = {{S00, S01, S02}, {S01, S11, S12}, {S02, S12, S22}};
  const float o = po.w;
  const bool opaque_enough = o >= kAlphaMin;
  const float r2 = opaque_enough ? fmaxf(2.f * logf(255.f * o), 0.f) : 0.f;
  const float nlo = opaque_enough ? -log2f(o) : 0.f;  // alpha = 2^-(|w|^2 - log2 o)

  for (int v = 0; v < n_views; ++v) {
    const ViewParams& vp = views[v];
    const int64_t slot = static_cast<int64_t>(v) * n + i;
    const f2x2 txy = f2x2_dot3_add(vp.R_hi + 0, vp.R_lo + 0, vp.R_hi + 3, vp.R_lo + 3, po.x, po.y,
                                   po.z, make_float2(vp.t_hi[0], vp.t_hi[1]),
                                   make_float2(vp.t_lo[0], vp.t_lo[1]));
    const f2 tx = f2x2_first(txy), ty = f2x2_second(txy);
    const f2 tz = f2_dot3_add(vp.R_hi + 6, vp.R_lo + 6, po.x, po.y, po.z, vp.t_hi[2], vp.t_lo[2]);
    bool visible = opaque_enough && f2_greater(tz, vp.near_hi, vp.near_lo);
    uint32_t count = 0;
    float depth = 0.f, depth_l = 0.f;
    ProjRecord R;
    R.w_hi = R.w_lo = R.m = make_float4(0.f, 0.f, 0.f, 0.f);
    CompactRecord R16 = {0.f, 0.f, 0u, 0u, 0.f, 0.f, 0.f, 0.f};
    // misc.y: |w|^2 at which alpha falls to 1/255, log2(255 o), widened by
    // 0.1% + 1e-3 so the blend's sub-tile test stays conservative in FP32
    const float qcut = opaque_enough ? fmaxf(log2f(255.f * o), 0.f) * 1.001f + 1e-3f : 0.f;
    R.misc = make_float4(o, qcut, nlo, 0.f);
    R16.o = o;
    R16.q_cut = qcut;
    R16.nlo = nlo;
    Footprint F;
    F.mx = F.my = F.hy = F.syr = F.dys = F.a = F.b2 = 0.f;
    F.rows = 0x0000FFFFu;  // no tile row (first row 65535 > last row 0)
    uint32_t col_clip = 0x0000FFFFu;  // 3-sigma coverage: no tile column
    if (visible) {
      float sxx, sxy, syy, det32, mx32, my32;  // 2D covariance and mean for the footprint
      if constexpr (kFast) {
        // reduced-precision form: the record keeps an FP16 W and an FP32
        // mean, so the 2D covariance, its eigen-decomposition and W run in
        // plain FP32 (correctly rounded divisions and roots); the depth stays
        // a float pair for the order
        depth = tz.hi;
        depth_l = tz.lo;
        R16.depth = depth;
        const float iz = __fdiv_rn(1.f, tz.hi);
        const float uxf = __fmul_rn(tx.hi, iz), uyf = __fmul_rn(ty.hi, iz);
        mx32 = fmaf(vp.fx_hi, uxf, vp.cx_hi);
        my32 = fmaf(vp.fy_hi, uyf, vp.cy_hi);
        const float jx = vp.fx_hi * iz, jy = vp.fy_hi * iz;
        const float ucx = fminf(fmaxf(uxf, -vp.limx_hi), vp.limx_hi);
        const float ucy = fminf(fmaxf(uyf, -vp.limy_hi), vp.limy_hi);
        float T0[3], T1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          T0[k] = jx * fmaf(-ucx, vp.R_hi[6 + k], vp.R_hi[k]);
          T1[k] = jy * fmaf(-ucy, vp.R_hi[6 + k], vp.R_hi[3 + k]);
        }
        float a = 0.f, b = 0.f, c = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float m0 = fmaf(T0[0], S[0][j].hi, fmaf(T0[1], S[1][j].hi, T0[2] * S[2][j].hi));
          const float m1 = fmaf(T1[0], S[0][j].hi, fmaf(T1[1], S[1][j].hi, T1[2] * S[2][j].hi));
          a = fmaf(m0, T0[j], a);
          c = fmaf(m1, T1[j], c);
          b = fmaf(m0, T1[j], b);
        }
        a += kLowPass;
        c += kLowPass;
        // a c - b^2 with the rounding error of b^2 put back (Kahan)
        const float bb = b * b;
        const float dt = fmaf(a, c, -bb) - fmaf(b, b, -bb);
        const float h = 0.5f * (a - c);
        const float rr = __fsqrt_rn(fmaf(h, h, bb));
        const float lam1 = 0.5f * (a + c) + rr;
        const float lam2 = __fdiv_rn(dt, lam1);
        float ex, ey;
        if (h >= 0.f) {
          ex = h + rr;
          ey = b;
        } else {
          ex = b;
          ey = rr - h;
        }
        const float en = __fsqrt_rn(fmaf(ex, ex, ey * ey));
        if (en > 0.f) {
          ex = __fdiv_rn(ex, en);
          ey = __fdiv_rn(ey, en);
        } else {
          ex = 1.f;
          ey = 0.f;
        }
        const float k1 = __fsqrt_rn(__fdiv_rn(kHalfLog2eHi, lam1));
        const float k2 = __fsqrt_rn(__fdiv_rn(kHalfLog2eHi, lam2));
        R16.mx = mx32;
        R16.my = my32;
        R16.w01 = static_cast<uint32_t>(__half_as_ushort(__float2half_rn(ex * k1))) |
                  (static_cast<uint32_t>(__half_as_ushort(__float2half_rn(ey * k1))) << 16);
        R16.w23 = static_cast<uint32_t>(__half_as_ushort(__float2half_rn(-ey * k2))) |
                  (static_cast<uint32_t>(__half_as_ushort(__float2half_rn(ex * k2))) << 16);
        sxx = a;
        sxy = b;
        syy = c;
        det32 = dt;
      } else {
        // one float-pair reciprocal of the depth, then (x, y) / z side by side
        const f2 iz = f2_div(f2_from(1.f), tz);
        const f2x2 uxy = f2x2_mul(f2x2_pack(tx, ty), f2x2_pack(iz, iz));
        const f2 ux = f2x2_first(uxy), uy = f2x2_second(uxy);
        const f2 fx = {vp.fx_hi, vp.fx_lo}, fy = {vp.fy_hi, vp.fy_lo};
        // the x and y halves of the pinhole map run side by side (f2x2)
        const f2x2 fxy = f2x2_pack(fx, fy);
        const f2x2 mxy = f2x2_add(f2x2_mul(fxy, f2x2_pack(ux, uy)),
                                  f2x2_pack(f2{vp.cx_hi, vp.cx_lo}, f2{vp.cy_hi, vp.cy_lo}));
        const f2 mx = f2x2_first(mxy), my = f2x2_second(mxy);
        depth = tz.hi;
        depth_l = tz.lo;
        R.misc.w = depth;
        R16.depth = depth;
        const f2x2 J = f2x2_mul(fxy, f2x2_pack(iz, iz));  // (fx / z, fy / z)
        const f2 uxc = f2_clamp(ux, vp.limx_hi, vp.limx_lo);
        const f2 uyc = f2_clamp(uy, vp.limy_hi, vp.limy_lo);
        const f2x2 U = f2x2_pack(uxc, uyc);
        // rows of J W side by side: T[k] = (T0[k], T1[k]) with
        // T0 = fx/z (W0 - ux W2), T1 = fy/z (W1 - uy W2)
        f2x2 T[3];
  #pragma unroll
        for (int k = 0; k < 3; ++k) {
          const f2 w0 = {vp.R_hi[k], vp.R_lo[k]}, w1 = {vp.R_hi[3 + k], vp.R_lo[3 + k]};
          const f2 w2 = {vp.R_hi[6 + k], vp.R_lo[6 + k]};
          T[k] = f2x2_mul(J, f2x2_sub(f2x2_pack(w0, w1), f2x2_mul(U, f2x2_pack(w2, w2))));
        }
        // Sigma' = T Sigma3D T^T: M = (m0, m1) = rows of T Sigma3D, then
        // (a, c) += (m0 T0[j], m1 T1[j]) side by side and b += m0 T1[j]
        f2x2 ac = f2x2_pack(f2_from(0.f), f2_from(0.f));
        f2 a, b = f2_from(0.f), c;
  #pragma unroll
        for (int j = 0; j < 3; ++j) {
          f2x2 M = f2x2_mul(T[0], f2x2_pack(S[0][j], S[0][j]));
          M = f2x2_fma(T[1], f2x2_pack(S[1][j], S[1][j]), M);
          M = f2x2_fma(T[2], f2x2_pack(S[2][j], S[2][j]), M);
          ac = f2x2_fma(M, T[j], ac);
          b = f2_fma(f2x2_first(M), f2x2_second(T[j]), b);
        }
        a = f2x2_first(ac);
        c = f2x2_second(ac);
        a = f2_add(a, f2_from(kLowPass));
        c = f2_add(c, f2_from(kLowPass));
        const f2 det = f2_sub(f2_mul(a, c), f2_mul(b, b));
        const f2 h = f2_scale(f2_sub(a, c), 0.5f);
        const f2 rr = f2_sqrt(f2_add(f2_mul(h, h), f2_mul(b, b)));
        const f2 lam1 = f2_add(f2_scale(f2_add(a, c), 0.5f), rr);
        const f2 lam2 = f2_div(det, lam1);
        // unit eigenvector of lambda1 from whichever form has no cancellation
        f2 ex, ey;
        if (h.hi >= 0.f) {
          ex = f2_add(h, rr);
          ey = b;
        } else {
          ex = b;
          ey = f2_sub(rr, h);
        }
        const f2 en = f2_sqrt(f2_add(f2_mul(ex, ex), f2_mul(ey, ey)));
        if (en.hi > 0.f) {
          const f2 ien = f2_div(f2_from(1.f), en);
          const f2x2 e = f2x2_mul(f2x2_pack(ex, ey), f2x2_pack(ien, ien));
          ex = f2x2_first(e);
          ey = f2x2_second(e);
        } else {
          ex = f2_from(1.f);
          ey = f2_from(0.f);
        }
        // axis scales sqrt(0.5 log2 e / lambda) as float pairs too: the FP64
        // near-tie re-check evaluates alpha from this record
        const f2 hl = {kHalfLog2eHi, kHalfLog2eLo};
        const f2 k1 = f2_sqrt(f2_div(hl, lam1));
        const f2 k2 = f2_sqrt(f2_div(hl, lam2));
        const f2x2 W0 = f2x2_mul(f2x2_pack(ex, ey), f2x2_pack(k1, k1));
        const f2x2 W1 = f2x2_mul(f2x2_pack(f2_neg(ey), ex), f2x2_pack(k2, k2));
        const f2 W00 = f2x2_first(W0), W01 = f2x2_second(W0);
        const f2 W10 = f2x2_first(W1), W11 = f2x2_second(W1);
        R.w_hi = make_float4(W00.hi, W01.hi, W10.hi, W11.hi);
        R.w_lo = make_float4(W00.lo, W01.lo, W10.lo, W11.lo);
        R.m = make_float4(mx.hi, my.hi, mx.lo, my.lo);
        if (rec16) {
          R16.mx = mx.hi;  // the float pair is normalised: hi is the FP32 rounding
          R16.my = my.hi;
          R16.w01 = static_cast<uint32_t>(f2_to_half_rn(W00)) |
                    (static_cast<uint32_t>(f2_to_half_rn(W01)) << 16);
          R16.w23 = static_cast<uint32_t>(f2_to_half_rn(W10)) |
                    (static_cast<uint32_t>(f2_to_half_rn(W11)) << 16);
        }
        sxx = a.hi;
        sxy = b.hi;
        syy = c.hi;
        det32 = det.hi;
        mx32 = mx.hi;
        my32 = my.hi;
      }
      // binning footprint (FP32 is plenty: the binning keeps a pixel of margin)
      const float r2b = binning_r2(r2);
      F.mx = mx32;
      F.my = my32;
      F.syr = syy * r2b;
      F.hy = sqrtf(F.syr);
      F.dys = sxy * sqrtf(r2b / sxx);
      F.a = sxy / syy;
      F.b2 = det32 / (syy * syy);
      const float hy = F.hy;
      const float py0 = ceilf(__fsub_rn(__fsub_rn(F.my, hy), 1.5f));
      const float py1 = floorf(__fadd_rn(__fadd_rn(F.my, hy), 0.5f));
      // visible when the widened bounding box meets the image; the exact
      // per-row tile spans are counted later, per depth chunk
      const float hx = sqrtf(sxx * r2b);
      const float px0 = ceilf(__fsub_rn(__fsub_rn(F.mx, hx), 1.5f));
      const float px1 = floorf(__fadd_rn(__fadd_rn(F.mx, hx), 0.5f));
      if (!(py1 >= 0.f && py0 <= vp.height - 1 && px1 >= 0.f && px0 <= vp.width - 1)) {
        visible = false;
      } else {
        int ty0 = static_cast<int>(fmaxf(py0, 0.f)) / kTile;
        int ty1 = static_cast<int>(fminf(py1, (float)(vp.height - 1))) / kTile;
        if (vp.cols) {
          // 3-sigma coverage: the tiles that the square of half side
          // r = ceil(3 sqrt(lambda_max)) around the mean overlaps, decided in
          // FP32 with every step rounded to nearest (no contraction)
          const float mid = __fmul_rn(0.5f, __fadd_rn(sxx, syy));
          const float hd = __fmul_rn(0.5f, __fsub_rn(sxx, syy));
          const float lmax =
              __fadd_rn(mid, __fsqrt_rn(__fadd_rn(__fmul_rn(hd, hd), __fmul_rn(sxy, sxy))));
          const float r = ceilf(__fmul_rn(3.f, __fsqrt_rn(lmax)));
          const float inv = 1.f / kTile;  // a power of two: the scaling is exact
          const float cx0 = fmaxf(floorf(__fmul_rn(__fsub_rn(F.mx, r), inv)), 0.f);
          const float cx1 = fminf(__fsub_rn(ceilf(__fmul_rn(__fadd_rn(F.mx, r), inv)), 1.f),
                                  static_cast<float>(vp.tiles_x - 1));
          const float cy0 = fmaxf(floorf(__fmul_rn(__fsub_rn(F.my, r), inv)), 0.f);
          const float cy1 = fminf(__fsub_rn(ceilf(__fmul_rn(__fadd_rn(F.my, r), inv)), 1.f),
                                  static_cast<float>(vp.tiles_y - 1));
          if (cx0 <= cx1 && cy0 <= cy1) {
            ty0 = max(ty0, static_cast<int>(cy0));
            ty1 = min(ty1, static_cast<int>(cy1));
            col_clip = static_cast<uint32_t>(cx0) | (static_cast<uint32_t>(cx1) << 16);
          } else {
            ty1 = ty0 - 1;
          }
        }
        if (ty0 <= ty1) {
          F.rows = static_cast<uint32_t>(ty0) | (static_cast<uint32_t>(ty1) << 16);
          count = 1;
        } else {
          visible = false;
        }
      }
    }
    if (vp.cols) vp.cols[slot] = col_clip;
    if (visible) {  // records are read only through tile lists, which hold visible slots
      if (rec16)
        rec16[slot] = R16;
      else
        rec[slot] = R;
    }
    foot[slot] = F;
    cnt[slot] = visible ? count : 0u;
    const uint32_t k = visible ? depth_key(depth) : 0xFFFFFFFFu;
    if (visible) {
      kmin = min(kmin, k);
      kmax = max(kmax, k);
      ++n_vis;
    }
    key[slot] = k;
    val[slot] = static_cast<uint32_t>(slot);
    depth_lo[slot] = float_order_key(depth_l);
  }
  }
  if (key_range) {
    kmin = __reduce_min_sync(0xffffffffu, kmin);
    kmax = __reduce_max_sync(0xffffffffu, kmax);
    n_vis = __reduce_add_sync(0xffffffffu, n_vis);
    if ((threadIdx.x & 31) == 0 && kmin <= kmax) {
      atomicMin(&key_range[0], kmin);
      atomicMax(&key_range[1], kmax);
      atomicAdd(&key_range[2], n_vis);
    }
  }
}

// The radix sort orders by the float depth key hi, stably by slot, so equal
// keys already come in (view, index) order.  Only elements of one view that
// share a key need another order: by the low word of the float-pair depth,
// then by slot -- the order of the full-precision depth with ties by index
// that the compositing of Eq. 1 walks.  A thread acts only where such a
// same-view run starts; the runs are short and sorted by insertion.
__device__ __forceinline__ void fix_tie_run(int64_t k, int64_t n_total, const SlotView& view_of,
                                            uint32_t kk, const uint32_t* __restrict__ key,
                                            uint32_t* __restrict__ val,
                                            const uint32_t* __restrict__ depth_lo) {
  const uint32_t v0 = val[k];
  const uint32_t view = view_of(v0);
  if (view_of(val[k + 1]) != view) return;                       // no same-view tie here
  if (k > 0 && key[k - 1] == kk && view_of(val[k - 1]) == view) return;  // not the run's start
  int64_t e = k + 2;
  while (e < n_total && key[e] == kk && view_of(val[e]) == view) ++e;
  for (int64_t a = k + 1; a < e; ++a) {
    const uint32_t va = val[a];
    const uint64_t ka = (static_cast<uint64_t>(depth_lo[va]) << 32) | va;
    int64_t b = a - 1;
    while (b >= k) {
      const uint32_t vb = val[b];
      const uint64_t kb = (static_cast<uint64_t>(depth_lo[vb]) << 32) | vb;
      if (kb <= ka) break;
      val[b + 1] = vb;
      --b;
    }
    val[b + 1] = va;
  }
}

// Each thread screens four consecutive positions for the start of a run of
// equal keys within one view.  Equal keys of different views are common (a
// batch holds many views of the same depths), so the screen compares the
// views of neighbours from one 16-byte key load and one 16-byte value load
// (when both arrays are 16-byte aligned) before a run is walked.
__global__ void depth_tie_fix_kernel(int64_t n_total, int64_t n, const uint32_t* __restrict__ key,
                                     uint32_t* __restrict__ val,
                                     const uint32_t* __restrict__ depth_lo,
                                     const uint32_t* __restrict__ n_dev) {
  if (n_dev) n_total = min(n_total, static_cast<int64_t>(*n_dev));
  const int64_t k0 = 4 * (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x);
  if (k0 + 1 >= n_total) return;
  uint32_t t[5];  // keys k0 .. k0 + 4 (0xFFFFFFFF past the end: never a run)
  uint32_t w[5];  // their values (slots), where a key is present
  const bool full = k0 + 4 <= n_total &&
                    ((reinterpret_cast<uintptr_t>(key) | reinterpret_cast<uintptr_t>(val)) & 15u) == 0;
  if (full) {
    const uint4 q = *reinterpret_cast<const uint4*>(key + k0);
    t[0] = q.x;
    t[1] = q.y;
    t[2] = q.z;
    t[3] = q.w;
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) t[i] = k0 + i < n_total ? key[k0 + i] : 0xFFFFFFFFu;
  }
  t[4] = k0 + 4 < n_total ? key[k0 + 4] : 0xFFFFFFFFu;
  bool any = false;  // an equal neighbour somewhere among the four
#pragma unroll
  for (int i = 0; i < 4; ++i) any = any || (t[i] != 0xFFFFFFFFu && t[i + 1] == t[i]);
  if (!any) return;
  if (full) {
    const uint4 q = *reinterpret_cast<const uint4*>(val + k0);
    w[0] = q.x;
    w[1] = q.y;
    w[2] = q.z;
    w[3] = q.w;
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i] = k0 + i < n_total ? val[k0 + i] : 0u;
  }
  w[4] = k0 + 4 < n_total ? val[k0 + 4] : 0u;
  const SlotView view_of(n);
  uint32_t vw[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) vw[i] = view_of(w[i]);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (t[i] != 0xFFFFFFFFu && t[i + 1] == t[i] && vw[i + 1] == vw[i] && k0 + i + 1 < n_total)
      fix_tie_run(k0 + i, n_total, view_of, t[i], key, val, depth_lo);
  }
}

// ---------------------------------------------------------------------------
// Per depth chunk: count and emit the (tile, Gaussian) entries of sorted
// positions [p0, p0 + n_pos) on tiles not yet saturated.  A warp takes 32
// consecutive positions and spreads all of their tile rows over its lanes,
// one (Gaussian, row) per lane per round, so large footprints do not hold up
// small ones.  The owner of row r is found by a binary search over the
// lanes' inclusive row counts.
// ---------------------------------------------------------------------------

struct RowJob {
  uint32_t g;      // slot of the owning Gaussian (view * n + index)
  int row;         // tile row
  int owner;       // lane that holds the owning Gaussian
  bool ok;         // r < R
};

// Every lane of the warp must call this (it shuffles).
__device__ __forceinline__ RowJob row_job(int r, int R, uint32_t incl_rows, uint32_t g_lane,
                                          int ty0_lane) {
  // owner = number of lanes whose inclusive row count is <= r
  int lo = 0;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const uint32_t v = __shfl_sync(0xffffffffu, incl_rows, lo + s - 1);
    if (v <= static_cast<uint32_t>(r)) lo += s;
  }
  const int owner = min(lo, 31);
  const uint32_t pi = __shfl_sync(0xffffffffu, incl_rows, max(owner - 1, 0));
  const uint32_t g = __shfl_sync(0xffffffffu, g_lane, owner);
  const int ty0 = __shfl_sync(0xffffffffu, ty0_lane, owner);
  RowJob j;
  j.ok = r < R;
  j.g = g;
  j.owner = owner;
  j.row = ty0 + (r - static_cast<int>(owner > 0 ? pi : 0u));
  return j;
}

// Unsaturated tiles of one job's row: [a, b] (global ids) and their number.
__device__ __forceinline__ uint32_t job_free(const RowJob& jb, SlotView sv,
                                             const ViewParams* __restrict__ views,
                                             const Footprint* __restrict__ foot,
                                             const uint64_t* __restrict__ sat, int* a, int* b) {
  *a = 0;
  *b = -1;
  if (!jb.ok) return 0;
  const int v = static_cast<int>(sv(jb.g));
  const Footprint f = foot[jb.g];
  int tx0, tx1;
  if (!row_span(f, jb.row, views[v].width, &tx0, &tx1)) return 0;
  if (!clip_cols(views[v], jb.g, &tx0, &tx1)) return 0;
  const int base = views[v].tile_base + jb.row * views[v].tiles_x;
  *a = base + tx0;
  *b = base + tx1;
  return count_free(sat, *a, *b);
}

// The lane's sorted position j (if < n_pos): its slot g, first tile row ty0
// and number of tile rows -- none when every tile of its footprint's
// bounding box is already saturated, as is the case for most slots of later
// depth chunks.  Over the footprint x(dy) - mx stays within +-hx, hx^2 =
// syr (a^2 + b2); the box takes one more pixel on each side than the rows'
// spans, so it holds every span whatever their rounding.
__device__ __forceinline__ void lane_rows(int64_t j, int64_t n_pos, int64_t p0, SlotView sv,
                                          const ViewParams* __restrict__ views,
                                          const uint32_t* __restrict__ sorted_val,
                                          const Footprint* __restrict__ foot,
                                          const uint64_t* __restrict__ sat, uint32_t* g,
                                          int* ty0, uint32_t* nrows) {
  *g = 0;
  *ty0 = 0;
  *nrows = 0;
  if (j >= n_pos) return;
  const uint32_t gg = sorted_val[p0 + j];
  *g = gg;
  const Footprint f = foot[gg];
  int t0, t1;
  footprint_rows(f, &t0, &t1);
  *ty0 = t0;
  if (t1 < t0) return;
  const ViewParams& vp = views[sv(gg)];
  const float hx = sqrtf(f.syr * fmaf(f.a, f.a, f.b2));
  const float x0 = fmaxf(ceilf(f.mx - hx - 2.5f), 0.f);
  const float x1 = fminf(floorf(f.mx + hx + 1.5f), static_cast<float>(vp.width - 1));
  if (!(x0 <= x1)) return;
  int c0 = static_cast<int>(x0) / kTile, c1 = static_cast<int>(x1) / kTile;
  if (vp.cols) {  // 3-sigma coverage
    const uint32_t c = vp.cols[gg];
    c0 = max(c0, static_cast<int>(c & 0xFFFFu));
    c1 = min(c1, static_cast<int>(c >> 16));
    if (c0 > c1) return;
  }
  if (vp.free_tab) {
    if (free_in_box(vp, t0, t1, c0, c1)) *nrows = static_cast<uint32_t>(t1 - t0 + 1);
    return;
  }
  for (int ty = t0; ty <= t1; ++ty) {
    const int base = vp.tile_base + ty * vp.tiles_x;
    if (any_free(sat, base + c0, base + c1)) {
      *nrows = static_cast<uint32_t>(t1 - t0 + 1);
      return;
    }
  }
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

__global__ void __launch_bounds__(256) chunk_count_kernel(
    int64_t p0, int64_t n_pos, SlotView sv, const ViewParams* __restrict__ views,
    const uint32_t* __restrict__ sorted_val,
    const Footprint* __restrict__ foot, const uint64_t* __restrict__ sat,
    uint32_t* __restrict__ out_cnt) {

  __shared__ uint32_t s_cnt[8][32];
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t g, nrows;
  int ty0;
  lane_rows(j, n_pos, p0, sv, views, sorted_val, foot, sat, &g, &ty0, &nrows);
  const uint32_t incl = warp_incl_scan(nrows, lane);
  const int R = static_cast<int>(__shfl_sync(0xffffffffu, incl, 31));
  s_cnt[warp][lane] = 0;
  __syncwarp();
  for (int r0 = 0; r0 < R; r0 += 32) {
    const RowJob jb = row_job(r0 + lane, R, incl, g, ty0);
    int a, b;
    const uint32_t fr = job_free(jb, sv, views, foot, sat, &a, &b);
    if (jb.ok && fr) atomicAdd(&s_cnt[warp][jb.owner], fr);
  }
  __syncwarp();
  if (j < n_pos) out_cnt[j] = s_cnt[warp][lane];
}

// Writes (tile, g) for every unsaturated tile id in [a, b], from position o,
// never at or past `end`; returns the next position.
__device__ __forceinline__ uint32_t emit_free(const uint64_t* __restrict__ sat, int a, int b,
                                              uint32_t g, uint32_t* __restrict__ out_key,
                                              uint32_t* __restrict__ out_val, uint32_t o,
                                              uint32_t end) {
  const int wa = a >> 6, wb = b >> 6;
  for (int w = wa; w <= wb; ++w) {
    uint64_t m = ~0ull;
    if (w == wa) m &= ~0ull << (a & 63);
    if (w == wb) m &= ~0ull >> (63 - (b & 63));
    uint64_t bits = ~sat[w] & m;
    while (bits && o < end) {
      const int bit = __ffsll(static_cast<long long>(bits)) - 1;
      bits &= bits - 1;
      out_key[o] = static_cast<uint32_t>(w * 64 + bit);
      out_val[o] = g;
      ++o;
    }
  }
  return o;
}

// Writes the list entries of sorted positions [p0, p0 + n_pos) in depth
// order: the warp's 32 Gaussians own the contiguous output range starting at
// offsets[first] (the exclusive scan of chunk_cnt); row r's entries start at
// that base plus the free tiles of all earlier rows of the warp.
__global__ void __launch_bounds__(256) emit_kernel(
    int64_t p0, int64_t n_pos, SlotView sv, const ViewParams* __restrict__ views,
    const uint32_t* __restrict__ sorted_val, const uint32_t* __restrict__ offsets,
    const uint32_t* __restrict__ chunk_cnt,
    const Footprint* __restrict__ foot, const uint64_t* __restrict__ sat,
    uint32_t* __restrict__ out_key, uint32_t* __restrict__ out_val,
    unsigned long long* __restrict__ counters) {

  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  uint32_t g, nrows;
  int ty0;
  lane_rows(j, n_pos, p0, sv, views, sorted_val, foot, sat, &g, &ty0, &nrows);
  const uint32_t incl = warp_incl_scan(nrows, lane);
  const int R = static_cast<int>(__shfl_sync(0xffffffffu, incl, 31));
  // the warp's output range [wbeg, wend)
  const int64_t jw = j - lane;  // first position of the warp
  const int64_t jl = min(jw + 31, n_pos - 1);
  uint32_t wbeg = 0, wend = 0;
  if (lane == 0 && jw < n_pos) {
    wbeg = offsets[jw];
    wend = offsets[jl] + chunk_cnt[jl];
  }
  wbeg = __shfl_sync(0xffffffffu, wbeg, 0);
  wend = __shfl_sync(0xffffffffu, wend, 0);
  uint32_t carry = 0;
  for (int r0 = 0; r0 < R; r0 += 32) {
    const RowJob jb = row_job(r0 + lane, R, incl, g, ty0);
    int a, b;
    const uint32_t fr = job_free(jb, sv, views, foot, sat, &a, &b);
    const uint32_t sc = warp_incl_scan(fr, lane);
    const uint32_t o = wbeg + carry + sc - fr;
    if (fr) emit_free(sat, a, b, jb.g, out_key, out_val, o, min(o + fr, wend));
    carry += __shfl_sync(0xffffffffu, sc, 31);
  }
  if (lane == 0 && jw < n_pos && wbeg + carry != wend) atomicAdd(&counters[kBinningMismatch], 1ull);
}

// Count, offset and emit in one pass.  Blocks take virtual ids in launch
// order (a ticket), so every block's predecessors are running or done.  A
// block (4 warps: a short wait at its barriers) counts its 128 positions'
// entries, publishes the count, then adds
// up its predecessors' published words (decoupled look-back: a word is
// either a block's own count or the inclusive prefix up to it; the walk
// stops at the first prefix), publishes its own prefix and emits from its
// offset.  No block waits on a later one.  Entries at or past `capacity`
// are not written; *total receives the entry count either way, so the
// caller can grow the buffer and run the chunk again.  A look-back that
// polls a predecessor's word more than spin_limit times gives up, counts a
// time-out (kLookbackTimeout) and uses 0.
constexpr unsigned long long kLbCount = 1ull << 32;   // word holds the block's own count
constexpr unsigned long long kLbPrefix = 2ull << 32;  // word holds the inclusive prefix

template <bool kDeviceRange>
__global__ void __launch_bounds__(128, 12) bin_fused_kernel(
    int64_t p0, int64_t n_pos, SlotView sv, const ViewParams* __restrict__ views,
    const uint32_t* __restrict__ sorted_val,
    const Footprint* __restrict__ foot, const uint64_t* __restrict__ sat,
    uint32_t* __restrict__ out_key, uint32_t* __restrict__ out_val, uint32_t capacity,
    unsigned long long* __restrict__ status, uint32_t* __restrict__ ticket,
    uint32_t* __restrict__ total, unsigned long long* __restrict__ counters, int spin_limit,
    const int64_t* __restrict__ range_dev) {

  __shared__ uint32_t s_vb, s_boff;
  if constexpr (kDeviceRange) {  // the chunk's positions [range_dev[0], range_dev[1])
    p0 = range_dev[0];
    n_pos = range_dev[1] - range_dev[0];
  }
  __shared__ uint32_t s_wtot[4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_vb = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t vb = s_vb;
  const int64_t j = static_cast<int64_t>(vb) * blockDim.x + threadIdx.x;
  uint32_t g, nrows;
  int ty0;
  lane_rows(j, n_pos, p0, sv, views, sorted_val, foot, sat, &g, &ty0, &nrows);
  const uint32_t incl = warp_incl_scan(nrows, lane);
  const int R = static_cast<int>(__shfl_sync(0xffffffffu, incl, 31));
  // count; the first kStash rounds' jobs are kept in registers for the emission
  constexpr int kStash = 3;
  int st_a[kStash], st_b[kStash];
  uint32_t st_fr[kStash], st_g[kStash];
  uint32_t wtot = 0;
#pragma unroll
  for (int k = 0; k < kStash; ++k) {
    st_a[k] = 0;
    st_b[k] = -1;
    st_fr[k] = 0;
    st_g[k] = 0;
    if (32 * k < R) {  // R is the same for the whole warp
      const RowJob jb = row_job(32 * k + lane, R, incl, g, ty0);
      const uint32_t fr = job_free(jb, sv, views, foot, sat, &st_a[k], &st_b[k]);
      st_fr[k] = fr;
      st_g[k] = jb.g;
      uint32_t sum = fr;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      wtot += sum;
    }
  }
  for (int r0 = 32 * kStash; r0 < R; r0 += 32) {
    const RowJob jb = row_job(r0 + lane, R, incl, g, ty0);
    int a, b;
    uint32_t fr = job_free(jb, sv, views, foot, sat, &a, &b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fr += __shfl_xor_sync(0xffffffffu, fr, o);
    wtot += fr;
  }
  if (lane == 0) s_wtot[warp] = wtot;
  __syncthreads();
  // offset of the block: decoupled look-back over the predecessors, 32 at a
  // time (lane l reads predecessor vb - 1 - l)
  if (warp == 0) {
    uint32_t btot = 0;
    for (int w = 0; w < 4; ++w) btot += s_wtot[w];
    if (lane == 0) atomicExch(&status[vb], (vb == 0 ? kLbPrefix : kLbCount) | btot);
    volatile unsigned long long* vs = status;
    uint32_t excl = 0;
    for (int64_t base = static_cast<int64_t>(vb) - 1; base >= 0; base -= 32) {
      const int64_t q = base - lane;
      unsigned long long word = kLbPrefix;  // before block 0: an empty prefix
      if (q >= 0) {
        word = vs[q];
        int spins = 0;
        while ((word >> 32) == 0ull && spins < spin_limit) {
          __nanosleep(32);
          word = vs[q];
          ++spins;
        }
        if ((word >> 32) == 0ull) {  // gave up: report, count it as an empty prefix
          atomicAdd(&counters[kLookbackTimeout], 1ull);
          word = kLbPrefix;
        }
      }
      const uint32_t pre = __ballot_sync(0xffffffffu, (word & ~0xFFFFFFFFull) == kLbPrefix);
      const int first = pre ? __ffs(pre) - 1 : 31;  // nearest predecessor holding a prefix
      uint32_t v = lane <= first ? static_cast<uint32_t>(word & 0xFFFFFFFFull) : 0u;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      excl += v;
      if (pre) break;
    }
    if (lane == 0) {
      if (vb > 0) atomicExch(&status[vb], kLbPrefix | (excl + btot));
      s_boff = excl;
      if (vb == gridDim.x - 1) *total = excl + btot;
    }
  }
  __syncthreads();
  uint32_t wbeg = s_boff;
  for (int w = 0; w < warp; ++w) wbeg += s_wtot[w];
  const uint32_t wend = wbeg + wtot;
  // emit, in the same (Gaussian, row) order as the count
  uint32_t carry = 0;
#pragma unroll
  for (int k = 0; k < kStash; ++k) {
    if (32 * k < R) {
      const uint32_t fr = st_fr[k];
      const uint32_t sc = warp_incl_scan(fr, lane);
      const uint32_t o = wbeg + carry + sc - fr;
      if (fr && o < capacity)
        emit_free(sat, st_a[k], st_b[k], st_g[k], out_key, out_val, o,
                  min(min(o + fr, wend), capacity));
      carry += __shfl_sync(0xffffffffu, sc, 31);
    }
  }
  for (int r0 = 32 * kStash; r0 < R; r0 += 32) {
    const RowJob jb = row_job(r0 + lane, R, incl, g, ty0);
    int a, b;
    const uint32_t fr = job_free(jb, sv, views, foot, sat, &a, &b);
    const uint32_t sc = warp_incl_scan(fr, lane);
    const uint32_t o = wbeg + carry + sc - fr;
    if (fr && o < capacity)
      emit_free(sat, a, b, jb.g, out_key, out_val, o, min(min(o + fr, wend), capacity));
    carry += __shfl_sync(0xffffffffu, sc, 31);
  }
  if (lane == 0 && wbeg + carry != wend) atomicAdd(&counters[kBinningMismatch], 1ull);
}

// Per view of the batch (one block each), the 2-D prefix sums of its
// unsaturated tiles: free_tab[r * (tiles_x + 1) + c] = unsaturated tiles in
// rows < r and columns < c (row 0 and column 0 are zero).  Running sums
// along each row, then down each column.
__global__ void __launch_bounds__(256) free_table_kernel(const ViewParams* __restrict__ views,
                                                         const uint64_t* __restrict__ sat) {
  const ViewParams& vp = views[blockIdx.x];
  uint32_t* tab = vp.free_tab;
  if (!tab) return;
  const int tx = vp.tiles_x, ty = vp.tiles_y, w1 = tx + 1;
  for (int c = threadIdx.x; c < w1; c += blockDim.x) tab[c] = 0u;
  for (int r = threadIdx.x; r < ty; r += blockDim.x) {
    const int g0 = vp.tile_base + r * tx;
    uint32_t* row = tab + static_cast<int64_t>(r + 1) * w1;
    uint32_t run = 0;
    row[0] = 0u;
    for (int c = 0; c < tx; ++c) {
      const int g = g0 + c;
      run += static_cast<uint32_t>(((sat[g >> 6] >> (g & 63)) & 1ull) == 0ull);
      row[c + 1] = run;
    }
  }
  __syncthreads();
  for (int c = threadIdx.x + 1; c < w1; c += blockDim.x) {
    uint32_t acc = 0;
    for (int r = 1; r <= ty; ++r) {
      uint32_t* e = tab + static_cast<int64_t>(r) * w1 + c;
      acc += *e;
      *e = acc;
    }
  }
}

// [start, end) of every tile's run in the tile-sorted list.  Each thread
// takes four consecutive entries (one 16-byte load when the list is 16-byte
// aligned, as the library's buffers are) and the entries on either side.
__global__ void ranges_kernel(int64_t n_entries, const uint32_t* __restrict__ key,
                              uint2* __restrict__ ranges, const uint32_t* __restrict__ n_dev) {
  if (n_dev) n_entries = min(n_entries, static_cast<int64_t>(*n_dev));
  const int64_t k0 = 4 * (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x);
  if (k0 >= n_entries) return;
  uint32_t t[6];  // entries k0 - 1 .. k0 + 4 (0xFFFFFFFF outside the list)
  t[0] = k0 > 0 ? key[k0 - 1] : 0xFFFFFFFFu;
  if (k0 + 4 <= n_entries && (reinterpret_cast<uintptr_t>(key) & 15u) == 0) {
    const uint4 q = *reinterpret_cast<const uint4*>(key + k0);
    t[1] = q.x;
    t[2] = q.y;
    t[3] = q.z;
    t[4] = q.w;
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) t[1 + i] = k0 + i < n_entries ? key[k0 + i] : 0xFFFFFFFFu;
  }
  t[5] = k0 + 4 < n_entries ? key[k0 + 4] : 0xFFFFFFFFu;
#pragma unroll
  for (int i = 1; i <= 4; ++i) {
    const int64_t k = k0 + i - 1;
    if (k >= n_entries) break;
    if (t[i - 1] != t[i]) ranges[t[i]].x = static_cast<uint32_t>(k);
    if (t[i + 1] != t[i]) ranges[t[i]].y = static_cast<uint32_t>(k + 1);
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

cudaError_t launch_scene_prep(int64_t n, const float* mean, const void* quat, int quat_dtype,
                              const void* scale, int scale_dtype, const void* opacity,
                              int opacity_dtype, float4* pos_op, float4* cov, unsigned int* err,
                              cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (n + threads - 1) / threads;
  scene_prep_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(
      n, mean, quat, quat_dtype, scale, scale_dtype, opacity, opacity_dtype, pos_op, cov, err);
  return cudaGetLastError();
}

cudaError_t launch_project(int64_t n, int n_views, const ViewParams* views, const float4* pos_op,
                           const float4* cov, ProjRecord* rec, CompactRecord* rec16,
                           Footprint* foot, uint32_t* cnt, uint32_t* key, uint32_t* val,
                           uint32_t* depth_lo, uint32_t* key_range, cudaStream_t stream) {
  if (n == 0 || n_views == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (n + threads - 1) / threads;
  // the reduced-precision form takes the FP32 projection
  if (rec16)
    project_kernel<true><<<static_cast<unsigned>(blocks), threads, 0, stream>>>(
        n, n_views, views, pos_op, cov, rec, rec16, foot, cnt, key, val, depth_lo, key_range);
  else
    project_kernel<false><<<static_cast<unsigned>(blocks), threads, 0, stream>>>(
        n, n_views, views, pos_op, cov, rec, rec16, foot, cnt, key, val, depth_lo, key_range);
  return cudaGetLastError();
}

cudaError_t launch_depth_tie_fix(int64_t n_total, int64_t n, const uint32_t* key, uint32_t* val,
                                 const uint32_t* depth_lo, cudaStream_t stream,
                                 const uint32_t* n_dev) {
  if (n_total < 2) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = ((n_total + 3) / 4 + threads - 1) / threads;
  depth_tie_fix_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(n_total, n, key, val,
                                                                              depth_lo, n_dev);
  return cudaGetLastError();
}

cudaError_t launch_chunk_count(int64_t p0, int64_t n_pos, int64_t n, const ViewParams* views,
                               const uint32_t* sorted_val,
                               const Footprint* foot, const uint64_t* sat, uint32_t* out_cnt,
                               cudaStream_t stream) {
  if (n_pos == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (n_pos + threads - 1) / threads;
  chunk_count_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(
      p0, n_pos, SlotView(n > 0 ? n : 1), views, sorted_val, foot, sat, out_cnt);
  return cudaGetLastError();
}

cudaError_t launch_emit(int64_t p0, int64_t n_pos, int64_t n, const ViewParams* views,
                        const uint32_t* sorted_val, const uint32_t* offsets,
                        const uint32_t* chunk_cnt, const Footprint* foot,
                        const uint64_t* sat, uint32_t* out_key, uint32_t* out_val,
                        unsigned long long* counters, cudaStream_t stream) {
  if (n_pos == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (n_pos + threads - 1) / threads;
  emit_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(
      p0, n_pos, SlotView(n > 0 ? n : 1), views, sorted_val, offsets, chunk_cnt, foot, sat, out_key, out_val,
      counters);
  return cudaGetLastError();
}

cudaError_t launch_bin_fused(int64_t p0, int64_t n_pos, int64_t n, const ViewParams* views,
                             const uint32_t* sorted_val,
                             const Footprint* foot, const uint64_t* sat, uint32_t* out_key,
                             uint32_t* out_val, uint32_t capacity, void* lookback,
                             uint32_t* total, unsigned long long* counters, cudaStream_t stream,
                             const int64_t* range_dev) {
  if (n_pos <= 0) return cudaMemsetAsync(total, 0, sizeof(uint32_t), stream);
  const int threads = 128;
  const int64_t blocks = (n_pos + threads - 1) / threads;
  uint32_t* ticket = static_cast<uint32_t*>(lookback);
  unsigned long long* status = reinterpret_cast<unsigned long long*>(
      static_cast<char*>(lookback) + 256);
  cudaError_t e = cudaMemsetAsync(lookback, 0, 256 + static_cast<size_t>(blocks) * 8, stream);
  if (e != cudaSuccess) return e;
  if (range_dev)
    bin_fused_kernel<true><<<static_cast<unsigned>(blocks), threads, 0, stream>>>(
        p0, n_pos, SlotView(n > 0 ? n : 1), views, sorted_val, foot, sat, out_key, out_val, capacity, status, ticket,
        total, counters, kLookbackSpinLimit, range_dev);
  else
    bin_fused_kernel<false><<<static_cast<unsigned>(blocks), threads, 0, stream>>>(
        p0, n_pos, SlotView(n > 0 ? n : 1), views, sorted_val, foot, sat, out_key, out_val, capacity, status, ticket,
        total, counters, kLookbackSpinLimit, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_lookback_probe(void* lookback, uint32_t* total, unsigned long long* counters,
                                  const ViewParams* views, const uint32_t* sorted_val,
                                  const Footprint* foot, const uint64_t* sat, uint32_t* out_key,
                                  uint32_t* out_val, int spin_limit, cudaStream_t stream) {
  // one block whose ticket comes out as 1: its predecessor (block 0) never
  // runs, so its status word stays empty and the look-back must give up
  uint32_t* ticket = static_cast<uint32_t*>(lookback);
  unsigned long long* status = reinterpret_cast<unsigned long long*>(
      static_cast<char*>(lookback) + 256);
  cudaError_t e = cudaMemsetAsync(lookback, 0, 256 + 16, stream);
  if (e != cudaSuccess) return e;
  const uint32_t one = 1u;
  e = cudaMemcpyAsync(ticket, &one, sizeof(one), cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return e;
  bin_fused_kernel<false><<<1, 128, 0, stream>>>(0, 1, SlotView(1), views, sorted_val, foot, sat, out_key,
                                                 out_val, 0u, status, ticket, total, counters,
                                                 spin_limit, nullptr);
  return cudaGetLastError();
}

size_t bin_fused_temp_bytes(int64_t n_pos) {
  return 256 + static_cast<size_t>((n_pos + 127) / 128) * 8;
}

cudaError_t launch_free_tables(const ViewParams* views, int n_views, const uint64_t* sat,
                               cudaStream_t stream) {
  if (n_views <= 0) return cudaSuccess;
  free_table_kernel<<<static_cast<unsigned>(n_views), 256, 0, stream>>>(views, sat);
  return cudaGetLastError();
}

cudaError_t launch_ranges(int64_t n_entries, const uint32_t* key, uint2* ranges,
                          cudaStream_t stream, const uint32_t* n_dev) {
  if (n_entries == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = ((n_entries + 3) / 4 + threads - 1) / threads;
  ranges_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(n_entries, key, ranges,
                                                                       n_dev);
  return cudaGetLastError();
}

}  // namespace fs
