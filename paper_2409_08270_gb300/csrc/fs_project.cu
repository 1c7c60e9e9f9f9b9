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
// diag(lambda1, lambda2)^-1/2 [e e']^T as a float pair (hi, lo) and
// c = -W_ws m2D, so alpha = o 2^-|W_ws (p - m2D)|^2.  Carrying the eigenvectors
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
// binning geometry
// ---------------------------------------------------------------------------

// Inflated r2 used for binning (conservative against FP32 rounding).  The
// binning arithmetic uses explicit round-to-nearest intrinsics so that the
// count (projection kernel) and the emission (emit kernel) evaluate it
// bit-identically whatever the compiler contracts elsewhere.
__device__ __forceinline__ float binning_r2(float r2) {
  return __fadd_rn(__fmul_rn(r2, 1.001f), 1e-3f);
}

__device__ __forceinline__ void footprint_rows(const Footprint& f, int* ty0, int* ty1) {
  *ty0 = static_cast<int>(f.rows & 0xFFFFu);
  *ty1 = static_cast<int>(f.rows >> 16);
}

// Tiles [tx0, tx1] of tile row ty touched by the footprint (false if none).
// The band of pixel-centre rows of the tile, widened by one pixel, is
// intersected with the ellipse; its x-extent over the band comes from the
// boundary x_R(dy) = (sxy dy + sqrt(det (syy r2 - dy^2))) / syy, which is
// concave (maximal at the ellipse's rightmost point, dy* = sxy sqrt(r2/sxx),
// clamped to the band), and the mirror image on the left.
__device__ __forceinline__ bool row_span(const Footprint& f, int ty, int width, int* tx0,
                                         int* tx1) {
  const float r2 = binning_r2(f.r2);
  const float yt = static_cast<float>(ty * kTile);
  const float y0 = __fsub_rn(__fadd_rn(yt, -0.5f), f.my);   // band widened by one pixel
  const float y1 = __fsub_rn(__fadd_rn(yt, 16.5f), f.my);
  const float hy = __fsqrt_rn(__fmul_rn(f.syy, r2));
  const float u0 = fmaxf(y0, -hy), u1 = fminf(y1, hy);
  if (!(u0 <= u1)) return false;
  const float dys = __fmul_rn(f.sxy, __fsqrt_rn(__fdiv_rn(r2, f.sxx)));
  const float dr = fminf(fmaxf(dys, u0), u1), dl = fminf(fmaxf(-dys, u0), u1);
  const float syr = __fmul_rn(f.syy, r2);
  const float sr = __fsqrt_rn(__fmul_rn(f.det, fmaxf(0.f, __fsub_rn(syr, __fmul_rn(dr, dr)))));
  const float sl = __fsqrt_rn(__fmul_rn(f.det, fmaxf(0.f, __fsub_rn(syr, __fmul_rn(dl, dl)))));
  const float xr = __fadd_rn(f.mx, __fdiv_rn(__fadd_rn(__fmul_rn(f.sxy, dr), sr), f.syy));
  const float xl = __fadd_rn(f.mx, __fdiv_rn(__fsub_rn(__fmul_rn(f.sxy, dl), sl), f.syy));
  float px0 = ceilf(__fsub_rn(xl, 1.5f)), px1 = floorf(__fadd_rn(xr, 0.5f));
  px0 = fmaxf(px0, 0.f);
  px1 = fminf(px1, static_cast<float>(width - 1));
  if (!(px0 <= px1)) return false;
  *tx0 = static_cast<int>(px0) / kTile;
  *tx1 = static_cast<int>(px1) / kTile;
  return true;
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

// One thread per Gaussian; it projects the Gaussian into every view of the
// batch so the scene is read once per batch.
__global__ void __launch_bounds__(256) project_kernel(
    int64_t n, int n_views, const ViewParams* __restrict__ views_g,
    const float4* __restrict__ pos_op, const float4* __restrict__ cov3,
    ProjRecord* __restrict__ rec, Footprint* __restrict__ foot, uint32_t* __restrict__ cnt,
    uint32_t* __restrict__ key, uint32_t* __restrict__ val, uint32_t* __restrict__ depth_lo) {
  __shared__ ViewParams views[kMaxViewsPerBatch];
  for (int k = threadIdx.x; k < n_views * (int)(sizeof(ViewParams) / 4); k += blockDim.x)
    reinterpret_cast<uint32_t*>(views)[k] = reinterpret_cast<const uint32_t*>(views_g)[k];
  __syncthreads();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;

  const float4 po = pos_op[i];
  const float4 ca = cov3[3 * i], cb = cov3[3 * i + 1], cc = cov3[3 * i + 2];
  const f2 S00 = {ca.x, ca.y}, S01 = {ca.z, ca.w}, S02 = {cb.x, cb.y};
  const f2 S11 = {cb.z, cb.w}, S12 = {cc.x, cc.y}, S22 = {cc.z, cc.w};
  const f2 S[3][3] = {{S00, S01, S02}, {S01, S11, S12}, {S02, S12, S22}};
  const float o = po.w;
  const bool opaque_enough = o >= kAlphaMin;
  const float r2 = opaque_enough ? fmaxf(2.f * logf(255.f * o), 0.f) : 0.f;

  for (int v = 0; v < n_views; ++v) {
    const ViewParams& vp = views[v];
    const int64_t slot = static_cast<int64_t>(v) * n + i;
    const f2 tx = f2_dot3_add(vp.R_hi + 0, vp.R_lo + 0, po.x, po.y, po.z, vp.t_hi[0], vp.t_lo[0]);
    const f2 ty = f2_dot3_add(vp.R_hi + 3, vp.R_lo + 3, po.x, po.y, po.z, vp.t_hi[1], vp.t_lo[1]);
    const f2 tz = f2_dot3_add(vp.R_hi + 6, vp.R_lo + 6, po.x, po.y, po.z, vp.t_hi[2], vp.t_lo[2]);
    bool visible = opaque_enough && f2_greater(tz, vp.near_hi, vp.near_lo);
    uint32_t count = 0;
    float depth = 0.f, depth_l = 0.f;
    ProjRecord R;
    R.w_hi = R.w_lo = R.c = make_float4(0.f, 0.f, 0.f, 0.f);
    R.misc = make_float4(o, 0.f, 0.f, 0.f);
    Footprint F;
    F.mx = F.my = F.sxy = F.det = F.r2 = 0.f;
    F.sxx = F.syy = 1.f;
    F.rows = 0;
    if (visible) {
      const f2 ux = f2_div(tx, tz), uy = f2_div(ty, tz);
      const f2 fx = {vp.fx_hi, vp.fx_lo}, fy = {vp.fy_hi, vp.fy_lo};
      const f2 mx = f2_add(f2_mul(fx, ux), f2{vp.cx_hi, vp.cx_lo});
      const f2 my = f2_add(f2_mul(fy, uy), f2{vp.cy_hi, vp.cy_lo});
      depth = tz.hi;
      depth_l = tz.lo;
      const f2 iz = f2_div(f2_from(1.f), tz);
      const f2 j0 = f2_mul(fx, iz), j1 = f2_mul(fy, iz);
      const f2 uxc = f2_clamp(ux, vp.limx_hi, vp.limx_lo);
      const f2 uyc = f2_clamp(uy, vp.limy_hi, vp.limy_lo);
      // rows of J W: T0 = fx/z (W0 - ux W2), T1 = fy/z (W1 - uy W2)
      f2 T0[3], T1[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const f2 w0 = {vp.R_hi[k], vp.R_lo[k]}, w1 = {vp.R_hi[3 + k], vp.R_lo[3 + k]};
        const f2 w2 = {vp.R_hi[6 + k], vp.R_lo[6 + k]};
        T0[k] = f2_mul(j0, f2_sub(w0, f2_mul(uxc, w2)));
        T1[k] = f2_mul(j1, f2_sub(w1, f2_mul(uyc, w2)));
      }
      // Sigma' = T Sigma3D T^T
      f2 a = f2_from(0.f), b = f2_from(0.f), c = f2_from(0.f);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        f2 m0 = f2_mul(T0[0], S[0][j]), m1 = f2_mul(T1[0], S[0][j]);
        m0 = f2_fma(T0[1], S[1][j], m0);
        m1 = f2_fma(T1[1], S[1][j], m1);
        m0 = f2_fma(T0[2], S[2][j], m0);
        m1 = f2_fma(T1[2], S[2][j], m1);
        a = f2_fma(m0, T0[j], a);
        b = f2_fma(m0, T1[j], b);
        c = f2_fma(m1, T1[j], c);
      }
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
        ex = f2_div(ex, en);
        ey = f2_div(ey, en);
      } else {
        ex = f2_from(1.f);
        ey = f2_from(0.f);
      }
      // axis scales only need FP32 accuracy
      const float k1 = sqrtf(static_cast<float>(kHalfLog2e) / lam1.hi);
      const float k2 = sqrtf(static_cast<float>(kHalfLog2e) / lam2.hi);
      const f2 W00 = f2_mul_f(ex, k1), W01 = f2_mul_f(ey, k1);
      const f2 W10 = f2_mul_f(f2_neg(ey), k2), W11 = f2_mul_f(ex, k2);
      const f2 c0 = f2_neg(f2_add(f2_mul(W00, mx), f2_mul(W01, my)));
      const f2 c1 = f2_neg(f2_add(f2_mul(W10, mx), f2_mul(W11, my)));
      R.w_hi = make_float4(W00.hi, W01.hi, W10.hi, W11.hi);
      R.w_lo = make_float4(W00.lo, W01.lo, W10.lo, W11.lo);
      R.c = make_float4(c0.hi, c1.hi, c0.lo, c1.lo);
      // binning footprint
      F.mx = mx.hi;
      F.my = my.hi;
      F.sxx = a.hi;
      F.sxy = b.hi;
      F.syy = c.hi;
      F.det = det.hi;
      F.r2 = r2;
      const float hy = __fsqrt_rn(__fmul_rn(F.syy, binning_r2(r2)));
      const float py0 = ceilf(__fsub_rn(__fsub_rn(F.my, hy), 1.5f));
      const float py1 = floorf(__fadd_rn(__fadd_rn(F.my, hy), 0.5f));
      if (!(py1 >= 0.f && py0 <= vp.height - 1)) {
        visible = false;
      } else {
        const int ty0 = static_cast<int>(fmaxf(py0, 0.f)) / kTile;
        const int ty1 = static_cast<int>(fminf(py1, (float)(vp.height - 1))) / kTile;
        F.rows = static_cast<uint32_t>(ty0) | (static_cast<uint32_t>(ty1) << 16);
        for (int t = ty0; t <= ty1; ++t) {
          int a0, a1;
          if (row_span(F, t, vp.width, &a0, &a1)) count += static_cast<uint32_t>(a1 - a0 + 1);
        }
        if (count == 0) visible = false;
      }
    }
    rec[slot] = R;
    foot[slot] = F;
    cnt[slot] = visible ? count : 0u;
    key[slot] = visible ? depth_key(depth) : 0xFFFFFFFFu;
    val[slot] = static_cast<uint32_t>(slot);
    depth_lo[slot] = float_order_key(depth_l);
  }
}

// The radix sort orders by the float depth key hi, stably by slot.  Runs of
// equal hi are re-ordered here by the low word of the float-pair depth (and
// then by slot), so the order is that of the full-precision depth with ties
// by index -- the order the compositing of Eq. 1 walks.  Runs are short; one
// thread sorts each run by insertion.
__global__ void depth_tie_fix_kernel(int64_t n, const uint32_t* __restrict__ key,
                                     uint32_t* __restrict__ val,
                                     const uint32_t* __restrict__ depth_lo) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k + 1 >= n) return;
  const uint32_t kk = key[k];
  if (kk == 0xFFFFFFFFu || key[k + 1] != kk) return;
  if (k > 0 && key[k - 1] == kk) return;  // not the start of the run
  int64_t e = k + 2;
  while (e < n && key[e] == kk) ++e;
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

// Number of list entries of sorted positions [p0, p0 + n_pos) that fall on
// tiles not yet saturated (sat[t] != 0: every pixel of tile t has stopped).
__global__ void __launch_bounds__(256) chunk_count_kernel(
    int64_t p0, int64_t n_pos, int64_t n, const ViewParams* __restrict__ views,
    const uint32_t* __restrict__ sorted_val, const uint32_t* __restrict__ cnt,
    const Footprint* __restrict__ foot, const uint8_t* __restrict__ sat,
    uint32_t* __restrict__ out_cnt) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n_pos) return;
  const uint32_t g = sorted_val[p0 + j];
  uint32_t c = 0;
  if (cnt[g] > 0) {
    const int v = static_cast<int>(g / n);
    const Footprint f = foot[g];
    const int tiles_x = views[v].tiles_x, width = views[v].width;
    const uint8_t* st = sat + views[v].tile_base;
    int ty0, ty1;
    footprint_rows(f, &ty0, &ty1);
    for (int ty = ty0; ty <= ty1; ++ty) {
      int tx0, tx1;
      if (!row_span(f, ty, width, &tx0, &tx1)) continue;
      for (int tx = tx0; tx <= tx1; ++tx) c += st[ty * tiles_x + tx] ? 0u : 1u;
    }
  }
  out_cnt[j] = c;
}

// ---------------------------------------------------------------------------
// emission of (tile, Gaussian) list entries in depth order
// ---------------------------------------------------------------------------

constexpr uint32_t kBigEmit = 64;  // longer lists are written by a whole warp

// Writes the list entries of sorted positions [p0, p0 + n_pos): for each
// Gaussian, in depth order, the (tile, Gaussian) pairs of its non-saturated
// tiles, at offsets[j] (the exclusive scan of chunk_cnt).
__global__ void __launch_bounds__(256) emit_kernel(
    int64_t p0, int64_t n_pos, int64_t n, const ViewParams* __restrict__ views,
    const uint32_t* __restrict__ sorted_val, const uint32_t* __restrict__ offsets,
    const uint32_t* __restrict__ chunk_cnt, const Footprint* __restrict__ foot,
    const uint8_t* __restrict__ sat, uint32_t* __restrict__ out_key,
    uint32_t* __restrict__ out_val, unsigned long long* __restrict__ counters) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  uint32_t g = 0, c = 0, off = 0;
  if (j < n_pos) {
    g = sorted_val[p0 + j];
    c = chunk_cnt[j];
    off = offsets[j];
  }
  const bool big = c > kBigEmit;
  if (c > 0 && !big) {
    const int v = static_cast<int>(g / n);
    const Footprint f = foot[g];
    const int tiles_x = views[v].tiles_x, width = views[v].width;
    const uint32_t base = static_cast<uint32_t>(views[v].tile_base);
    const uint32_t end = off + c;  // never write past this Gaussian's allotment
    const uint8_t* st = sat + base;
    uint32_t o = off;
    int ty0, ty1;
    footprint_rows(f, &ty0, &ty1);
    for (int ty = ty0; ty <= ty1; ++ty) {
      int tx0, tx1;
      if (!row_span(f, ty, width, &tx0, &tx1)) continue;
      for (int tx = tx0; tx <= tx1 && o < end; ++tx) {
        const int t = ty * tiles_x + tx;
        if (st[t]) continue;
        out_key[o] = base + static_cast<uint32_t>(t);
        out_val[o] = g;
        ++o;
      }
    }
    if (o != end) atomicAdd(&counters[kBinningMismatch], 1ull);
  }
  // long lists: the warp takes them one at a time, one tile row per lane
  uint32_t m = __ballot_sync(0xffffffffu, big);
  while (m) {
    const int src = __ffs(m) - 1;
    m &= m - 1;
    const uint32_t gb = __shfl_sync(0xffffffffu, g, src);
    uint32_t ob = __shfl_sync(0xffffffffu, off, src);
    const uint32_t end = ob + __shfl_sync(0xffffffffu, c, src);
    const int v = static_cast<int>(gb / n);
    const Footprint f = foot[gb];
    const int tiles_x = views[v].tiles_x, width = views[v].width;
    const uint32_t base = static_cast<uint32_t>(views[v].tile_base);
    int ty0, ty1;
    footprint_rows(f, &ty0, &ty1);
    const uint8_t* st = sat + base;
    for (int r0 = ty0; r0 <= ty1; r0 += 32) {
      const int ty = r0 + lane;
      int tx0 = 0, tx1 = -1;
      if (ty > ty1 || !row_span(f, ty, width, &tx0, &tx1)) {
        tx0 = 0;
        tx1 = -1;
      }
      uint32_t len = 0;
      for (int tx = tx0; tx <= tx1; ++tx) len += st[ty * tiles_x + tx] ? 0u : 1u;
      uint32_t incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      uint32_t w = ob + incl - len;
      for (int tx = tx0; tx <= tx1 && w < end; ++tx) {
        const int t = ty * tiles_x + tx;
        if (st[t]) continue;
        out_key[w] = base + static_cast<uint32_t>(t);
        out_val[w] = gb;
        ++w;
      }
      ob += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0 && ob != end) atomicAdd(&counters[kBinningMismatch], 1ull);
  }
}

// [start, end) of every tile's run in the tile-sorted list.
__global__ void ranges_kernel(int64_t n_entries, const uint32_t* __restrict__ key,
                              uint2* __restrict__ ranges) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n_entries) return;
  const uint32_t t = key[k];
  if (k == 0 || key[k - 1] != t) ranges[t].x = static_cast<uint32_t>(k);
  if (k == n_entries - 1 || key[k + 1] != t) ranges[t].y = static_cast<uint32_t>(k + 1);
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
                           const float4* cov, ProjRecord* rec, Footprint* foot, uint32_t* cnt,
                           uint32_t* key, uint32_t* val, uint32_t* depth_lo, cudaStream_t stream) {
  if (n == 0 || n_views == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (n + threads - 1) / threads;
  project_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(
      n, n_views, views, pos_op, cov, rec, foot, cnt, key, val, depth_lo);
  return cudaGetLastError();
}

cudaError_t launch_depth_tie_fix(int64_t n, const uint32_t* key, uint32_t* val,
                                 const uint32_t* depth_lo, cudaStream_t stream) {
  if (n < 2) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (n + threads - 1) / threads;
  depth_tie_fix_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(n, key, val,
                                                                              depth_lo);
  return cudaGetLastError();
}

cudaError_t launch_chunk_count(int64_t p0, int64_t n_pos, int64_t n, const ViewParams* views,
                               const uint32_t* sorted_val, const uint32_t* cnt,
                               const Footprint* foot, const uint8_t* sat, uint32_t* out_cnt,
                               cudaStream_t stream) {
  if (n_pos == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (n_pos + threads - 1) / threads;
  chunk_count_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(
      p0, n_pos, n, views, sorted_val, cnt, foot, sat, out_cnt);
  return cudaGetLastError();
}

cudaError_t launch_emit(int64_t p0, int64_t n_pos, int64_t n, const ViewParams* views,
                        const uint32_t* sorted_val, const uint32_t* offsets,
                        const uint32_t* chunk_cnt, const Footprint* foot, const uint8_t* sat,
                        uint32_t* out_key, uint32_t* out_val, unsigned long long* counters,
                        cudaStream_t stream) {
  if (n_pos == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (n_pos + threads - 1) / threads;
  emit_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(
      p0, n_pos, n, views, sorted_val, offsets, chunk_cnt, foot, sat, out_key, out_val, counters);
  return cudaGetLastError();
}

cudaError_t launch_ranges(int64_t n_entries, const uint32_t* key, uint2* ranges,
                          cudaStream_t stream) {
  if (n_entries == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (n_entries + threads - 1) / threads;
  ranges_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(n_entries, key, ranges);
  return cudaGetLastError();
}

}  // namespace fs
