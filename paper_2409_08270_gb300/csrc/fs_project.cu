// Scene preparation, EWA projection and tile binning (Sec. 3.1).
//
// Projection of Gaussian i into view v (all FP32 / float-pair, no FP64 pipe):
//   t = R m + t_c                      float pairs (compensated dot product)
//   m2D = (fx tx/tz + cx, fy ty/tz + cy)   float pairs
//   J = perspective Jacobian at t with tx/tz, ty/tz clamped to 1.3 tan(fov/2)
//   Sigma2D = J W Rq diag(s^2) Rq^T W^T J^T + 0.3 I
// The thin eigenvalue of Sigma2D is what makes elongated Gaussians
// ill-conditioned; it is computed as det/lambda1 with det taken from the
// Cauchy-Binet form det(M M^T) = sum_l (s_j s_k n_l)^2, n = rows(J W Rq)
// crossed, which is a sum of squares and loses nothing to cancellation.
// The record stores the whitening matrix W (|W d|^2 = 0.5 log2(e) d^T
// Sigma2D^-1 d) built from the eigen-decomposition, and c = -W m2D as float
// pairs, so the blend evaluates alpha = o 2^(-|W p + b|^2) with per-tile
// offsets b = W o_tile + c that are exact to about 1e-10.
#include <cuda_fp16.h>

#include "fs_common.cuh"
#include "fs_internal.h"

namespace fs {

// ---------------------------------------------------------------------------
// scene preparation: normalise quaternions, pack attributes, validate
// ---------------------------------------------------------------------------

__device__ __forceinline__ float load_attr(const void* p, int64_t idx, int dtype) {
  if (dtype == 0) return static_cast<const float*>(p)[idx];
  const uint16_t bits = static_cast<const uint16_t*>(p)[idx];
  if (dtype == 2) return __uint_as_float(static_cast<uint32_t>(bits) << 16);  // bf16
  return __half2float(__ushort_as_half(bits));                                 // fp16
}

__global__ void scene_prep_kernel(int64_t n, const float* __restrict__ mean, const void* quat,
                                  int quat_dtype, const void* scale, int scale_dtype,
                                  const void* opacity, int opacity_dtype, float4* __restrict__ pos_op,
                                  float4* __restrict__ q_out, float4* __restrict__ s_out,
                                  unsigned int* __restrict__ err) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float mx = mean[3 * i], my = mean[3 * i + 1], mz = mean[3 * i + 2];
  const float o = load_attr(opacity, i, opacity_dtype);
  float qw = load_attr(quat, 4 * i, quat_dtype), qx = load_attr(quat, 4 * i + 1, quat_dtype);
  float qy = load_attr(quat, 4 * i + 2, quat_dtype), qz = load_attr(quat, 4 * i + 3, quat_dtype);
  const float s0 = load_attr(scale, 3 * i, scale_dtype), s1 = load_attr(scale, 3 * i + 1, scale_dtype);
  const float s2 = load_attr(scale, 3 * i + 2, scale_dtype);
  bool bad = !(isfinite(mx) && isfinite(my) && isfinite(mz) && isfinite(o) && isfinite(qw) &&
               isfinite(qx) && isfinite(qy) && isfinite(qz) && isfinite(s0) && isfinite(s1) &&
               isfinite(s2));
  // Normalised once per scene; the FP32 unit quaternion defines the rotation
  // to a few ulp, i.e. it turns a Gaussian by ~1e-7 rad at most.
  const double nn = (double)qw * qw + (double)qx * qx + (double)qy * qy + (double)qz * qz;
  if (!(nn > 0.0)) bad = true;
  if (bad) {
    atomicOr(err, 1u);
    pos_op[i] = make_float4(0.f, 0.f, -1e30f, 0.f);
    q_out[i] = make_float4(1.f, 0.f, 0.f, 0.f);
    s_out[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const float inv = static_cast<float>(1.0 / sqrt(nn));
  pos_op[i] = make_float4(mx, my, mz, o);
  q_out[i] = make_float4(qw * inv, qx * inv, qy * inv, qz * inv);
  s_out[i] = make_float4(fabsf(s0), fabsf(s1), fabsf(s2), 0.f);
}

// ---------------------------------------------------------------------------
// projection
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool f2_greater(f2 a, float b_hi, float b_lo) {
  return a.hi > b_hi || (a.hi == b_hi && a.lo > b_lo);
}

// One thread per Gaussian; it projects the Gaussian into every view of the
// batch so the scene is read once per batch.
__global__ void __launch_bounds__(256) project_kernel(
    int64_t n, int n_views, const ViewParams* __restrict__ views_g,
    const float4* __restrict__ pos_op, const float4* __restrict__ quat,
    const float4* __restrict__ scale, ProjRecord* __restrict__ rec, uint2* __restrict__ rect,
    uint32_t* __restrict__ cnt, uint32_t* __restrict__ key, uint32_t* __restrict__ val) {
  __shared__ ViewParams views[kMaxViewsPerBatch];
  for (int k = threadIdx.x; k < n_views * (int)(sizeof(ViewParams) / 4); k += blockDim.x)
    reinterpret_cast<uint32_t*>(views)[k] = reinterpret_cast<const uint32_t*>(views_g)[k];
  __syncthreads();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;

  const float4 po = pos_op[i];
  const float4 q = quat[i];
  const float4 s = scale[i];
  // rotation of the unit quaternion (w, x, y, z)
  const float w = q.x, x = q.y, y = q.z, z = q.w;
  float Rq[3][3];
  Rq[0][0] = 1.f - 2.f * (y * y + z * z);
  Rq[0][1] = 2.f * (x * y - w * z);
  Rq[0][2] = 2.f * (x * z + w * y);
  Rq[1][0] = 2.f * (x * y + w * z);
  Rq[1][1] = 1.f - 2.f * (x * x + z * z);
  Rq[1][2] = 2.f * (y * z - w * x);
  Rq[2][0] = 2.f * (x * z - w * y);
  Rq[2][1] = 2.f * (y * z + w * x);
  Rq[2][2] = 1.f - 2.f * (x * x + y * y);
  const float o = po.w;
  const bool opaque_enough = o >= kAlphaMin;
  // r2 bounds d^T Sigma^-1 d where alpha can still reach 1/255
  const float r2 = opaque_enough ? fmaxf(2.f * logf(255.f * o), 0.f) : 0.f;

  for (int v = 0; v < n_views; ++v) {
    const ViewParams& vp = views[v];
    const int64_t slot = static_cast<int64_t>(v) * n + i;
    const f2 tx = f2_dot3_add(vp.R_hi + 0, vp.R_lo + 0, po.x, po.y, po.z, vp.t_hi[0], vp.t_lo[0]);
    const f2 ty = f2_dot3_add(vp.R_hi + 3, vp.R_lo + 3, po.x, po.y, po.z, vp.t_hi[1], vp.t_lo[1]);
    const f2 tz = f2_dot3_add(vp.R_hi + 6, vp.R_lo + 6, po.x, po.y, po.z, vp.t_hi[2], vp.t_lo[2]);
    bool visible = opaque_enough && f2_greater(tz, vp.near_hi, vp.near_lo);
    uint2 rc = make_uint2(0u, 0u);
    uint32_t count = 0;
    float depth = 0.f;
    ProjRecord R;
    R.w = make_float4(0.f, 0.f, 0.f, 0.f);
    R.c = make_float4(0.f, 0.f, 0.f, 0.f);
    R.misc = make_float4(o, 0.f, 0.f, 0.f);
    if (visible) {
      const f2 ux = f2_div(tx, tz), uy = f2_div(ty, tz);
      const f2 mx = f2_add(f2_mul(f2{vp.fx_hi, vp.fx_lo}, ux), f2{vp.cx_hi, vp.cx_lo});
      const f2 my = f2_add(f2_mul(f2{vp.fy_hi, vp.fy_lo}, uy), f2{vp.cy_hi, vp.cy_lo});
      depth = tz.hi;
      // Jacobian rows J0 = fx/z (1, 0, -ux), J1 = fy/z (0, 1, -uy), clamped ux, uy
      const float iz = 1.f / tz.hi;
      const float uxc = fminf(fmaxf(ux.hi, -vp.limx), vp.limx);
      const float uyc = fminf(fmaxf(uy.hi, -vp.limy), vp.limy);
      const float j0 = vp.fx_hi * iz, j1 = vp.fy_hi * iz;
      float T0[3], T1[3];  // rows of J W
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        T0[k] = j0 * (vp.R_hi[k] - uxc * vp.R_hi[6 + k]);
        T1[k] = j1 * (vp.R_hi[3 + k] - uyc * vp.R_hi[6 + k]);
      }
      float A0[3], A1[3];  // rows of J W Rq
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        A0[k] = T0[0] * Rq[0][k] + T0[1] * Rq[1][k] + T0[2] * Rq[2][k];
        A1[k] = T1[0] * Rq[0][k] + T1[1] * Rq[1][k] + T1[2] * Rq[2][k];
      }
      const float sv[3] = {s.x, s.y, s.z};
      float a = 0.f, b = 0.f, c = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float m0 = A0[k] * sv[k], m1 = A1[k] * sv[k];
        a = fmaf(m0, m0, a);
        b = fmaf(m0, m1, b);
        c = fmaf(m1, m1, c);
      }
      // Cauchy-Binet: det(M M^T) with M = A diag(s)
      const float n0 = A0[1] * A1[2] - A0[2] * A1[1];
      const float n1 = A0[2] * A1[0] - A0[0] * A1[2];
      const float n2 = A0[0] * A1[1] - A0[1] * A1[0];
      const float d0 = sv[1] * sv[2] * n0, d1 = sv[0] * sv[2] * n1, d2 = sv[0] * sv[1] * n2;
      const float det0 = d0 * d0 + d1 * d1 + d2 * d2;
      // low-pass: Sigma2D = Sigma' + 0.3 I
      const float det = det0 + kLowPass * (a + c) + kLowPass * kLowPass;
      a += kLowPass;
      c += kLowPass;
      const float h = 0.5f * (a - c);
      const float rr = sqrtf(h * h + b * b);
      const float lam1 = 0.5f * (a + c) + rr;
      const float lam2 = det / lam1;
      // unit eigenvector of lam1, computed from whichever form has no cancellation
      float ex, ey;
      if (h >= 0.f) { ex = h + rr; ey = b; } else { ex = b; ey = rr - h; }
      const float en = sqrtf(ex * ex + ey * ey);
      if (en > 0.f) { ex /= en; ey /= en; } else { ex = 1.f; ey = 0.f; }
      const float k1 = sqrtf(static_cast<float>(kHalfLog2e) / lam1);
      const float k2 = sqrtf(static_cast<float>(kHalfLog2e) / lam2);
      const float W00 = k1 * ex, W01 = k1 * ey, W10 = -k2 * ey, W11 = k2 * ex;
      // c = -W m2D in float pairs
      const f2 c0 = f2_add(f2_mul_f(mx, -W00), f2_mul_f(my, -W01));
      const f2 c1 = f2_add(f2_mul_f(mx, -W10), f2_mul_f(my, -W11));
      R.w = make_float4(W00, W01, W10, W11);
      R.c = make_float4(c0.hi, c1.hi, c0.lo, c1.lo);
      // conservative pixel box of the alpha >= 1/255 ellipse, one pixel margin
      const float hx = sqrtf(a * r2), hy = sqrtf(c * r2);
      const float px0 = ceilf(mx.hi - hx - 1.5f), px1 = floorf(mx.hi + hx + 0.5f);
      const float py0 = ceilf(my.hi - hy - 1.5f), py1 = floorf(my.hi + hy + 0.5f);
      if (!(px1 >= 0.f && py1 >= 0.f && px0 <= vp.width - 1 && py0 <= vp.height - 1)) {
        visible = false;
      } else {
        const int tx0 = max(0, static_cast<int>(fmaxf(px0, 0.f)) / kTile);
        const int ty0 = max(0, static_cast<int>(fmaxf(py0, 0.f)) / kTile);
        const int tx1 = min(vp.tiles_x - 1, static_cast<int>(fminf(px1, (float)vp.width)) / kTile);
        const int ty1 = min(vp.tiles_y - 1, static_cast<int>(fminf(py1, (float)vp.height)) / kTile);
        if (tx0 > tx1 || ty0 > ty1) {
          visible = false;
        } else {
          rc = make_uint2(static_cast<uint32_t>(tx0) | (static_cast<uint32_t>(ty0) << 16),
                          static_cast<uint32_t>(tx1) | (static_cast<uint32_t>(ty1) << 16));
          count = static_cast<uint32_t>((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
        }
      }
    }
    rec[slot] = R;
    rect[slot] = rc;
    cnt[slot] = visible ? count : 0u;
    key[slot] = visible ? depth_key(depth) : 0xFFFFFFFFu;
    val[slot] = static_cast<uint32_t>(slot);
  }
}

// ---------------------------------------------------------------------------
// emission of (tile, Gaussian) list entries in depth order
// ---------------------------------------------------------------------------

__global__ void emit_kernel(int64_t k_total, int64_t n, const ViewParams* __restrict__ views,
                            const uint32_t* __restrict__ sorted_val,
                            const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ cnt,
                            const uint2* __restrict__ rect, uint32_t* __restrict__ out_key,
                            uint32_t* __restrict__ out_val) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= k_total) return;
  const uint32_t g = sorted_val[k];
  const uint32_t c = cnt[g];
  if (c == 0) return;
  const int v = static_cast<int>(g / n);
  const uint2 rc = rect[g];
  const int tx0 = rc.x & 0xFFFF, ty0 = rc.x >> 16, tx1 = rc.y & 0xFFFF, ty1 = rc.y >> 16;
  const int tiles_x = views[v].tiles_x;
  const uint32_t base = static_cast<uint32_t>(views[v].tile_base);
  uint32_t o = offsets[k];
  for (int ty = ty0; ty <= ty1; ++ty)
    for (int tx = tx0; tx <= tx1; ++tx) {
      out_key[o] = base + static_cast<uint32_t>(ty * tiles_x + tx);
      out_val[o] = g;
      ++o;
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
                              int opacity_dtype, float4* pos_op, float4* q_out, float4* s_out,
                              unsigned int* err, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (n + threads - 1) / threads;
  scene_prep_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(
      n, mean, quat, quat_dtype, scale, scale_dtype, opacity, opacity_dtype, pos_op, q_out, s_out,
      err);
  return cudaGetLastError();
}

cudaError_t launch_project(int64_t n, int n_views, const ViewParams* views, const float4* pos_op,
                           const float4* quat, const float4* scale, ProjRecord* rec, uint2* rect,
                           uint32_t* cnt, uint32_t* key, uint32_t* val, cudaStream_t stream) {
  if (n == 0 || n_views == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (n + threads - 1) / threads;
  project_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(
      n, n_views, views, pos_op, quat, scale, rec, rect, cnt, key, val);
  return cudaGetLastError();
}

cudaError_t launch_emit(int64_t k_total, int64_t n, const ViewParams* views,
                        const uint32_t* sorted_val, const uint32_t* offsets, const uint32_t* cnt,
                        const uint2* rect, uint32_t* out_key, uint32_t* out_val,
                        cudaStream_t stream) {
  if (k_total == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (k_total + threads - 1) / threads;
  emit_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(
      k_total, n, views, sorted_val, offsets, cnt, rect, out_key, out_val);
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
