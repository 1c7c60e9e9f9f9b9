// Tile-binning geometry shared by the binning kernels and the near-tie
// re-check: which 16x16 tiles a Gaussian's alpha >= 1/255 footprint reaches.
#pragma once

#include "fs_common.cuh"

namespace fs {

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

// Saturated tiles are bits of a bit array over the batch's tile ids.
// Number of unsaturated tiles among ids [a, b].
__device__ __forceinline__ uint32_t count_free(const uint64_t* __restrict__ sat, int a, int b) {
  uint32_t c = 0;
  const int wa = a >> 6, wb = b >> 6;
  for (int w = wa; w <= wb; ++w) {
    uint64_t m = ~0ull;
    if (w == wa) m &= ~0ull << (a & 63);
    if (w == wb) m &= ~0ull >> (63 - (b & 63));
    c += static_cast<uint32_t>(__popcll(~sat[w] & m));
  }
  return c;
}

// Whether any tile id in [a, b] is unsaturated.
__device__ __forceinline__ bool any_free(const uint64_t* __restrict__ sat, int a, int b) {
  const int wa = a >> 6, wb = b >> 6;
  for (int w = wa; w <= wb; ++w) {
    uint64_t m = ~0ull;
    if (w == wa) m &= ~0ull << (a & 63);
    if (w == wb) m &= ~0ull >> (63 - (b & 63));
    if (~sat[w] & m) return true;
  }
  return false;
}

// Unsaturated tiles of rows [r0, r1] x columns [c0, c1] of a view, from its
// prefix table (four reads).
__device__ __forceinline__ uint32_t free_in_box(const ViewParams& vp, int r0, int r1, int c0,
                                                int c1) {
  const int w1 = vp.tiles_x + 1;
  const uint32_t* t = vp.free_tab;
  return t[(r1 + 1) * w1 + c1 + 1] - t[r0 * w1 + c1 + 1] - t[(r1 + 1) * w1 + c0] +
         t[r0 * w1 + c0];
}

// Hardware square root (relative error ~2^-23): far inside the one-pixel
// margin of the spans below, and the same instruction wherever a span is
// evaluated, so every kernel that bins gets identical spans.
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Tiles [tx0, tx1] of tile row ty touched by the footprint (false if none).
// The band of pixel-centre rows of the tile, widened by one pixel, is
// intersected with the ellipse; over the band the right boundary x(dy) is
// concave, so its maximum is at the rightmost point dy* clamped to the band
// (and the left boundary's minimum at -dy*, clamped).
__device__ __forceinline__ bool row_span(const Footprint& f, int ty, int width, int* tx0,
                                         int* tx1) {
  const float yt = static_cast<float>(ty * kTile);
  const float y0 = __fsub_rn(__fadd_rn(yt, -0.5f), f.my);   // band widened by one pixel
  const float y1 = __fsub_rn(__fadd_rn(yt, 16.5f), f.my);
  const float u0 = fmaxf(y0, -f.hy), u1 = fminf(y1, f.hy);
  if (!(u0 <= u1)) return false;
  const float dr = fminf(fmaxf(f.dys, u0), u1), dl = fminf(fmaxf(-f.dys, u0), u1);
  const float sr = sqrt_approx(__fmul_rn(f.b2, fmaxf(0.f, __fsub_rn(f.syr, __fmul_rn(dr, dr)))));
  const float sl = sqrt_approx(__fmul_rn(f.b2, fmaxf(0.f, __fsub_rn(f.syr, __fmul_rn(dl, dl)))));
  const float xr = __fadd_rn(__fadd_rn(f.mx, __fmul_rn(f.a, dr)), sr);
  const float xl = __fsub_rn(__fadd_rn(f.mx, __fmul_rn(f.a, dl)), sl);
  float px0 = ceilf(__fsub_rn(xl, 1.5f)), px1 = floorf(__fadd_rn(xr, 0.5f));
  px0 = fmaxf(px0, 0.f);
  px1 = fminf(px1, static_cast<float>(width - 1));
  if (!(px0 <= px1)) return false;
  *tx0 = static_cast<int>(px0) / kTile;
  *tx1 = static_cast<int>(px1) / kTile;
  return true;
}

// Under 3-sigma coverage, [tx0, tx1] narrowed to the slot's tile columns
// (false if nothing is left); unchanged under exact coverage.
__device__ __forceinline__ bool clip_cols(const ViewParams& vp, int64_t slot, int* tx0,
                                          int* tx1) {
  if (!vp.cols) return true;
  const uint32_t c = vp.cols[slot];
  *tx0 = max(*tx0, static_cast<int>(c & 0xFFFFu));
  *tx1 = min(*tx1, static_cast<int>(c >> 16));
  return *tx0 <= *tx1;
}

}  // namespace fs
