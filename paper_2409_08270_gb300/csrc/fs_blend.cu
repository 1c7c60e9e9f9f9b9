// Front-to-back alpha blending of every mask pixel and accumulation of
// alpha_i T_i into the contribution table (Sec. 3.1 Eq. 1, Sec. 3.2 Eq. 6,
// Sec. 3.3 Eq. 7, Sec. 4.2: "the product alpha_i T_i is aggregated into the
// buffer A_e of the pixel's label through atomic operations").
//
// One 256-thread CTA per 16x16 tile of one view; one thread per pixel.
//  * The tile's pixels are re-assigned to threads in label order (bitonic
//    sort of (label, pixel) keys), so almost every warp holds pixels of a
//    single label.  Which thread walks which pixel does not change any
//    pixel's result.
//  * The tile's depth-sorted Gaussian list is staged 256 records at a time in
//    shared memory; each staging thread turns the record's float-pair offset
//    into this tile's b = W o_tile + c.
//  * Per pixel, per Gaussian: w = W p_local + b, alpha = min(0.99, o 2^-|w|^2);
//    alpha < 1/255 is skipped; the pixel stops before a Gaussian that would
//    take T below 1e-4; otherwise alpha*T is its contribution.
//  * Reduction without per-pixel atomics: each warp writes its 32 pixels'
//    contributions for 32 Gaussians into a padded 32x36 smem block, then lane
//    g sums row g (Gaussian g) over each run of equal labels (vectorised when
//    the warp has one label).  The per-warp sums are combined per (Gaussian,
//    label slot) in shared memory and flushed with one global atomic add per
//    non-zero (Gaussian, label) per staged batch.
#include "fs_common.cuh"
#include "fs_internal.h"

namespace fs {

namespace {

constexpr int kBatch = 256;
constexpr int kWarps = kBlendThreads / 32;
constexpr int kRowPad = 36;     // 32 floats + 4: conflict-free STS.32 and LDS.128
constexpr int kMaxSlots = 4;    // labels per tile combined in shared memory
constexpr int kNoLabel = 0x7FFFFF;

struct BlendSmem {
  float4 w[kBatch];                   // whitening matrix of each staged Gaussian
  float4 bo[kBatch];                  // (b0, b1, opacity, -)
  int32_t gid[kBatch];                // scene index of each staged Gaussian
  float buf[kWarps][32][kRowPad];     // per-warp (Gaussian x pixel) contributions
  float part[kMaxSlots][kBatch];      // CTA partial sums per (label slot, Gaussian)
  int32_t sortkey[kBlendThreads];
  int32_t slot_label[kBlendThreads];
  int32_t lane_slot[kWarps][32];
  uint32_t warp_tmp[kWarps];
  int32_t label0;
};

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

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
  uint32_t pre = 0, all = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const uint32_t c = s_warp[w];
    if (w < warp) pre += c;
    all += c;
  }
  __syncthreads();
  *total = all;
  return pre + inc - x;
}

template <typename TableT>
__device__ __forceinline__ void table_add(TableT* p, float v) {
  atomicAdd(p, static_cast<TableT>(v));
}

// Per-pixel state of a batch before its first depth chunk: T = 1 for pixels
// with a label in [0, E), 0 ("stopped") for the others; a tile with no
// labelled pixel starts saturated.  Counts the pixels with bad labels.
template <typename LabelT>
__global__ void __launch_bounds__(kBlendThreads) state_init_kernel(
    const ViewParams* __restrict__ views, int E, float* __restrict__ state,
    uint8_t* __restrict__ sat, unsigned long long* __restrict__ counters) {
  const int v = blockIdx.y;
  const int tiles_x = views[v].tiles_x;
  const int tile = blockIdx.x;
  if (tile >= tiles_x * views[v].tiles_y) return;  // whole block
  const int W = views[v].width, H = views[v].height;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int px = tx * kTile + (threadIdx.x & 15), py = ty * kTile + (threadIdx.x >> 4);
  const bool inside = px < W && py < H;
  bool valid = false;
  if (inside) {
    const int64_t p = static_cast<int64_t>(py) * W + px;
    const int label = static_cast<int>(static_cast<const LabelT*>(views[v].mask)[p]);
    valid = label >= 0 && label < E;
    state[views[v].state_off + p] = valid ? 1.f : 0.f;
  }
  const int n_bad = __syncthreads_count(inside && !valid);
  const int any = __syncthreads_or(valid);
  if (threadIdx.x == 0) {
    if (n_bad) atomicAdd(&counters[kBadLabels], static_cast<unsigned long long>(n_bad));
    sat[views[v].tile_base + tile] = any ? 0 : 1;
  }
}

template <typename LabelT, typename TableT>
__global__ void __launch_bounds__(kBlendThreads, 4) blend_kernel(
    const ViewParams* __restrict__ views, const uint2* __restrict__ ranges,
    const uint32_t* __restrict__ list_val, const ProjRecord* __restrict__ rec, int64_t n, int E,
    TableT* __restrict__ table, float* __restrict__ state, uint8_t* __restrict__ sat,
    unsigned long long* __restrict__ counters) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BlendSmem& S = *reinterpret_cast<BlendSmem*>(smem_raw);

  const int v = blockIdx.y;
  const int tiles_x = views[v].tiles_x;
  const int n_tiles = tiles_x * views[v].tiles_y;
  const int tile = blockIdx.x;
  if (tile >= n_tiles) return;  // whole block
  const int W = views[v].width, H = views[v].height;
  const LabelT* __restrict__ mask = static_cast<const LabelT*>(views[v].mask);
  const uint2 rg = ranges[views[v].tile_base + tile];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tx = tile % tiles_x, ty = tile / tiles_x;

  // ---- labels of the tile's pixels -------------------------------------
  int label = -1;
  bool inside, valid;
  {
    const int px = tx * kTile + (tid & 15), py = ty * kTile + (tid >> 4);
    inside = px < W && py < H;
    if (inside) label = static_cast<int>(mask[static_cast<int64_t>(py) * W + px]);
    valid = inside && label >= 0 && label < E;
  }
  (void)inside;
  if (rg.y <= rg.x) return;  // no list entry for this tile in this chunk: whole block

  // ---- assign pixels to threads in label order ------------------------
  if (tid == 0) S.label0 = label;
  __syncthreads();
  const bool uniform = __syncthreads_and(valid && label == S.label0);
  int key = ((valid ? label : kNoLabel) << 8) | tid;
  if (!uniform) {
    S.sortkey[tid] = key;
    __syncthreads();
    for (int k = 2; k <= kBlendThreads; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        const int ixj = tid ^ j;
        if (ixj > tid) {
          const int a = S.sortkey[tid], b = S.sortkey[ixj];
          if ((a > b) == ((tid & k) == 0)) {
            S.sortkey[tid] = b;
            S.sortkey[ixj] = a;
          }
        }
        __syncthreads();
      }
    }
    key = S.sortkey[tid];
  } else {
    S.sortkey[tid] = key;
    __syncthreads();
  }
  const int pix = key & 255;
  const int lab = key >> 8;
  valid = lab != kNoLabel;
  // pixel centre relative to the tile centre, in [-7.5, 7.5]
  const float xl = static_cast<float>(pix & 15) - 7.5f;
  const float yl = static_cast<float>(pix >> 4) - 7.5f;

  // ---- label slots of the tile (distinct labels, in order) -------------
  const int prev_lab = tid > 0 ? (S.sortkey[tid - 1] >> 8) : -1;
  const bool slot_start = valid && lab != prev_lab;
  uint32_t n_slots;
  const uint32_t ex = block_exclusive_scan(slot_start ? 1u : 0u, S.warp_tmp, &n_slots);
  const int slot = valid ? static_cast<int>(ex + (slot_start ? 1u : 0u)) - 1 : -1;
  if (slot_start) S.slot_label[slot] = lab;
  S.lane_slot[warp][lane] = slot;
  const bool cta_agg = n_slots <= static_cast<uint32_t>(kMaxSlots);
  if (cta_agg)
    for (uint32_t s = 0; s < n_slots; ++s) S.part[s][tid] = 0.f;
  // runs of equal labels inside the warp
  const int prev_lane_lab = __shfl_up_sync(0xffffffffu, lab, 1);
  const uint32_t segmask = __ballot_sync(0xffffffffu, lane == 0 || lab != prev_lane_lab);
  const int slot0 = __shfl_sync(0xffffffffu, slot, 0);
  const bool warp_uniform = (segmask == 1u) && slot0 >= 0;
  __syncthreads();

  // ---- walk the tile's list front to back ------------------------------
  // T resumes from the previous depth chunk; T == 0 marks a stopped pixel.
  const int64_t spix = views[v].state_off +
                       static_cast<int64_t>(ty * kTile + (pix >> 4)) * W + tx * kTile + (pix & 15);
  float T = valid ? state[spix] : 0.f;
  bool done = !(T > 0.f);
  uint32_t n_eval = 0;  // pairs this thread evaluated
  const float ox = static_cast<float>(tx * kTile + 8), oy = static_cast<float>(ty * kTile + 8);
  uint32_t n_staged = 0;  // list entries staged by this block (thread 0 counts)
  const uint32_t gbase = static_cast<uint32_t>(static_cast<int64_t>(v) * n);
  float* const row = &S.buf[warp][lane][0];

  for (uint32_t base = rg.x; base < rg.y; base += kBatch) {
    if (__syncthreads_count(!done) == 0) break;
    const int nin = static_cast<int>(min(static_cast<uint32_t>(kBatch), rg.y - base));
    n_staged += static_cast<uint32_t>(nin);
    if (tid < nin) {
      // b = W o + c for the tile centre o, with W = W_hi + W_lo and c as float
      // pairs: W_hi o exactly (TwoProduct), W_lo o in FP32 (a 2^-24 correction)
      const uint32_t g = list_val[base + tid];
      const ProjRecord r = rec[g];
      f2 b0 = f2_add(two_prod(r.w_hi.x, ox), two_prod(r.w_hi.y, oy));
      f2 b1 = f2_add(two_prod(r.w_hi.z, ox), two_prod(r.w_hi.w, oy));
      b0 = f2_add(b0, f2{r.c.x, r.c.z});
      b1 = f2_add(b1, f2{r.c.y, r.c.w});
      b0 = f2_add(b0, f2_from(fmaf(r.w_lo.x, ox, r.w_lo.y * oy)));
      b1 = f2_add(b1, f2_from(fmaf(r.w_lo.z, ox, r.w_lo.w * oy)));
      S.w[tid] = r.w_hi;
      S.bo[tid] = make_float4(b0.hi + b0.lo, b1.hi + b1.lo, r.misc.x, 0.f);
      S.gid[tid] = static_cast<int32_t>(g - gbase);
    }
    __syncthreads();

    if (__any_sync(0xffffffffu, !done)) {
      for (int j0 = 0; j0 < nin; j0 += 32) {
        const int nj = min(32, nin - j0);
        for (int jj = 0; jj < nj; ++jj) {
          float c = 0.f;
          if (!done) {
            ++n_eval;
            const float4 wm = S.w[j0 + jj];
            const float4 bo = S.bo[j0 + jj];
            const float w0 = fmaf(wm.x, xl, fmaf(wm.y, yl, bo.x));
            const float w1 = fmaf(wm.z, xl, fmaf(wm.w, yl, bo.y));
            const float q = fmaf(w0, w0, w1 * w1);
            const float alpha = fminf(kAlphaMax, bo.z * ex2_approx(-q));
            if (alpha >= kAlphaMin) {
              const float test_T = T * (1.f - alpha);
              if (test_T < kTMin) {
                done = true;
              } else {
                c = alpha * T;
                T = test_T;
              }
            }
          }
          S.buf[warp][jj][lane] = c;
        }
        __syncwarp();
        if (lane < nj) {
          const int j = j0 + lane;
          if (warp_uniform) {
            float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const float4 x = reinterpret_cast<const float4*>(row)[k];
              s4.x += x.x;
              s4.y += x.y;
              s4.z += x.z;
              s4.w += x.w;
            }
            const float sum = (s4.x + s4.y) + (s4.z + s4.w);
            if (sum != 0.f) {
              if (cta_agg)
                atomicAdd(&S.part[slot0][j], sum);
              else
                table_add(&table[static_cast<int64_t>(S.gid[j]) * E + S.slot_label[slot0]], sum);
            }
          } else {
            uint32_t m = segmask;
            while (m) {
              const int s = __ffs(m) - 1;
              m &= m - 1;
              const int e = m ? __ffs(m) - 1 : 32;
              const int sl = S.lane_slot[warp][s];
              if (sl < 0) continue;
              float sum = 0.f;
              for (int l = s; l < e; ++l) sum += row[l];
              if (sum != 0.f) {
                if (cta_agg)
                  atomicAdd(&S.part[sl][j], sum);
                else
                  table_add(&table[static_cast<int64_t>(S.gid[j]) * E + S.slot_label[sl]], sum);
              }
            }
          }
        }
        __syncwarp();
        if (__all_sync(0xffffffffu, done)) break;
      }
    }
    __syncthreads();
    if (cta_agg && tid < nin) {
      const int64_t rowbase = static_cast<int64_t>(S.gid[tid]) * E;
      for (uint32_t s = 0; s < n_slots; ++s) {
        const float p = S.part[s][tid];
        if (p != 0.f) {
          table_add(&table[rowbase + S.slot_label[s]], p);
          S.part[s][tid] = 0.f;
        }
      }
    }
  }
  if (valid) state[spix] = done ? 0.f : T;
  const int all_done = __syncthreads_and(done);
  if (tid == 0 && all_done) sat[views[v].tile_base + tile] = 1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n_eval += __shfl_xor_sync(0xffffffffu, n_eval, o);
  if (lane == 0 && n_eval) atomicAdd(&counters[kPairs], static_cast<unsigned long long>(n_eval));
  if (tid == 0 && n_staged) atomicAdd(&counters[kStaged], static_cast<unsigned long long>(n_staged));
}

template <typename LabelT, typename TableT>
cudaError_t launch_typed(const ViewParams* views, int n_views, int max_tiles, const uint2* ranges,
                         const uint32_t* list_val, const ProjRecord* rec, int64_t n, int E,
                         void* table, float* state, uint8_t* sat, unsigned long long* counters,
                         cudaStream_t stream) {
  const size_t smem = sizeof(BlendSmem);
  cudaError_t e = cudaFuncSetAttribute(blend_kernel<LabelT, TableT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  dim3 grid(static_cast<unsigned>(max_tiles), static_cast<unsigned>(n_views));
  blend_kernel<LabelT, TableT><<<grid, kBlendThreads, smem, stream>>>(
      views, ranges, list_val, rec, n, E, static_cast<TableT*>(table), state, sat, counters);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_state_init(const ViewParams* views, int n_views, int max_tiles_per_view, int E,
                              int mask_dtype, float* state, uint8_t* sat,
                              unsigned long long* counters, cudaStream_t stream) {
  if (n_views == 0 || max_tiles_per_view == 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>(max_tiles_per_view), static_cast<unsigned>(n_views));
  if (mask_dtype == 4)
    state_init_kernel<uint8_t><<<grid, kBlendThreads, 0, stream>>>(views, E, state, sat, counters);
  else
    state_init_kernel<int32_t><<<grid, kBlendThreads, 0, stream>>>(views, E, state, sat, counters);
  return cudaGetLastError();
}

cudaError_t launch_blend(const ViewParams* views, int n_views, int max_tiles_per_view,
                         const uint2* ranges, const uint32_t* list_val, const ProjRecord* rec,
                         int64_t n, int E, int mask_dtype, void* table, int table_dtype,
                         float* state, uint8_t* sat, unsigned long long* counters,
                         cudaStream_t stream) {
  if (n_views == 0 || max_tiles_per_view == 0) return cudaSuccess;
  const int mt = max_tiles_per_view;
  if (mask_dtype == 4) {
    if (table_dtype == 0)
      return launch_typed<uint8_t, float>(views, n_views, mt, ranges, list_val, rec, n, E, table,
                                          state, sat, counters, stream);
    return launch_typed<uint8_t, double>(views, n_views, mt, ranges, list_val, rec, n, E, table,
                                         state, sat, counters, stream);
  }
  if (table_dtype == 0)
    return launch_typed<int32_t, float>(views, n_views, mt, ranges, list_val, rec, n, E, table,
                                        state, sat, counters, stream);
  return launch_typed<int32_t, double>(views, n_views, mt, ranges, list_val, rec, n, E, table,
                                       state, sat, counters, stream);
}

}  // namespace fs
