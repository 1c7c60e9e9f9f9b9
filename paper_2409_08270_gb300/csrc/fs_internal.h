// Internal launcher interface between the host runtime and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fs {

constexpr int kMaxViewsPerBatch = 32;
constexpr int kMaxLabels = 4096;

struct ViewParams;
struct ProjRecord;
struct Footprint;

// scan / sort (fs_sort.cu) --------------------------------------------------
// Temporary storage needed by exclusive_scan for n elements (bytes).
size_t scan_temp_bytes(int64_t n);
// out[k] = sum_{j<k} in[gather ? gather[j] : j]; *total = the full sum (device).
cudaError_t exclusive_scan(const uint32_t* in, const uint32_t* gather, uint32_t* out, int64_t n,
                           uint32_t* total, void* temp, cudaStream_t stream);
// Temporary storage of radix_sort_pairs for n elements (bytes).
size_t radix_temp_bytes(int64_t n);
// Stable LSD radix sort of (key, val) pairs on the low `bits` bits of key.
// Ping-pongs between (keys, vals) and (keys_alt, vals_alt); *in_alt tells the
// caller which pair holds the result.
cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                             uint32_t* vals_alt, int64_t n, int bits, void* temp, bool* in_alt,
                             cudaStream_t stream);

// projection / binning (fs_project.cu) --------------------------------------
// pos_op[n] = (m, o); cov[3n] = Sigma3D as float pairs (FP64 once per scene)
cudaError_t launch_scene_prep(int64_t n, const float* mean, const void* quat, int quat_dtype,
                              const void* scale, int scale_dtype, const void* opacity,
                              int opacity_dtype, float4* pos_op, float4* cov, unsigned int* err,
                              cudaStream_t stream);
cudaError_t launch_project(int64_t n, int n_views, const ViewParams* views, const float4* pos_op,
                           const float4* cov, ProjRecord* rec, Footprint* foot, uint32_t* cnt,
                           uint32_t* key, uint32_t* val, uint32_t* depth_lo, cudaStream_t stream);
// re-orders runs of equal 32-bit depth keys by the depth's low word, then slot
// (n_total elements; slot / n is the view of a slot)
cudaError_t launch_depth_tie_fix(int64_t n_total, int64_t n, const uint32_t* key, uint32_t* val,
                                 const uint32_t* depth_lo, cudaStream_t stream);
cudaError_t launch_chunk_count(int64_t p0, int64_t n_pos, int64_t n, const ViewParams* views,
                               const uint32_t* sorted_val, const uint32_t* cnt,
                               const Footprint* foot, const uint64_t* sat, uint32_t* out_cnt,
                               cudaStream_t stream);
cudaError_t launch_emit(int64_t p0, int64_t n_pos, int64_t n, const ViewParams* views,
                        const uint32_t* sorted_val, const uint32_t* offsets,
                        const uint32_t* chunk_cnt, const uint32_t* cnt, const Footprint* foot,
                        const uint64_t* sat, uint32_t* out_key, uint32_t* out_val,
                        unsigned long long* counters, cudaStream_t stream);
cudaError_t launch_ranges(int64_t n_entries, const uint32_t* key, uint2* ranges,
                          cudaStream_t stream);

// blend / accumulate (fs_blend.cu) ------------------------------------------
// mask_dtype: 4 = uint8, 5 = int32.  table_dtype: 0 = f32, 1 = f64.
// state: per-pixel transmittance of the batch (0 = stopped).  sat / subsat:
// bit arrays over the batch's tile ids / 4 * tile id + sub-tile: set = every
// pixel of the tile / 8x8 sub-tile stopped (cleared by the caller before
// state_init).
cudaError_t launch_state_init(const ViewParams* views, int n_views, int max_tiles_per_view, int E,
                              int mask_dtype, float* state, uint64_t* sat, uint64_t* subsat,
                              unsigned long long* counters, cudaStream_t stream);
cudaError_t launch_blend(const ViewParams* views, int n_views, int max_tiles_per_view,
                         const uint2* ranges, const uint32_t* list_val, const ProjRecord* rec,
                         int64_t n, int E, int mask_dtype, void* table, int table_dtype,
                         float* state, uint64_t* sat, uint64_t* subsat,
                         unsigned long long* counters, cudaStream_t stream);

// assignment (fs_assign.cu) -------------------------------------------------
cudaError_t launch_assign(const void* table, int table_dtype, int64_t n, int E, float gamma,
                          uint64_t* member_bits, int32_t* label, float* margin,
                          cudaStream_t stream);

// Sets the calling thread's fs_last_error() message (fs_api.cu).
void set_last_error(const char* msg);

// device counters (unsigned long long) written by the kernels
enum Counter { kBadLabels = 0, kPairs = 1, kStaged = 2, kBinningMismatch = 3, kNumCounters = 4 };

}  // namespace fs
