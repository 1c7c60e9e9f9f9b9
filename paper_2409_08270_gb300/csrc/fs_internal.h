// Internal launcher interface between the host runtime and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

struct fs_ctx;
struct fs_camera;

namespace fs {

constexpr int kMaxViewsPerBatch = 64;
constexpr int kMaxLabels = 4096;

struct ViewParams;
struct ProjRecord;
struct CompactRecord;
struct Footprint;

// scan / sort (fs_sort.cu) --------------------------------------------------
// Temporary storage needed by exclusive_scan for n elements (bytes).
size_t scan_temp_bytes(int64_t n);
// out[k] = sum_{j<k} in[gather ? gather[j] : j]; *total = the full sum (device).
cudaError_t exclusive_scan(const uint32_t* in, const uint32_t* gather, uint32_t* out, int64_t n,
                           uint32_t* total, void* temp, cudaStream_t stream);
// Passes radix_sort_pairs makes for a `bits`-bit key (8- or 9-bit digits).
int radix_passes(int bits);
// Temporary storage of radix_sort_pairs for n elements (bytes).
size_t radix_temp_bytes(int64_t n);
// Stable LSD radix sort of (key, val) pairs on the low `bits` bits of
// min(key - kmin, span) (the keys themselves are moved unchanged).
// Ping-pongs between (keys, vals) and (keys_alt, vals_alt); *in_alt tells the
// caller which pair holds the result.  n_dev (may be NULL): the count to sort
// is min(n, *n_dev), read on the device (the grid is sized for n); range_dev
// (may be NULL): kmin and span from a device key range {min, max}.
cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                             uint32_t* vals_alt, int64_t n, int bits, void* temp, bool* in_alt,
                             cudaStream_t stream, uint32_t kmin = 0u,
                             uint32_t span = 0xFFFFFFFFu, const uint32_t* n_dev = nullptr,
                             const uint32_t* range_dev = nullptr);

// projection / binning (fs_project.cu) --------------------------------------
// pos_op[n] = (m, o); cov[3n] = Sigma3D as float pairs (FP64 once per scene)
cudaError_t launch_scene_prep(int64_t n, const float* mean, const void* quat, int quat_dtype,
                              const void* scale, int scale_dtype, const void* opacity,
                              int opacity_dtype, float4* pos_op, float4* cov, unsigned int* err,
                              cudaStream_t stream);
// rec16 != NULL: reduced-precision records (FP16 whitening matrix, FP32 mean)
// are written to rec16 instead of the float-pair records to rec.  Records are
// written for visible slots only (nothing reads the others'); footprints,
// counts, keys, values and low depth words for every slot.
// key_range (3 uint32, may be NULL): atomic min / max of the visible slots'
// depth keys and their number (the caller initialises it to {0xFFFFFFFF, 0,
// 0}).  After the depth sort the visible slots are the first ones.
cudaError_t launch_project(int64_t n, int n_views, const ViewParams* views, const float4* pos_op,
                           const float4* cov, ProjRecord* rec, CompactRecord* rec16,
                           Footprint* foot, uint32_t* cnt, uint32_t* key, uint32_t* val,
                           uint32_t* depth_lo, uint32_t* key_range, cudaStream_t stream);
// re-orders runs of equal 32-bit depth keys by the depth's low word, then slot
// (n_total elements; slot / n is the view of a slot)
cudaError_t launch_depth_tie_fix(int64_t n_total, int64_t n, const uint32_t* key, uint32_t* val,
                                 const uint32_t* depth_lo, cudaStream_t stream,
                                 const uint32_t* n_dev = nullptr);
// Binning of sorted positions [p0, p0 + n_pos): one list entry (key = tile
// id, value = slot) per (tile, Gaussian) whose footprint reaches the tile,
// unless the tile's `sat` bit is set.
cudaError_t launch_chunk_count(int64_t p0, int64_t n_pos, int64_t n, const ViewParams* views,
                               const uint32_t* sorted_val, const Footprint* foot,
                               const uint64_t* sat, uint32_t* out_cnt, cudaStream_t stream);
cudaError_t launch_emit(int64_t p0, int64_t n_pos, int64_t n, const ViewParams* views,
                        const uint32_t* sorted_val, const uint32_t* offsets,
                        const uint32_t* chunk_cnt, const Footprint* foot,
                        const uint64_t* sat, uint32_t* out_key, uint32_t* out_val,
                        unsigned long long* counters, cudaStream_t stream);
// Count, scan and emit of sorted positions [p0, p0 + n_pos) in one launch
// (decoupled look-back).  Entries at positions >= capacity are not written;
// *total (device) receives the entry count.  lookback: bin_fused_temp_bytes
// of scratch (cleared by the launcher).
cudaError_t launch_bin_fused(int64_t p0, int64_t n_pos, int64_t n, const ViewParams* views,
                             const uint32_t* sorted_val, const Footprint* foot,
                             const uint64_t* sat, uint32_t* out_key, uint32_t* out_val,
                             uint32_t capacity, void* lookback, uint32_t* total,
                             unsigned long long* counters, cudaStream_t stream,
                             const int64_t* range_dev = nullptr);
size_t bin_fused_temp_bytes(int64_t n_pos);
// Polls of a predecessor's look-back word before the wait gives up (about 2 s).
constexpr int kLookbackSpinLimit = 1 << 26;
// Diagnostic: the fused binning on one block whose predecessor never
// publishes, with a wait bound of spin_limit polls (lookback: 512 B, total:
// one word, counters: kNumCounters; the other arrays need one element each).
cudaError_t launch_lookback_probe(void* lookback, uint32_t* total, unsigned long long* counters,
                                  const ViewParams* views, const uint32_t* sorted_val,
                                  const Footprint* foot, const uint64_t* sat, uint32_t* out_key,
                                  uint32_t* out_val, int spin_limit, cudaStream_t stream);
// Each view's prefix table of unsaturated tiles (ViewParams::free_tab, where
// set) from the batch's saturation bits: one block per view.
cudaError_t launch_free_tables(const ViewParams* views, int n_views, const uint64_t* sat,
                               cudaStream_t stream);
cudaError_t launch_ranges(int64_t n_entries, const uint32_t* key, uint2* ranges,
                          cudaStream_t stream, const uint32_t* n_dev = nullptr);

// Captured solves (fs_graph.cu) ----------------------------------------------
// Device-side sizes for a solve captured into a CUDA graph: no host readback.
// bnd[0 .. chunks] = the depth-chunk boundaries over the batch's visible slots
// (key_range[2], valid when key_range[0] <= key_range[1]).
cudaError_t launch_chunk_bounds(const uint32_t* key_range, int chunks, int64_t* bnd,
                                cudaStream_t stream);
// bound[ci] = the last sorted slot of chunk ci < chunks - 1 (0xFFFFFFFF: empty)
cudaError_t launch_chunk_last(const int64_t* bnd, int chunks, const uint32_t* sorted_val,
                              uint32_t* bound, cudaStream_t stream);
// dst[k] = src[k] for k < min(*n_dev, cap)
cudaError_t launch_copy_count(const uint32_t* src, uint32_t* dst, const uint32_t* n_dev,
                              int64_t cap, cudaStream_t stream);
// counts kGraphOverflow when *total > capacity or the range rng[0 .. 1] holds
// more than rng_cap positions, and kGraphKeyRange when the visible depth keys
// need more than key_bits bits (each pointer may be NULL: no check)
cudaError_t launch_graph_check(const uint32_t* total, uint32_t capacity,
                               const uint32_t* key_range, int key_bits, const int64_t* rng,
                               int64_t rng_cap, unsigned long long* counters,
                               cudaStream_t stream);

// blend / accumulate (fs_blend.cu) ------------------------------------------
// mask_dtype: 4 = uint8, 5 = int32.  table_dtype: 0 = f32, 1 = f64.
// state: per-pixel transmittance of the batch, scaled by 2^126 / 255 (0 =
// stopped).  sat / subsat:
// bit arrays over the batch's tile ids / 4 * tile id + sub-tile: set = every
// pixel of the tile / 8x8 sub-tile stopped (cleared by the caller before
// state_init).
cudaError_t launch_state_init(const ViewParams* views, int n_views, int max_tiles_per_view, int E,
                              int mask_dtype, float* state, uint64_t* sat, uint64_t* subsat,
                              unsigned long long* counters, cudaStream_t stream);
// sat_chunk (may be NULL): per batch tile, set to `chunk` when the tile
// saturates during this launch (its later chunks get no list entries).
// Records: float pairs in rec, or reduced precision in rec16.
// census: also count the evaluated (pixel, Gaussian) pairs (kPairs) and the
// pairs that take part in the compositing, alpha >= 1/255 up to and
// including the pixel's stop (kCensusPairs) -- a slower variant.
cudaError_t launch_blend(const ViewParams* views, int n_views, int max_tiles_per_view,
                         const uint2* ranges, const uint32_t* list_val, const ProjRecord* rec,
                         const CompactRecord* rec16, int64_t n, int E, int mask_dtype,
                         void* table, int table_dtype, float* state, uint64_t* sat,
                         uint64_t* subsat, uint8_t* sat_chunk, int chunk,
                         unsigned long long* counters, bool census, cudaStream_t stream);

// assignment (fs_assign.cu) -------------------------------------------------
cudaError_t launch_assign(const void* table, int table_dtype, int64_t n, int E, float gamma,
                          uint64_t* member_bits, int32_t* label, float* margin,
                          cudaStream_t stream);

// Object removal (Sec. 4.4): flag[i] = no bit of `remove` set in member_bits[i];
// keep[offs[i]] = i for flagged i (offs: exclusive scan of flag).
cudaError_t launch_keep_flags(int64_t n, const uint64_t* member_bits, uint64_t remove,
                              uint32_t* flag, cudaStream_t stream);
cudaError_t launch_keep_scatter(int64_t n, const uint32_t* flag, const uint32_t* offs,
                                int32_t* keep, cudaStream_t stream);

// dst[i] = (float) src[i], i < count
cudaError_t launch_round_table(int64_t count, const double* src, float* dst, cudaStream_t stream);
// Table rows re-decided from FP64 rows R[n_rows][E] (row j is Gaussian F[j]):
// the table row is overwritten with R's (rounded to table_dtype).
cudaError_t launch_assign_rows(const double* R, const uint32_t* F, int64_t n_rows, int E,
                               float gamma, void* table, int table_dtype, uint64_t* member_bits,
                               int32_t* label, float* margin, cudaStream_t stream);

// FP64 near-tie re-check (fs_recheck.cu) -------------------------------------
// flag[i] = margin[i] < tau
cudaError_t launch_flag_margin(int64_t n, const float* margin, float tau, uint32_t* flag,
                               cudaStream_t stream);
// F[offs[i]] = i and map[i] = offs[i] for flagged i; map[i] = -1 otherwise
cudaError_t launch_scatter_flagged(int64_t n, const uint32_t* flag, const uint32_t* offs,
                                   uint32_t* F, int32_t* map, cudaStream_t stream);
// clears the skip bits of every tile a flagged Gaussian reaches in the batch;
// *visible += the number of visible (view, flagged Gaussian) pairs.  With
// kept chunk lists (bound: the last slot of each depth chunk; dkey / dlo: the
// batch's depth keys and low words; sat_chunk: the chunk in which each tile
// saturated, 0xFF = never), sets the `deep` bit of every tile that saturated
// before the flagged Gaussian's own chunk.  bound == NULL: no kept lists.
cudaError_t launch_mark_tiles(int64_t n_flagged, int n_views, int64_t n, const uint32_t* F,
                              const ViewParams* views, const uint32_t* cnt, const Footprint* foot,
                              uint64_t* skip, uint32_t* visible, const uint32_t* bound,
                              int chunks, const uint32_t* dkey, const uint32_t* dlo,
                              const uint8_t* sat_chunk, uint64_t* deep, cudaStream_t stream);
// dst[i] += src[i], i < count
cudaError_t launch_add_rows(int64_t count, const double* src, double* dst, cudaStream_t stream);
// flag[slot] = the slot's footprint reaches an unskipped tile
cudaError_t launch_candidates(int64_t k_total, int64_t n, const ViewParams* views,
                              const uint32_t* cnt, const Footprint* foot, const uint64_t* skip,
                              uint32_t* flag, cudaStream_t stream);
// (out_key, out_val)[offs[slot]] = (key_src[slot], slot) for flagged slots
cudaError_t launch_compact(int64_t k_total, const uint32_t* flag, const uint32_t* offs,
                           const uint32_t* key_src, uint32_t* out_key, uint32_t* out_val,
                           cudaStream_t stream);
// Depth-ordered tile lists for the re-check: `chunks` consecutive depth
// chunks, each with its list values and per-batch-tile ranges; sat_chunk and
// deep as in launch_mark_tiles (NULL when the lists are complete).
constexpr int kMaxChunks = 16;
struct RecheckLists {
  const uint32_t* val[kMaxChunks];
  const uint2* ranges[kMaxChunks];
  int chunks;
  const uint8_t* sat_chunk;
  const uint64_t* deep;
  // the re-checked Gaussians (n_flagged of them) and the batch's per-slot
  // visibility: a deep tile walks only the pixels one of them can reach
  // (NULL: every labelled pixel of a deep tile)
  const uint32_t* flagged;
  int n_flagged;
  const uint32_t* cnt;
};
// Float-pair compositing of the tiles whose skip bit is clear; adds alpha*T of
// Gaussian i (map[i] >= 0) at a pixel of label e into R[map[i] * E + e].
cudaError_t launch_recheck_blend(const ViewParams* views, int n_views, int max_tiles_per_view,
                                 const RecheckLists& lists, const uint64_t* skip,
                                 const ProjRecord* rec, const CompactRecord* rec16,
                                 const float4* pos_op, int64_t n, int E, int mask_dtype,
                                 const int32_t* map, double* R, unsigned long long* counters,
                                 cudaStream_t stream);

// Novel-view mask rendering (fs_render.cu) ----------------------------------
// Per-view outputs of the mask renderer: the mask (FS_U8 / FS_I32, H x W),
// and optionally rho^e and D^e for objects e = 1 .. E-1 ((E-1) x H x W FP32).
struct RenderOut {
  void* mask;
  float* rho;
  float* depth;
};
// flag[k] = 1 iff sorted slot k is visible (cnt != 0) and member[slot % n] & bit
cudaError_t launch_member_select(int64_t k_total, int64_t n, const uint32_t* sorted_val,
                                 const uint32_t* cnt, const uint64_t* member, uint64_t bit,
                                 uint32_t* flag, cudaStream_t stream);
// out[offs[k]] = sorted_val[k] for flagged k (order kept)
cudaError_t launch_member_scatter(int64_t k_total, const uint32_t* flag, const uint32_t* offs,
                                  const uint32_t* sorted_val, uint32_t* out, cudaStream_t stream);
// Object e's tile lists composited per pixel and folded into the masks:
// rho^e > tau and D^e below best[] (per batch pixel, at state_off) takes label
// e; first != 0 starts every pixel at label 0 and best = +inf.
cudaError_t launch_render(const ViewParams* views, const RenderOut* outs, int n_views,
                          int max_tiles_per_view, const uint2* ranges, const uint32_t* list_val,
                          const ProjRecord* rec, const CompactRecord* rec16, int e, bool first,
                          float tau, float* best, int out_dtype, cudaStream_t stream);

// Context workspace management for the request server (fs_api.cu).
size_t ctx_workspace_bytes(const fs_ctx* c);
void ctx_release_workspace(fs_ctx* c);
void ctx_set_batching(fs_ctx* c, int views_per_batch, int depth_chunks);

// View parameters of a camera (fs_api.cu): float pairs of R, t and the
// intrinsics, near plane 0.2, Jacobian clamp 1.3 tan(half field of view),
// tile counts; tile_base, state_off and mask are left zero.
void fill_view(const fs_camera& cam, ViewParams* vp);

// Sets the calling thread's fs_last_error() message (fs_api.cu).
void set_last_error(const char* msg);

// device counters (unsigned long long) written by the kernels
enum Counter {
  kBadLabels = 0,
  kPairs = 1,
  kStaged = 2,
  kBinningMismatch = 3,
  kRecheckPairs = 4,
  kRecheckIncomplete = 5,
  kCensusPairs = 6,
  kLookbackTimeout = 7,
  kRounds = 8,           // census: compositing rounds of the blend
  kSteps = 9,            // census: staging steps of the blend (per block)
  kRoundsMixed = 10,     // census: rounds of warps with more than one label
  kRoundsSlots = 11,     // census: Gaussian slots of those rounds (sum of nq)
  kGraphOverflow = 12,   // a captured solve's lists outgrew the capture's plan
  kGraphKeyRange = 13,   // a captured solve's depth keys outgrew the plan's sort bits
  kNumCounters = 14
};

}  // namespace fs
