/*
 * flashsplat.h -- C ABI of the GB300 FlashSplat library (libflashsplat.so).
 *
 * FlashSplat (arXiv 2409.08270) segments a reconstructed 3D Gaussian Splatting
 * scene from 2D label masks in one pass: every mask pixel of every view is
 * alpha-composited through the scene (Sec. 3.1, Eq. 1), each Gaussian's
 * alpha_i*T_i is accumulated into the column of the pixel's label (Sec. 3.2,
 * Eq. 6; Sec. 3.3, Eq. 7; Supp. Sec. 6: the table A in R^{E x N}), and the
 * optimal label per Gaussian is the closed-form biased argmax of its row
 * (Sec. 3.2 "Regularized ILP for Noise Reduction"; Sec. 3.3, Eq. 7).
 *
 * Conventions (fixed where the paper is silent):
 *   - Gaussian i: mean m_i (3), unit quaternion q_i = (w, x, y, z) (any
 *     non-zero norm; normalised inside), linear scales s_i (3, > 0),
 *     activated opacity o_i in [0, 1].  Sigma3D = R(q) diag(s^2) R(q)^T.
 *   - Camera: world->camera rotation R (row-major 3x3) and translation t,
 *     OpenCV axes (x right, y down, z forward), pinhole fx, fy, cx, cy.
 *     Pixel (u, v) is sampled at (u + 0.5, v + 0.5).
 *   - EWA projection, +0.3 px^2 on the 2D covariance diagonal; Gaussians with
 *     view depth <= 0.2 or opacity < 1/255 are culled.
 *   - alpha = min(0.99, o exp(-0.5 d^T Sigma2D^-1 d)); alpha < 1/255 is
 *     skipped; a pixel stops before a Gaussian that would take T below 1e-4.
 *   - Depth order: view-space z of the mean, ties by lower Gaussian index.
 *   - Table layout: Gaussian-major, element (i, e) at index i*E + e.
 *
 * Threading and streams: a context is bound to one device.  Calls on one
 * context must not run concurrently from several host threads.  Work is
 * enqueued on the caller's CUDA stream (cudaStream_t passed as void*; NULL =
 * legacy default stream) and is asynchronous unless stated otherwise;
 * fs_synchronize() waits for it and reports device-side errors.
 *
 * Errors: every call returns an fs_status; no C++ exception crosses the ABI.
 * fs_last_error() returns a message for the calling thread's last failure.
 */
#ifndef FLASHSPLAT_H
#define FLASHSPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FS_VERSION_MAJOR 0
#define FS_VERSION_MINOR 1

typedef enum fs_status {
  FS_OK = 0,
  FS_INVALID_ARGUMENT = 1, /* bad pointer, size, dtype, zero quaternion, ... */
  FS_OUT_OF_MEMORY = 2,    /* a device or pinned-host allocation failed */
  FS_CUDA_ERROR = 3,       /* a CUDA runtime call or kernel failed */
  FS_TIMEOUT = 4,          /* a bounded device-side wait gave up */
  FS_UNSUPPORTED = 5,      /* valid request outside what this build handles */
  FS_CANCELLED = 6
} fs_status;

typedef enum fs_dtype {
  FS_F32 = 0,
  FS_F64 = 1,
  FS_BF16 = 2,
  FS_F16 = 3,
  FS_U8 = 4,
  FS_I32 = 5
} fs_dtype;

typedef enum fs_memory {
  FS_MEM_HOST = 0,   /* host memory (pinned memory makes copies asynchronous) */
  FS_MEM_DEVICE = 1  /* device memory on the context's device */
} fs_memory;

typedef struct fs_ctx fs_ctx;
typedef struct fs_scene fs_scene;

/* Context options.  Zero-initialise and set what you need; 0 = default. */
typedef struct fs_options {
  int32_t views_per_batch;  /* views binned and blended per launch group (default 50, at most 64) */
  int32_t time_stages;      /* non-zero: time every stage (FS_STAGE_*) with CUDA events */
  int32_t depth_chunks;     /* front-to-back binning chunks per batch (default 6, 1 = off) */
  /* fs_solve re-evaluates in FP64 every Gaussian whose FP32 decision margin
   * (see fs_assign) is below this value (default 1e-4 when 0; negative = off).
   * The FP32 table's entries are within ~1e-5 relative of exact, which moves
   * a margin by at most ~2e-5; 1e-4 leaves a factor of five.
   * Larger values re-check more Gaussians; a value above every margin
   * re-renders every seen Gaussian's contributions in FP64. */
  float recheck_margin;
  /* 0: keep each view's projection resident for the re-check when device
   * memory allows (about 108 B per Gaussian and view), else project again;
   * 1: always project again. */
  int32_t recheck_reproject;
  /* 0: per-view projected records in float pairs (64 B); FS_F16: the
   * reduced-precision form -- each (view, Gaussian) keeps its projected mean
   * in FP32 and its whitening matrix W (|W d|^2 = 0.5 log2(e) d^T
   * Sigma2D^-1 d) in FP16 (a 32 B record with the opacity and its alpha
   * cut), and alpha = o 2^-|W (p - m)|^2 is evaluated from those rounded
   * values (blending in FP32, table in FP64). */
  int32_t record_precision;
  /* non-zero: the blend also counts, in fs_stats.pairs and
   * fs_stats.census_pairs, the (pixel, Gaussian) pairs it evaluates and the
   * pairs that take part in the compositing (alpha >= 1/255, reached before
   * the pixel stops, the stopping one included).  A slower variant, for
   * measurement; the results are the same. */
  int32_t census;
  /* Which pixels a Gaussian reaches (FS_COVERAGE_*).  FS_COVERAGE_EXACT
   * (0): every pixel where alpha >= 1/255 can hold, so the result does not
   * depend on the tile size.  FS_COVERAGE_3SIGMA: only the pixels of the
   * 16x16 tiles that the square of half side r = ceil(3 sqrt(lambda_max))
   * around the projected mean overlaps (tiles floor((mx - r) / 16) ..
   * ceil((mx + r) / 16) - 1 in x, likewise in y), the coverage of the
   * standard 3D-GS rasteriser that Sec. 4.2 builds on; lambda_max is the
   * larger eigenvalue of the 2D covariance with its 0.3 px^2 low-pass.  The
   * radius and the tiles are decided in FP32 from the FP32-rounded
   * covariance and mean: r = ceil(3 sqrt(m + sqrt(h^2 + b^2))), m = (a + c)
   * / 2, h = (a - c) / 2, every step rounded to nearest. */
  int32_t coverage;
  int32_t reserved[8];
} fs_options;

enum { FS_COVERAGE_EXACT = 0, FS_COVERAGE_3SIGMA = 1 };

/* A Gaussian scene (Sec. 3.1: G_i = {m_i, q_i, s_i, o_i}; colour unused). */
typedef struct fs_gaussians {
  int64_t n;             /* number of Gaussians, 0 <= n < 2^31 */
  const void* mean;      /* [n][3] FS_F32 */
  const void* quat;      /* [n][4] (w, x, y, z), FS_F32 or FS_BF16 */
  const void* scale;     /* [n][3] linear scales, FS_F32 or FS_BF16 */
  const void* opacity;   /* [n] activated opacity, FS_F32 or FS_F16 */
  int32_t quat_dtype;
  int32_t scale_dtype;
  int32_t opacity_dtype;
  int32_t memory;        /* fs_memory of all four arrays */
} fs_gaussians;

/* A pinhole camera (world -> camera). */
typedef struct fs_camera {
  double R[9];           /* row-major rotation */
  double t[3];
  double fx, fy, cx, cy;
  int32_t width, height; /* mask size in pixels, each in [1, 65535] */
} fs_camera;

/* Counters of the last fs_accumulate / fs_solve on a context. */
typedef struct fs_stats {
  int64_t views;           /* views processed */
  int64_t pixels;          /* mask pixels walked */
  int64_t list_entries;    /* (tile, Gaussian) pairs binned, summed over views */
  int64_t bad_labels;      /* pixels whose label was outside [0, E) (skipped) */
  int64_t pairs;           /* (pixel, Gaussian) pairs evaluated by the blend (census only) */
  int64_t kernel_launches; /* kernels launched by the library */
  double blend_ms;         /* summed blend time (= stage_ms[FS_STAGE_BLEND]) */
  int64_t blend_launches;  /* blend launches timed */
  int64_t staged_entries;  /* list entries the blend staged before its tiles saturated */
  int64_t rechecked;       /* Gaussians re-evaluated in FP64 by fs_solve */
  int64_t recheck_pairs;   /* (pixel, list entry) pairs the re-check evaluated */
  int64_t recheck_rebinned;/* view batches the re-check binned anew (see fs_solve) */
  int64_t census_pairs;    /* pairs with alpha >= 1/255 reached before the pixel's
                              stop, the stop included (census only) */
  int64_t census_rounds;   /* blend: compositing rounds of a warp (census only) */
  int64_t census_steps;    /* blend: list-staging steps of a block (census only) */
  int64_t census_rounds_mixed; /* blend: rounds of warps whose pixels carry more
                              than one label (census only) */
  double stage_ms[8];      /* summed device time per stage, indexed by FS_STAGE_*
                              (fs_options.time_stages, uncaptured work), else 0 */
} fs_stats;

/* Stages of a solve timed under fs_options.time_stages (fs_stats.stage_ms):
 * the projection of every Gaussian into a view batch, the batch's depth
 * sort with its tie fix, the pixel-state set-up, the tile binning of each
 * depth chunk, its tile sort and ranges, the blend, the near-tie re-check,
 * and the assignment with the table's rounding.  A batch projected on the
 * side stream while the previous batch blends is timed on that stream, so
 * the stages can add up to more than the solve. */
enum {
  FS_STAGE_PROJECT = 0,
  FS_STAGE_DEPTH_SORT = 1,
  FS_STAGE_PIXEL_STATE = 2,
  FS_STAGE_BINNING = 3,
  FS_STAGE_TILE_SORT = 4,
  FS_STAGE_BLEND = 5,
  FS_STAGE_RECHECK = 6,
  FS_STAGE_ASSIGN = 7,
  FS_NUM_STAGES = 8
};

/* Outputs of fs_solve.  Any pointer may be NULL to skip that output. */
typedef struct fs_result {
  int32_t memory;         /* fs_memory of every output below */
  int32_t table_dtype;    /* FS_F32 or FS_F64: element type of `table` */
  void* table;            /* [n][E] contribution table A (Gaussian-major) */
  uint64_t* member_bits;  /* [n] bit e set iff S[e, i] = 1 (needs E <= 64) */
  int32_t* label;         /* [n] the unique e with S[e, i] = 1, else -1 */
  float* margin;          /* [n] min over e of the relative decision margin */
} fs_result;

/* Version as MAJOR*1000 + MINOR. */
int32_t fs_version(void);

/* Message for the calling thread's most recent failed call ("" if none).
 * The pointer stays valid until the next failing call on the same thread. */
const char* fs_last_error(void);

/* Create a context on CUDA device `device`.  opt may be NULL.  The library
 * owns the context and its device workspace; release with fs_destroy.
 * Errors: FS_INVALID_ARGUMENT (out NULL, device out of range),
 * FS_UNSUPPORTED (device is not compute capability 10.3), FS_CUDA_ERROR. */
fs_status fs_create(fs_ctx** out, int32_t device, const fs_options* opt);

/* Destroy a context (waits for its outstanding work).  NULL is a no-op.
 * Scenes created on it must be destroyed first. */
fs_status fs_destroy(fs_ctx* ctx);

/* Make a scene resident on the context's device (Sec. 3.1, Sec. 4.2: only
 * {m, q, s, o} are used).  Any context on the same device may use the scene
 * (read-only) while it lives.  The library copies the arrays into its own device
 * storage (quaternions normalised, the 3D covariance precomputed in FP64);
 * the caller may free its buffers when the call returns (the call is
 * synchronous).  Errors: FS_INVALID_ARGUMENT (NULL pointers, n out of
 * range, dtype not allowed for the field, a zero quaternion, a non-finite
 * value), FS_OUT_OF_MEMORY, FS_CUDA_ERROR. */
fs_status fs_scene_create(fs_ctx* ctx, const fs_gaussians* g, fs_scene** out);

/* Free a scene's device storage (waits for work that uses it).  NULL is a
 * no-op. */
fs_status fs_scene_destroy(fs_scene* scene);

/* Number of Gaussians in a scene (0 for NULL). */
int64_t fs_scene_size(const fs_scene* scene);

/*
 * fs_accumulate -- add the contributions of n_views masks to a table
 * (Sec. 3.2 Eq. 6, Sec. 3.3 Eq. 7, Sec. 4.2, Supp. Sec. 6):
 *
 *   table[i*E + e] += sum_{v, pixels p with M^v_p = e} alpha_i(p) T_i(p)
 *
 * cams[n_views]: host array.  masks[n_views]: host array of pointers, view
 * v's labels row-major [cams[v].height][cams[v].width], element type
 * mask_dtype (FS_U8 or FS_I32), in mask_memory (FS_MEM_HOST or
 * FS_MEM_DEVICE).  Pixels whose label is outside [0, E) are skipped and
 * counted in fs_stats.bad_labels.  E in [1, 4096].
 * table: device memory [n][E] of table_dtype (FS_F32, or FS_F64 for the
 * FP64 cross-view reduction), NOT cleared: contributions are added, so a
 * solve can be split over several calls (view subsets) and resumed.
 * Host masks are copied on `stream` and must stay valid until the stream
 * reaches the end of the call.  Asynchronous.
 * Errors: FS_INVALID_ARGUMENT, FS_OUT_OF_MEMORY (workspace growth),
 * FS_CUDA_ERROR.
 */
fs_status fs_accumulate(fs_ctx* ctx, const fs_scene* scene, const fs_camera* cams,
                        int32_t n_views, const void* const* masks, int32_t mask_dtype,
                        int32_t mask_memory, int32_t E, void* table, int32_t table_dtype,
                        void* stream);

/*
 * fs_assign -- closed-form optimal labels from a contribution table
 * (Sec. 3.2: L1-normalise, add the background bias gamma to the background
 * entry, argmax; Sec. 3.3 Eq. 7: object e against "others" = sum of every
 * other column; Supp. Sec. 6: segmentation matrix S in {0,1}^{E x N}).
 *
 * For every Gaussian i and label e, with S_i = sum_e A[i, e]:
 *   member(e, i)  <=>  A[i,e]/n_i  >  (S_i - A[i,e])/n_i + gamma,
 *   n_i = max(|S_i - A[i,e]| + |A[i,e]|, 1e-12)   (a tie is not a member).
 * gamma in [-1, 1].  table: device [n][E] of table_dtype (FS_F32 / FS_F64).
 * Outputs (device, each may be NULL): member_bits[n] (needs E <= 64),
 * label[n] (the unique member e, else -1), margin[n]
 * (min_e |(1-gamma) A[i,e] - (1+gamma)(S_i - A[i,e])| / S_i; +inf if
 * S_i = 0).  Asynchronous.  Errors: FS_INVALID_ARGUMENT, FS_UNSUPPORTED
 * (member_bits with E > 64), FS_CUDA_ERROR.
 */
fs_status fs_assign(fs_ctx* ctx, const void* table, int32_t table_dtype, int64_t n, int32_t E,
                    float gamma, uint64_t* member_bits, int32_t* label, float* margin,
                    void* stream);

/*
 * fs_solve -- the whole path: clear a table, fs_accumulate all views, then
 * fs_assign with gamma (Sec. 3.2-3.3), then re-check near ties.  The blend
 * runs in FP32, so a Gaussian whose decision margin is within the table's
 * FP32 error of zero (relative error ~1e-5) could be labelled differently
 * from an exact evaluation.  Every Gaussian whose margin is below
 * fs_options.recheck_margin is therefore re-evaluated: every pixel its
 * footprint reaches, in every view, is composited again front to back at
 * about 1e-11 relative precision (float-pair arithmetic: alpha, T, the 1/255
 * and 1e-4 decisions; FP64 sums), its table row is replaced by those sums
 * (rounded to the table's type) and its bits/label/margin are decided again
 * from them in FP64.  The depth-ordered tile lists of the main pass are kept
 * for this when device memory allows (about 4 B per list entry); a view
 * batch whose kept lists end before an exact walk does is binned anew
 * (counted in fs_stats.recheck_rebinned).
 * The table itself is accumulated in FP64 (the cross-view sum of Eq. 6/7: a
 * Gaussian seen in many views collects up to ~1e5 additions, too many for
 * FP32 at 1e-5) and rounded once to out->table_dtype.
 * Outputs go where `out` says (out->memory: device buffers, or host buffers
 * filled by asynchronous copies on `stream` -- pinned host memory keeps them
 * asynchronous).  When out->table is NULL the table lives in the context's
 * workspace.  The call reads counts back between steps and so returns after
 * the device work is queued; call fs_synchronize before reading host
 * outputs.  Errors: as fs_accumulate and fs_assign.
 */
fs_status fs_solve(fs_ctx* ctx, const fs_scene* scene, const fs_camera* cams, int32_t n_views,
                   const void* const* masks, int32_t mask_dtype, int32_t mask_memory, int32_t E,
                   float gamma, const fs_result* out, void* stream);

/*
 * fs_keep_after_removal -- object removal (Sec. 4.4): the Gaussians left when
 * every Gaussian of the selected objects' subsets {G_i}_e is deleted from the
 * scene.  member_bits: device [n], bit e set iff S[e, i] = 1 (the output of
 * fs_solve / fs_assign; the paper assigns with gamma = -0.4 for removal so
 * that the subsets reach into the object's boundary).  remove: bit e set =
 * object e is removed.  keep_index: device int32 [n]; receives the kept
 * Gaussians' indices in increasing order (its first *n_keep entries).
 * n_keep: host.  The call waits for the count (it synchronises `stream`).
 * Errors: FS_INVALID_ARGUMENT, FS_OUT_OF_MEMORY, FS_CUDA_ERROR.
 */
fs_status fs_keep_after_removal(fs_ctx* ctx, const uint64_t* member_bits, int64_t n,
                                uint64_t remove, int32_t* keep_index, int64_t* n_keep,
                                void* stream);

/* Wait for the context's work on `stream` and report errors recorded by its
 * kernels: FS_TIMEOUT when a bounded device-side wait gave up (the tile
 * binning's wait for a preceding block's offset, about 2 s per poll
 * sequence; that solve's lists are then incomplete), FS_CUDA_ERROR for an
 * internal inconsistency.  Fills *stats if non-NULL. */
fs_status fs_synchronize(fs_ctx* ctx, void* stream, fs_stats* stats);

/* Diagnostic (no counterpart in the paper): runs the tile binning's
 * decoupled look-back on one block whose predecessor never publishes its
 * offset, with the wait bounded at `spins` polls (>= 1), on `device`, and
 * returns FS_TIMEOUT when the bounded wait gives up as it must -- FS_OK would
 * mean the bound is not enforced.  Synchronous; allocates a few hundred
 * bytes of device memory for the duration of the call. */
fs_status fs_check_wait_timeout(int32_t device, int32_t spins);

/* Test hooks (no counterpart in the paper): the library's own primitives on
 * caller-owned device buffers, so that tests can check each one alone
 * against a plain CPU result.  Synchronous on `device`; each call allocates
 * its temporary device storage for its own duration.  FS_INVALID_ARGUMENT for
 * a bad device, NULL array with n > 0, or a size out of range.
 *
 * fs_test_sort_pairs: stable sort, in place, of n (key, val) pairs (two
 *   device arrays of n uint32, n < 2^31) by key, for keys below 2^bits
 *   (1 <= bits <= 32; the passes take whole 8- or 9-bit digits, so bits
 *   above `bits` must be zero): the radix sort that orders the depth keys
 *   and the tile ids of the binning (Sec. 4.2's tile lists).
 * fs_test_exclusive_scan: out[k] = in[0] + ... + in[k - 1] (mod 2^32) over
 *   n device uint32 (n < 2^31); *total (host) = the sum of all n.
 * fs_test_tile_ranges: for n keys in non-decreasing order (device uint32,
 *   each < n_tiles, checked on the host), ranges (device, n_tiles pairs of
 *   uint32) receives per tile t the run [first, last + 1) of key t, and
 *   [0, 0) for a tile without an entry. */
fs_status fs_test_sort_pairs(int32_t device, uint32_t* keys, uint32_t* vals, int64_t n,
                             int32_t bits);
fs_status fs_test_exclusive_scan(int32_t device, const uint32_t* in, uint32_t* out, int64_t n,
                                 uint32_t* total);
fs_status fs_test_tile_ranges(int32_t device, const uint32_t* keys, int64_t n, int32_t n_tiles,
                              uint32_t* ranges);

/* ---- request server (continuous batching) -----------------------------------
 * Segmentation requests against resident scenes, served by `slots` workers
 * that each own a context and a CUDA stream.  A request (scene, cameras,
 * host masks, E, gamma) is queued on submission; a free slot admits the
 * oldest queued request whose estimated device footprint fits beside the
 * requests already running (budget_bytes), so requests that arrive while
 * others run start as soon as a slot and memory free up, and their work
 * overlaps on the device.  Each request is an fs_solve (Sec. 3.2-3.3,
 * near-tie re-check included) on the slot's stream.  The paper has no
 * serving layer; this is the batching pattern the solve is deployed with.
 */
typedef struct fs_server fs_server;

typedef struct fs_server_options {
  int32_t device;         /* CUDA device */
  int32_t slots;          /* concurrent requests (default 4) */
  int64_t budget_bytes;   /* device bytes the running requests may use
                             (default: half the free memory at creation) */
  int32_t autotune;       /* non-zero: the first request of each scene also
                             times a few (views per batch, depth chunks)
                             settings on a sample of its views and keeps the
                             fastest for the scene's later requests */
  int32_t graphs;         /* > 0: requests run as replays of captured solves
                             (fs_graph_*), one per scene for its last
                             (cameras, E, gamma, mask dtype), at most `graphs`
                             scenes kept (least recently used dropped);
                             a request with a new key captures its scene
                             again.  0: plain fs_solve per request */
  int32_t reserved[8];
} fs_server_options;

/* Outcome and timing of one request (steady-clock seconds). */
typedef struct fs_server_info {
  int32_t status;         /* fs_status of the request's solve */
  int32_t done;           /* 1 once finished (or cancelled) */
  double submit_s;        /* when fs_server_submit accepted it */
  double start_s;         /* when a slot admitted it */
  double done_s;          /* when its results were on the host */
  int32_t slot;           /* the slot that ran it */
  int32_t views_per_batch, depth_chunks;  /* the settings it ran with */
  int32_t pad;
  int64_t bytes_estimate; /* the footprint admission used */
  fs_stats stats;         /* the solve's counters */
} fs_server_info;

/* Create a server (threads start immediately).  Errors: FS_INVALID_ARGUMENT,
 * FS_UNSUPPORTED (device), FS_OUT_OF_MEMORY, FS_CUDA_ERROR. */
fs_status fs_server_create(const fs_server_options* opt, fs_server** out);

/* Make a scene resident for the server's requests (as fs_scene_create);
 * *scene_id identifies it in fs_server_submit.  Thread-safe. */
fs_status fs_server_add_scene(fs_server* srv, const fs_gaussians* g, int32_t* scene_id);

/* Queue a request.  cams[n_views] and the host masks (row-major H x W,
 * FS_U8 or FS_I32) are copied before the call returns.  *ticket identifies
 * the request.  Thread-safe.  Errors: FS_INVALID_ARGUMENT (bad scene id,
 * cameras, dtype, E or gamma). */
fs_status fs_server_submit(fs_server* srv, int32_t scene_id, const fs_camera* cams,
                           int32_t n_views, const void* const* masks, int32_t mask_dtype,
                           int32_t E, float gamma, int64_t* ticket);

/* Results of a request: wait != 0 blocks until it is done; otherwise
 * FS_TIMEOUT is returned while it is still queued or running.  Copies the
 * scene's n member bits / labels / margins into the caller's host buffers
 * (each may be NULL; member_bits needs E <= 64), fills *info (may be NULL)
 * and forgets the request.  Returns the request's own status once done. */
fs_status fs_server_fetch(fs_server* srv, int64_t ticket, int32_t wait, uint64_t* member_bits,
                          int32_t* label, float* margin, fs_server_info* info);

/* fs_server_fetch with a bounded wait: blocks at most timeout_ms milliseconds
 * (0: not at all; negative: until done) and returns FS_TIMEOUT, leaving the
 * request in place, if it has not finished by then. */
fs_status fs_server_fetch_for(fs_server* srv, int64_t ticket, int32_t timeout_ms,
                              uint64_t* member_bits, int32_t* label, float* margin,
                              fs_server_info* info);

/* Drop a request that has not started (FS_CANCELLED when fetched);
 * FS_UNSUPPORTED if it is already running or done. */
fs_status fs_server_cancel(fs_server* srv, int64_t ticket);

/* Stop accepting requests, finish the running ones, drop the queued ones,
 * join the threads and free everything. */
fs_status fs_server_destroy(fs_server* srv);

/* ---- captured solves (CUDA graph) -------------------------------------------
 * fs_graph_create captures one solve of (scene, cams, masks, E, gamma) into a
 * CUDA graph that fs_graph_launch replays with a single launch on any stream:
 * the whole accumulation (projection, depth sort, binning, blending, the
 * FP64 cross-view sum) and the assignment, with no host synchronisation
 * inside.  It first runs the solve once uncaptured on a context of its own
 * (the options of `ctx`, without timing or census) to fix the solve's shapes:
 * the depth-sort bits of each view batch, the sorted positions each depth
 * chunk spans and its list entries; the capture then reads every count from
 * device memory and sizes its grids and lists for that plan.  After the
 * replay, fs_graph_launch runs the near-tie re-check (when the options turn
 * it on; its work depends on the labels) on a second context of the graph's
 * own, projecting the views again (nothing may move the captured buffers),
 * and rounds the table to FP32 when asked, outside the graph.
 *   masks[V]: device buffers, read at every replay: the caller may write new
 *     masks into them between replays.  With every label in [0, E) the
 *     shapes depend on the scene and cameras only, so any such masks replay
 *     exactly; a replay whose shapes outgrow the plan (possible only if the
 *     scene's device memory changed) is not run past it and reports
 *     FS_UNSUPPORTED at fs_graph_synchronize.
 *   out: device buffers, written by every replay.
 * The scene must outlive the graph; one replay at a time per graph.  The
 * FP64 table of a replay equals an uncaptured fs_solve's up to the order of
 * the FP64 atomic additions (any two solves differ in the same way).
 * Errors: as fs_solve; FS_INVALID_ARGUMENT for host outputs or masks. */
typedef struct fs_graph fs_graph;
fs_status fs_graph_create(fs_ctx* ctx, const fs_scene* scene, const fs_camera* cams,
                          int32_t n_views, const void* const* masks, int32_t mask_dtype,
                          int32_t E, float gamma, const fs_result* out, fs_graph** graph);
fs_status fs_graph_launch(fs_graph* graph, void* stream);
/* Waits for `stream` and reports the replay's device-side errors, as
 * fs_synchronize does for a context. */
fs_status fs_graph_synchronize(fs_graph* graph, void* stream, fs_stats* stats);
fs_status fs_graph_destroy(fs_graph* graph);

/* ---- novel-view masks -------------------------------------------------------
 * fs_render_masks: 2D masks for views -- typically ones that had no mask --
 * from a segmentation (Sec. 3.4 "depth-guided novel view mask rendering";
 * Supp. Sec. 8.2 on why the quantisation is needed).  Object e = 1 .. E-1 is
 * the subset {G_i}_e = {i : bit e of member_bits[i] set} (fs_solve's S); each
 * is rendered on its own with the solve's rules (Eq. 1 over its Gaussians
 * only, FP32): rho^e = sum alpha T, and its depth D^e = sum alpha T z /
 * rho^e with z the view-space depth of each Gaussian's mean (0 where rho^e
 * is 0).  A pixel's mask value is the object with rho^e > tau of smallest
 * D^e, equal depths to the smaller e, and 0 where no object passes.  With
 * E = 2 this is the binary mask [rho^1 > tau]; Sec. 4.6 uses tau = 0.1.
 * Coverage follows the context's fs_options.coverage.
 *   member_bits: n words in device memory (bit e: object e)
 *   masks_out[v]: device buffer of H x W values, out_dtype FS_U8 or FS_I32
 *   rho_out[v], depth_out[v]: NULL (the array or an entry), or device buffers
 *     of (E-1) x H x W FP32 receiving rho^e and D^e, object-major
 * Synchronises `stream` once per view batch and object (list sizes).  Errors:
 * FS_INVALID_ARGUMENT (NULL arguments, bad cameras, E outside [2, 64], tau
 * NaN, bad dtype), FS_OUT_OF_MEMORY, FS_CUDA_ERROR. */
fs_status fs_render_masks(fs_ctx* ctx, const fs_scene* scene, const fs_camera* cams,
                          int32_t n_views, const uint64_t* member_bits, int32_t E, float tau,
                          void* const* masks_out, int32_t out_dtype, float* const* rho_out,
                          float* const* depth_out, void* stream);

/* ---- solve without allocating ----------------------------------------------
 * The paper has no counterpart of this call; it exists for callers that may
 * not allocate device memory -- e.g. a plugin inside an application that owns
 * all device memory through its own pool, or a latency-critical loop that
 * cannot afford cudaMalloc/cudaFree, which may synchronise the whole device.
 *
 * fs_solve_noalloc renders and accumulates like fs_solve and assigns with the
 * same rule, for small scenes, without a context and without allocating
 * anything.  Two differences from fs_solve: the views are summed with FP32
 * atomics straight into the caller's FP32 table (no FP64 cross-view
 * reduction), and there is no near-tie re-check -- so a Gaussian whose
 * decision margin is within the FP32 table's error (about 1e-5 relative) may
 * be labelled differently from fs_solve.  Pixels whose label is outside
 * [0, E) are skipped, as in fs_solve, but not counted anywhere.  Coverage is
 * always FS_COVERAGE_EXACT.  Its working
 * memory is a fixed array of about 13 MB in the library's device memory that
 * every GPU loading the library holds until the process exits.  Limits:
 * 1..FS_NOALLOC_MAX_GAUSSIANS Gaussians, views of at most FS_NOALLOC_MAX_SIDE
 * pixels per side, at most FS_NOALLOC_MAX_LIST_ENTRIES (tile, Gaussian) pairs
 * per view and depth chunk; larger inputs are rejected (FS_INVALID_ARGUMENT,
 * or FS_UNSUPPORTED when the pair count is exceeded mid-solve, after which the
 * table is incomplete).
 *   device: CUDA device to run on.  g: FS_F32 attributes in device memory.
 *   cams[n_views], masks[n_views]: host arrays; masks point to device
 *   memory (FS_U8 or FS_I32).  table: device [n][E] FP32, overwritten.
 *   member_bits / label / margin: device outputs as in fs_assign (each may
 *   be NULL).  stream: the caller's stream (NULL = legacy default stream).
 * The first call on a device looks up the array's device address once (make
 * that first call before any stream capture).  The call returns after the
 * work has completed (it reads counts back between steps).  All calls share
 * the one array, which keeps the previous call's contents (what must start
 * at zero is cleared on every call); calls whose work overlaps on the GPU --
 * from several host threads or on several streams -- race and must not be
 * made.  Errors are reported like every other call (fs_last_error). */
#define FS_NOALLOC_MAX_GAUSSIANS 16384
#define FS_NOALLOC_MAX_SIDE 512
#define FS_NOALLOC_MAX_LIST_ENTRIES (1 << 19)
fs_status fs_solve_noalloc(int32_t device, const fs_gaussians* g, const fs_camera* cams,
                           int32_t n_views, const void* const* masks, int32_t mask_dtype,
                           int32_t E, float gamma, float* table, uint64_t* member_bits,
                           int32_t* label, float* margin, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FLASHSPLAT_H */
