// Host runtime of libflashsplat: contexts, resident scenes, the batched
// per-view pipeline (project -> depth sort -> scan -> emit -> tile sort ->
// ranges -> blend), the assignment, and the C ABI of include/flashsplat.h.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/flashsplat.h"
#include "fs_common.cuh"
#include "fs_internal.h"

struct fs_ctx;

namespace {

thread_local char g_last_error[512] = "";

fs_status fail(fs_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return st;
}

fs_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(FS_OUT_OF_MEMORY, "%s: %s", what, cudaGetErrorString(e));
  return fail(FS_CUDA_ERROR, "%s: %s", what, cudaGetErrorString(e));
}

#define FS_CUDA(expr, what)                      \
  do {                                           \
    cudaError_t e_ = (expr);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

#define FS_TRY(expr)                 \
  do {                               \
    fs_status s_ = (expr);           \
    if (s_ != FS_OK) return s_;      \
  } while (0)

// Keeps the caller's current device and restores it on scope exit.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// A growable device allocation.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  fs_status ensure(size_t need, const char* what) {
    if (need <= bytes) return FS_OK;
    size_t want = std::max(need, static_cast<size_t>(bytes + bytes / 4));  // grow geometrically
    if (p) {
      cudaFree(p);
      p = nullptr;
      bytes = 0;
    }
    want = (want + 255) & ~static_cast<size_t>(255);
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return fail(FS_OUT_OF_MEMORY, "cudaMalloc(%zu) for %s failed: %s", want, what,
                  cudaGetErrorString(e));
    }
    bytes = want;
    return FS_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

struct HostBuf {
  void* p = nullptr;
  size_t bytes = 0;
  fs_status ensure(size_t need) {
    if (need <= bytes) return FS_OK;
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMallocHost(&p, need);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return fail(FS_OUT_OF_MEMORY, "cudaMallocHost(%zu) failed", need);
    }
    bytes = need;
    return FS_OK;
  }
  void release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

size_t dtype_size(int dt) {
  switch (dt) {
    case FS_F32: return 4;
    case FS_F64: return 8;
    case FS_BF16: return 2;
    case FS_F16: return 2;
    case FS_U8: return 1;
    case FS_I32: return 4;
    default: return 0;
  }
}

void split(double x, float* hi, float* lo) {
  const float h = static_cast<float>(x);
  *hi = h;
  *lo = static_cast<float>(x - static_cast<double>(h));
}

int ceil_log2(int64_t x) {
  int b = 0;
  while ((static_cast<int64_t>(1) << b) < x) ++b;
  return b;
}

// kernels launched by exclusive_scan / radix_sort_pairs for n elements
int64_t scan_launches(int64_t n) { return n > 0 ? 3 : 0; }
int64_t radix_launches(int64_t n, int bits) {
  if (n <= 1 || bits <= 0) return 0;
  const int64_t nb = (n + 4095) / 4096;
  return static_cast<int64_t>(fs::radix_passes(bits)) * (2 + scan_launches(nb * 512));
}

}  // namespace

// Per-view parameters of a camera (float pairs of R, t and the intrinsics,
// the near plane, the Jacobian clamp at 1.3 tan(half field of view), tiles).
void fs::fill_view(const fs_camera& cam, fs::ViewParams* vp) {
  memset(vp, 0, sizeof(*vp));
  for (int k = 0; k < 9; ++k) split(cam.R[k], &vp->R_hi[k], &vp->R_lo[k]);
  for (int k = 0; k < 3; ++k) split(cam.t[k], &vp->t_hi[k], &vp->t_lo[k]);
  split(cam.fx, &vp->fx_hi, &vp->fx_lo);
  split(cam.fy, &vp->fy_hi, &vp->fy_lo);
  split(cam.cx, &vp->cx_hi, &vp->cx_lo);
  split(cam.cy, &vp->cy_hi, &vp->cy_lo);
  split(0.2, &vp->near_hi, &vp->near_lo);
  split(1.3 * (0.5 * cam.width / cam.fx), &vp->limx_hi, &vp->limx_lo);
  split(1.3 * (0.5 * cam.height / cam.fy), &vp->limy_hi, &vp->limy_lo);
  vp->width = cam.width;
  vp->height = cam.height;
  vp->tiles_x = (cam.width + fs::kTile - 1) / fs::kTile;
  vp->tiles_y = (cam.height + fs::kTile - 1) / fs::kTile;
}

void fs::set_last_error(const char* msg) {
  snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
}

struct fs_ctx {
  int device = 0;
  int views_per_batch = 50;
  int depth_chunks = 6;  // front-to-back chunks per batch (sizes 1/32, 1/32, 1/16, ..., 1/2)
  int n_sm = 0;
  bool time_stages = false;
  std::vector<cudaEvent_t> events;  // (start, stop) pairs around timed stages
  std::vector<int> event_stage;     // the stage (FS_STAGE_*) of each pair
  size_t events_used = 0;
  bool stage_outer = false;         // a stage holding others (the re-check) is open
  // workspace
  DevBuf views, rec, foot, cnt, key_a, val_a, key_b, val_b, offs, ccnt, dlo, state, sat, subsat;
  DevBuf free_tab;  // the batch's per-view prefix tables of unsaturated tiles
  DevBuf lk_a, lv_a, lk_b, lv_b, ranges, sort_tmp, scan_tmp, total, counters;
  DevBuf mask_stage, table_tmp, table32_tmp, bits_tmp, label_tmp, margin_tmp;
  // near-tie re-check: resident per-view depth keys, flagged set, FP64 rows
  float recheck_margin = 1e-4f;  // <= 0: off
  bool recheck_reproject = false;
  bool compact = false;  // reduced-precision records (FP16 whitening matrix, FP32 mean)
  bool census = false;   // blend counts its pairs (slower variant)
  bool sigma3 = false;   // 3-sigma tile coverage (per-slot tile columns in `cols`)
  DevBuf dkey, rk_flag, rk_offs, rk_F, rk_map, rk_R, rk_Rb, cols;
  DevBuf rd_flag, rd_offs, rd_val, render_out;  // novel-view mask rendering
  DevBuf chunk_bnd;                             // captured solves: chunk boundaries
  HostBuf render_out_host;
  DevBuf key_range;  // min / max visible depth key of the batch (two slots, by batch parity)
  // the next batch's projection runs on a side stream while the current
  // batch bins and blends (resident projections only); its depth keys go to
  // the second set of sort buffers
  DevBuf key_a2, val_a2, key_b2, val_b2;
  cudaStream_t side = nullptr;
  cudaEvent_t prologue_done[2] = {nullptr, nullptr}, buffers_free = nullptr;
  DevBuf lb_tmp;     // look-back words of the fused binning
  // the main pass's tile lists, kept for the re-check (see kept_layout)
  bool kl_valid = false;
  int kl_chunks = 1;
  std::vector<DevBuf> kl_val;
  std::vector<int64_t> kl_tile_off;
  DevBuf kl_ranges, kl_satc, kl_bound;
  std::vector<const void*> mask_dev;  // device pointer of every view's mask (last solve)
  HostBuf views_host, total_host, counters_host;
  fs_stats stats{};
  int scenes = 0;
};

struct fs_scene {
  fs_ctx* ctx = nullptr;
  int64_t n = 0;
  DevBuf pos_op, cov;  // (m, o) and Sigma3D as float pairs
};

namespace {
DevBuf* const* workspace_bufs(fs_ctx* c, size_t* count) {
  static thread_local DevBuf* bufs[64];
  size_t k = 0;
  DevBuf* list[] = {&c->rec, &c->foot, &c->cnt, &c->key_a, &c->val_a, &c->key_b, &c->val_b,
                    &c->offs, &c->ccnt, &c->dlo, &c->state, &c->sat, &c->subsat, &c->lk_a,
                    &c->lv_a, &c->lk_b, &c->lv_b, &c->ranges, &c->sort_tmp, &c->scan_tmp,
                    &c->mask_stage, &c->table_tmp, &c->table32_tmp, &c->bits_tmp,
                    &c->label_tmp, &c->margin_tmp, &c->dkey, &c->rk_flag, &c->rk_offs,
                    &c->rk_F, &c->rk_map, &c->rk_R, &c->rk_Rb, &c->kl_ranges, &c->kl_satc,
                    &c->kl_bound, &c->key_range, &c->lb_tmp, &c->key_a2, &c->val_a2,
                    &c->key_b2, &c->val_b2, &c->cols, &c->rd_flag, &c->rd_offs, &c->rd_val,
                    &c->render_out, &c->chunk_bnd, &c->free_tab};
  for (DevBuf* b : list) bufs[k++] = b;
  *count = k;
  return bufs;
}
}  // namespace

// Device bytes the context's growable workspace holds now.
size_t fs::ctx_workspace_bytes(const fs_ctx* c) {
  size_t count = 0, total = 0;
  DevBuf* const* b = workspace_bufs(const_cast<fs_ctx*>(c), &count);
  for (size_t k = 0; k < count; ++k) total += b[k]->bytes;
  for (const DevBuf& v : c->kl_val) total += v.bytes;
  return total;
}

// Frees the growable workspace (after the context's work has finished).
void fs::ctx_release_workspace(fs_ctx* c) {
  DeviceGuard g(c->device);
  cudaDeviceSynchronize();
  size_t count = 0;
  DevBuf* const* b = workspace_bufs(c, &count);
  for (size_t k = 0; k < count; ++k) b[k]->release();
  for (DevBuf& v : c->kl_val) v.release();
  c->kl_valid = false;
}

// Per-solve batching (views per batch, depth chunks), as fs_options sets them.
void fs::ctx_set_batching(fs_ctx* c, int views_per_batch, int depth_chunks) {
  if (views_per_batch > 0) c->views_per_batch = std::min(views_per_batch, fs::kMaxViewsPerBatch);
  if (depth_chunks > 0) c->depth_chunks = std::min(depth_chunks, 16);
}

extern "C" {

int32_t fs_version(void) { return FS_VERSION_MAJOR * 1000 + FS_VERSION_MINOR; }

const char* fs_last_error(void) { return g_last_error; }

fs_status fs_create(fs_ctx** out, int32_t device, const fs_options* opt) {
  if (!out) return fail(FS_INVALID_ARGUMENT, "fs_create: out is NULL");
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= count)
    return fail(FS_INVALID_ARGUMENT, "fs_create: device %d out of range [0, %d)", device, count);
  cudaDeviceProp prop;
  FS_CUDA(cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties");
  if (!(prop.major == 10 && prop.minor == 3))
    return fail(FS_UNSUPPORTED, "fs_create: device %d is sm_%d%d; this build targets sm_103a",
                device, prop.major, prop.minor);
  fs_ctx* c = new (std::nothrow) fs_ctx();
  if (!c) return fail(FS_OUT_OF_MEMORY, "fs_create: host allocation failed");
  c->device = device;
  c->n_sm = prop.multiProcessorCount;
  if (opt && opt->views_per_batch > 0)
    c->views_per_batch = std::min(opt->views_per_batch, fs::kMaxViewsPerBatch);
  c->time_stages = opt && opt->time_stages;
  if (opt && opt->depth_chunks > 0) c->depth_chunks = std::min(opt->depth_chunks, 16);
  if (opt && opt->recheck_margin != 0.f)
    c->recheck_margin = opt->recheck_margin > 0.f ? opt->recheck_margin : 0.f;
  if (opt && !(opt->recheck_margin == opt->recheck_margin))
    c->recheck_margin = 0.f;  // NaN: off
  c->recheck_reproject = opt && opt->recheck_reproject;
  if (opt && opt->record_precision != 0 && opt->record_precision != FS_F16) {
    delete c;
    return fail(FS_INVALID_ARGUMENT, "fs_create: record_precision must be 0 or FS_F16");
  }
  c->compact = opt && opt->record_precision == FS_F16;
  if (opt && opt->coverage != FS_COVERAGE_EXACT && opt->coverage != FS_COVERAGE_3SIGMA) {
    delete c;
    return fail(FS_INVALID_ARGUMENT, "fs_create: coverage must be FS_COVERAGE_EXACT or "
                                     "FS_COVERAGE_3SIGMA");
  }
  c->sigma3 = opt && opt->coverage == FS_COVERAGE_3SIGMA;
  c->census = opt && opt->census;
  DeviceGuard g(device);
  fs_status st;
  if ((st = c->views.ensure(sizeof(fs::ViewParams) * 2 * fs::kMaxViewsPerBatch, "views")) != FS_OK ||
      (st = c->views_host.ensure(sizeof(fs::ViewParams) * 2 * fs::kMaxViewsPerBatch)) != FS_OK ||
      (st = c->total.ensure(256, "total")) != FS_OK ||
      (st = c->total_host.ensure(256)) != FS_OK ||
      (st = c->counters.ensure(sizeof(unsigned long long) * fs::kNumCounters, "counters")) != FS_OK ||
      (st = c->counters_host.ensure(sizeof(unsigned long long) * fs::kNumCounters)) != FS_OK) {
    delete c;
    return st;
  }
  cudaMemset(c->counters.p, 0, c->counters.bytes);
  *out = c;
  return FS_OK;
}

fs_status fs_destroy(fs_ctx* c) {
  if (!c) return FS_OK;
  if (c->scenes > 0)
    return fail(FS_INVALID_ARGUMENT, "fs_destroy: %d scene(s) still alive", c->scenes);
  DeviceGuard g(c->device);
  cudaDeviceSynchronize();
  DevBuf* bufs[] = {&c->subsat, &c->ccnt, &c->dlo, &c->state, &c->sat, &c->views, &c->rec, &c->foot, &c->cnt, &c->key_a, &c->val_a, &c->key_b,
                    &c->val_b, &c->offs, &c->lk_a, &c->lv_a, &c->lk_b, &c->lv_b, &c->ranges,
                    &c->sort_tmp, &c->scan_tmp, &c->total, &c->counters, &c->mask_stage,
                    &c->table_tmp, &c->table32_tmp, &c->bits_tmp, &c->label_tmp, &c->margin_tmp,
                    &c->dkey, &c->rk_flag, &c->rk_offs, &c->rk_F, &c->rk_map, &c->rk_R,
                    &c->rk_Rb, &c->kl_ranges, &c->kl_satc, &c->kl_bound, &c->key_range, &c->lb_tmp,
                    &c->key_a2, &c->val_a2, &c->key_b2, &c->val_b2, &c->cols,
                    &c->rd_flag, &c->rd_offs, &c->rd_val, &c->render_out, &c->chunk_bnd,
                    &c->free_tab};
  for (DevBuf& b : c->kl_val) b.release();
  for (DevBuf* b : bufs) b->release();
  c->views_host.release();
  c->render_out_host.release();
  c->total_host.release();
  c->counters_host.release();
  for (cudaEvent_t e : c->events) cudaEventDestroy(e);
  for (cudaEvent_t e : c->prologue_done)
    if (e) cudaEventDestroy(e);
  if (c->buffers_free) cudaEventDestroy(c->buffers_free);
  if (c->side) cudaStreamDestroy(c->side);
  delete c;
  return FS_OK;
}

fs_status fs_scene_create(fs_ctx* c, const fs_gaussians* g, fs_scene** out) {
  if (!c || !g || !out) return fail(FS_INVALID_ARGUMENT, "fs_scene_create: NULL argument");
  *out = nullptr;
  const int64_t n = g->n;
  if (n < 0 || n >= (static_cast<int64_t>(1) << 31))
    return fail(FS_INVALID_ARGUMENT, "fs_scene_create: n = %lld out of range", (long long)n);
  if (n > 0 && (!g->mean || !g->quat || !g->scale || !g->opacity))
    return fail(FS_INVALID_ARGUMENT, "fs_scene_create: NULL attribute pointer");
  if (!(g->quat_dtype == FS_F32 || g->quat_dtype == FS_BF16) ||
      !(g->scale_dtype == FS_F32 || g->scale_dtype == FS_BF16) ||
      !(g->opacity_dtype == FS_F32 || g->opacity_dtype == FS_F16))
    return fail(FS_INVALID_ARGUMENT, "fs_scene_create: unsupported attribute dtype");
  if (g->memory != FS_MEM_HOST && g->memory != FS_MEM_DEVICE)
    return fail(FS_INVALID_ARGUMENT, "fs_scene_create: bad memory kind %d", g->memory);
  DeviceGuard guard(c->device);
  fs_scene* s = new (std::nothrow) fs_scene();
  if (!s) return fail(FS_OUT_OF_MEMORY, "fs_scene_create: host allocation failed");
  s->ctx = c;
  s->n = n;
  const size_t nn = static_cast<size_t>(n > 0 ? n : 1);
  fs_status st;
  if ((st = s->pos_op.ensure(nn * 16, "scene")) != FS_OK ||
      (st = s->cov.ensure(nn * 48, "scene")) != FS_OK) {
    s->pos_op.release(); s->cov.release();
    delete s;
    return st;
  }
  const size_t b_mean = nn * 12, b_quat = nn * 4 * dtype_size(g->quat_dtype);
  const size_t b_scale = nn * 3 * dtype_size(g->scale_dtype);
  const size_t b_op = nn * dtype_size(g->opacity_dtype);
  DevBuf stage;
  const void *dm = g->mean, *dq = g->quat, *ds = g->scale, *dop = g->opacity;
  cudaError_t e = cudaSuccess;
  if (n > 0 && g->memory == FS_MEM_HOST) {
    st = stage.ensure(b_mean + b_quat + b_scale + b_op + 64 * 4, "scene staging");
    if (st != FS_OK) {
      s->pos_op.release(); s->cov.release();
      delete s;
      return st;
    }
    char* base = stage.as<char>();
    size_t o1 = (b_mean + 63) & ~63ull, o2 = o1 + ((b_quat + 63) & ~63ull);
    size_t o3 = o2 + ((b_scale + 63) & ~63ull);
    e = cudaMemcpy(base, g->mean, b_mean, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + o1, g->quat, b_quat, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + o2, g->scale, b_scale, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + o3, g->opacity, b_op, cudaMemcpyHostToDevice);
    dm = base; dq = base + o1; ds = base + o2; dop = base + o3;
  }
  unsigned int* d_err = c->total.as<unsigned int>();
  if (e == cudaSuccess) e = cudaMemset(d_err, 0, sizeof(unsigned int));
  if (e == cudaSuccess)
    e = fs::launch_scene_prep(n, static_cast<const float*>(dm), dq, g->quat_dtype, ds,
                              g->scale_dtype, dop, g->opacity_dtype, s->pos_op.as<float4>(),
                              s->cov.as<float4>(), d_err, nullptr);
  unsigned int h_err = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h_err, d_err, sizeof(h_err), cudaMemcpyDeviceToHost);
  stage.release();
  if (e != cudaSuccess) {
    s->pos_op.release(); s->cov.release();
    delete s;
    return cuda_fail(e, "fs_scene_create");
  }
  if (h_err) {
    s->pos_op.release(); s->cov.release();
    delete s;
    return fail(FS_INVALID_ARGUMENT,
                "fs_scene_create: a Gaussian has a zero quaternion or a non-finite attribute");
  }
  c->scenes++;
  *out = s;
  return FS_OK;
}

fs_status fs_scene_destroy(fs_scene* s) {
  if (!s) return FS_OK;
  DeviceGuard g(s->ctx->device);
  cudaDeviceSynchronize();
  s->pos_op.release();
  s->cov.release();
  s->ctx->scenes--;
  delete s;
  return FS_OK;
}

int64_t fs_scene_size(const fs_scene* s) { return s ? s->n : 0; }

}  // extern "C"

namespace {

fs_status check_camera(const fs_camera& cam, int v) {
  for (int k = 0; k < 9; ++k)
    if (!isfinite(cam.R[k])) return fail(FS_INVALID_ARGUMENT, "camera %d: non-finite R", v);
  for (int k = 0; k < 3; ++k)
    if (!isfinite(cam.t[k])) return fail(FS_INVALID_ARGUMENT, "camera %d: non-finite t", v);
  // R must be a rotation: R R^T = I
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double d = 0;
      for (int k = 0; k < 3; ++k) d += cam.R[3 * a + k] * cam.R[3 * b + k];
      if (fabs(d - (a == b ? 1.0 : 0.0)) > 1e-5)
        return fail(FS_INVALID_ARGUMENT, "camera %d: R is not orthonormal", v);
    }
  if (!(cam.fx > 0 && cam.fy > 0 && isfinite(cam.fx) && isfinite(cam.fy) && isfinite(cam.cx) &&
        isfinite(cam.cy)))
    return fail(FS_INVALID_ARGUMENT, "camera %d: bad intrinsics", v);
  if (cam.width < 1 || cam.height < 1 || cam.width > 65535 || cam.height > 65535)
    return fail(FS_INVALID_ARGUMENT, "camera %d: size %dx%d out of range", v, cam.width, cam.height);
  return FS_OK;
}

// Per-view mask device pointers for views [0, V).  Host masks are staged in
// one buffer that holds every view, so a later pass can read them again.
fs_status stage_masks(fs_ctx* c, const fs_camera* cams, int32_t V, const void* const* masks,
                      int32_t mask_dtype, int32_t mask_memory, cudaStream_t stream) {
  const size_t msize = dtype_size(mask_dtype);
  c->mask_dev.assign(V, nullptr);
  if (mask_memory == FS_MEM_DEVICE) {
    for (int v = 0; v < V; ++v) c->mask_dev[v] = masks[v];
    return FS_OK;
  }
  size_t total = 0;
  for (int v = 0; v < V; ++v)
    total += ((static_cast<size_t>(cams[v].width) * cams[v].height * msize) + 255) & ~size_t(255);
  FS_TRY(c->mask_stage.ensure(total > 0 ? total : 256, "mask staging"));
  size_t off = 0;
  for (int v = 0; v < V; ++v) {
    const size_t mbytes = static_cast<size_t>(cams[v].width) * cams[v].height * msize;
    char* dst = c->mask_stage.as<char>() + off;
    FS_CUDA(cudaMemcpyAsync(dst, masks[v], mbytes, cudaMemcpyHostToDevice, stream), "mask upload");
    c->mask_dev[v] = dst;
    off += (mbytes + 255) & ~size_t(255);
  }
  return FS_OK;
}

// The view parameters of views [v0, v0 + nb), written to the host array vh.
// fs_options.time_stages (work that is not being captured): an event pair
// around one stage's launches on `strm`.  stage_begin gives the pair's index
// (-1 when not timing); stage_end closes the pair on the same stream.
fs_status stage_begin(fs_ctx* c, int stage, cudaStream_t strm, bool capturing, int* idx) {
  *idx = -1;
  if (!c->time_stages || capturing || c->stage_outer) return FS_OK;
  while (c->events.size() < c->events_used + 2) {
    cudaEvent_t e;
    FS_CUDA(cudaEventCreate(&e), "cudaEventCreate");
    c->events.push_back(e);
  }
  const size_t pair = c->events_used / 2;
  if (c->event_stage.size() <= pair) c->event_stage.resize(pair + 1);
  c->event_stage[pair] = stage;
  *idx = static_cast<int>(c->events_used);
  c->events_used += 2;
  FS_CUDA(cudaEventRecord(c->events[*idx], strm), "cudaEventRecord");
  return FS_OK;
}

fs_status stage_end(fs_ctx* c, int idx, cudaStream_t strm) {
  if (idx >= 0) FS_CUDA(cudaEventRecord(c->events[idx + 1], strm), "cudaEventRecord");
  return FS_OK;
}

struct BatchLayout {
  int total_tiles = 0;
  int max_tiles = 0;
  int64_t pixels = 0;
};

// Cells of the prefix tables of views [v0, v0 + nb): (tiles_x + 1) x
// (tiles_y + 1) per view.
int64_t free_cells(const fs_camera* cams, int32_t v0, int nb) {
  int64_t cells = 0;
  for (int k = 0; k < nb; ++k) {
    const int64_t tx = (cams[v0 + k].width + fs::kTile - 1) / fs::kTile;
    const int64_t ty = (cams[v0 + k].height + fs::kTile - 1) / fs::kTile;
    cells += (tx + 1) * (ty + 1);
  }
  return cells;
}

// Sizes the prefix tables for the largest batch of the solve once, before
// any batch is laid out, so that no batch's tables move while another
// batch's work is queued.
fs_status ensure_free_tabs(fs_ctx* c, const fs_camera* cams, int32_t V, int vb) {
  int64_t most = 1;
  for (int32_t v0 = 0; v0 < V; v0 += vb)
    most = std::max(most, free_cells(cams, v0, std::min(vb, V - v0)));
  return c->free_tab.ensure(static_cast<size_t>(most) * 4, "tile prefix tables");
}

BatchLayout layout_batch(fs_ctx* c, fs::ViewParams* vh, const fs_camera* cams, int32_t v0,
                         int nb, uint32_t* cols) {
  BatchLayout L;
  // the prefix tables, where ensure_free_tabs made room (else the binning
  // walks the saturation bits)
  const bool tabs = c->free_tab.bytes >= static_cast<size_t>(free_cells(cams, v0, nb)) * 4;
  int64_t cell = 0;
  for (int k = 0; k < nb; ++k) {
    fs::fill_view(cams[v0 + k], &vh[k]);
    vh[k].cols = cols;
    vh[k].free_tab = tabs ? c->free_tab.as<uint32_t>() + cell : nullptr;
    cell += static_cast<int64_t>(vh[k].tiles_x + 1) * (vh[k].tiles_y + 1);
    vh[k].tile_base = L.total_tiles;
    vh[k].state_off = L.pixels;
    vh[k].mask = c->mask_dev[v0 + k];
    const int nt = vh[k].tiles_x * vh[k].tiles_y;
    L.total_tiles += nt;
    L.max_tiles = std::max(L.max_tiles, nt);
    L.pixels += static_cast<int64_t>(cams[v0 + k].width) * cams[v0 + k].height;
  }
  return L;
}

// Views per batch: (view, Gaussian) slots of one batch must fit in 31 bits.
int batch_views(const fs_ctx* c, int64_t n) {
  const int64_t max_vb = ((static_cast<int64_t>(1) << 31) - 1) / n;
  return static_cast<int>(std::min<int64_t>(c->views_per_batch, max_vb));
}

// Projection storage of a batch: either the batch window (slot = view in
// batch * n + i) or, when `keep` is set, the slice of a buffer that holds
// every view of the solve, so the near-tie re-check can read it again.
struct ProjPtrs {
  fs::ProjRecord* rec;       // float-pair records, or NULL
  fs::CompactRecord* rec16;  // reduced-precision records, or NULL
  fs::Footprint* foot;
  uint32_t* cnt;
  uint32_t* dlo;
  uint32_t* dkey;  // resident depth keys (keep only)
  uint32_t* cols;  // 3-sigma tile columns, or NULL (exact coverage)
};

ProjPtrs proj_ptrs(const fs_ctx* c, bool keep, int32_t v0, int64_t n) {
  const int64_t off = keep ? static_cast<int64_t>(v0) * n : 0;
  return {c->compact ? nullptr : c->rec.as<fs::ProjRecord>() + off,
          c->compact ? c->rec.as<fs::CompactRecord>() + off : nullptr,
          c->foot.as<fs::Footprint>() + off,
          c->cnt.as<uint32_t>() + off, c->dlo.as<uint32_t>() + off,
          keep ? c->dkey.as<uint32_t>() + off : nullptr,
          c->sigma3 ? c->cols.as<uint32_t>() + off : nullptr};
}

fs_status ensure_window(fs_ctx* c, int64_t n, int vb, int32_t V, bool keep) {
  const int64_t kcap = static_cast<int64_t>(vb) * n;
  const int64_t pcap = keep ? static_cast<int64_t>(V) * n : kcap;
  const size_t rec_bytes = c->compact ? sizeof(fs::CompactRecord) : sizeof(fs::ProjRecord);
  FS_TRY(c->rec.ensure(static_cast<size_t>(pcap) * rec_bytes, "records"));
  FS_TRY(c->foot.ensure(static_cast<size_t>(pcap) * sizeof(fs::Footprint), "footprints"));
  FS_TRY(c->cnt.ensure(static_cast<size_t>(pcap) * 4, "counts"));
  FS_TRY(c->dlo.ensure(static_cast<size_t>(pcap) * 4, "depth low words"));
  if (keep) FS_TRY(c->dkey.ensure(static_cast<size_t>(pcap) * 4, "depth keys"));
  if (c->sigma3) FS_TRY(c->cols.ensure(static_cast<size_t>(pcap) * 4, "tile columns"));
  FS_TRY(c->key_a.ensure(static_cast<size_t>(kcap) * 4, "keys"));
  FS_TRY(c->val_a.ensure(static_cast<size_t>(kcap) * 4, "vals"));
  FS_TRY(c->key_b.ensure(static_cast<size_t>(kcap) * 4, "keys"));
  FS_TRY(c->val_b.ensure(static_cast<size_t>(kcap) * 4, "vals"));
  FS_TRY(c->offs.ensure(static_cast<size_t>(kcap) * 4, "offsets"));
  FS_TRY(c->scan_tmp.ensure(fs::scan_temp_bytes(kcap), "scan temp"));
  FS_TRY(c->sort_tmp.ensure(fs::radix_temp_bytes(kcap), "sort temp"));
  FS_TRY(c->ccnt.ensure(static_cast<size_t>(kcap) * 4, "chunk counts"));
  return FS_OK;
}

// Reads a device uint32 total back (synchronises the stream).
fs_status read_total(fs_ctx* c, cudaStream_t stream, int64_t* out) {
  uint32_t* total_h = c->total_host.as<uint32_t>();
  FS_CUDA(cudaMemcpyAsync(total_h, c->total.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream),
          "count readback");
  FS_CUDA(cudaStreamSynchronize(stream), "count readback");
  *out = *total_h;
  return FS_OK;
}

// Binning of sorted positions [p0, p0 + n_pos) into tile lists (count, scan,
// emit, stable tile sort, ranges) on tiles whose `sat` bit is clear.  The
// sorted list values go to *val_dst (grown as needed) and the per-tile ranges
// to ranges_dst.  Returns the entry count in *I_out.
//
// Captured form (range_dev != NULL): the chunk's positions are read on the
// device from range_dev[0 .. 1] (at most n_pos of them: the grid), nothing is
// read back, and the lists are sized for plan_cap entries (the capture's
// plan); a replay that outgrows either is counted (kGraphOverflow).
fs_status bin_positions(fs_ctx* c, int64_t p0, int64_t n_pos, int64_t n,
                        const fs::ViewParams* vd, int nb, const uint32_t* sorted_val,
                        const ProjPtrs& P,
                        const uint64_t* sat, int total_tiles, int tile_bits, int64_t kcap,
                        bool count_entries, DevBuf* val_dst, uint2* ranges_dst,
                        cudaStream_t stream, int64_t* I_out, const int64_t* range_dev = nullptr,
                        int64_t plan_cap = 0) {
  unsigned long long* ctr = c->counters.as<unsigned long long>();
  *I_out = 0;
  FS_CUDA(cudaMemsetAsync(ranges_dst, 0, static_cast<size_t>(total_tiles) * 8, stream),
          "ranges clear");
  FS_TRY(c->lb_tmp.ensure(fs::bin_fused_temp_bytes(n_pos), "binning look-back"));
  // the views' prefix tables of the tiles still unsaturated
  FS_CUDA(fs::launch_free_tables(vd, nb, sat, stream), "tile prefix tables");
  if (range_dev) {
    uint32_t* total = c->total.as<uint32_t>();
    const uint32_t capacity = static_cast<uint32_t>(plan_cap);
    FS_CUDA(fs::launch_bin_fused(0, n_pos, n, vd, sorted_val, P.foot, sat, c->lk_a.as<uint32_t>(),
                                 val_dst->as<uint32_t>(), capacity, c->lb_tmp.p, total, ctr,
                                 stream, range_dev),
            "binning");
    FS_CUDA(fs::launch_graph_check(total, capacity, nullptr, 0, range_dev, n_pos, ctr, stream),
            "plan check");
    *I_out = plan_cap;
    if (plan_cap == 0) return FS_OK;
    bool alt2 = false;
    FS_CUDA(fs::radix_sort_pairs(c->lk_a.as<uint32_t>(), val_dst->as<uint32_t>(),
                                 c->lk_b.as<uint32_t>(), c->lv_b.as<uint32_t>(), plan_cap,
                                 tile_bits, c->sort_tmp.p, &alt2, stream, 0u, 0xFFFFFFFFu, total),
            "tile sort");
    const uint32_t* lkey = alt2 ? c->lk_b.as<uint32_t>() : c->lk_a.as<uint32_t>();
    if (alt2)
      FS_CUDA(fs::launch_copy_count(c->lv_b.as<uint32_t>(), val_dst->as<uint32_t>(), total,
                                    plan_cap, stream),
              "list copy");
    FS_CUDA(fs::launch_ranges(plan_cap, lkey, ranges_dst, stream, total), "ranges");
    return FS_OK;
  }
  // count, offsets and emission in one launch into the buffers' current
  // capacity; a chunk with more entries than fit runs again after growing
  int64_t I = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    const size_t cap_bytes = std::min(c->lk_a.bytes, val_dst->bytes);
    const uint32_t capacity = static_cast<uint32_t>(std::min<size_t>(cap_bytes / 4, 0x7FFFFFFFu));
    c->stats.kernel_launches += 1;
    int tb = -1;
    FS_TRY(stage_begin(c, FS_STAGE_BINNING, stream, false, &tb));
    FS_CUDA(fs::launch_bin_fused(p0, n_pos, n, vd, sorted_val, P.foot, sat,
                                 c->lk_a.as<uint32_t>(), val_dst->as<uint32_t>(), capacity,
                                 c->lb_tmp.p, c->total.as<uint32_t>(), ctr, stream),
            "binning");
    FS_TRY(stage_end(c, tb, stream));
    FS_TRY(read_total(c, stream, &I));
    if (I >= (static_cast<int64_t>(1) << 31))
      return fail(FS_UNSUPPORTED, "%lld list entries in one chunk; use fewer views per batch",
                  (long long)I);
    if (I <= static_cast<int64_t>(capacity)) break;
    FS_TRY(c->lk_a.ensure(static_cast<size_t>(I) * 4, "list keys"));
    FS_TRY(val_dst->ensure(static_cast<size_t>(I) * 4, "list values"));
  }
  if (count_entries) c->stats.list_entries += I;
  *I_out = I;
  if (I == 0) return FS_OK;
  FS_TRY(c->lk_b.ensure(static_cast<size_t>(I) * 4, "list keys"));
  FS_TRY(c->lv_b.ensure(static_cast<size_t>(I) * 4, "list values"));
  FS_TRY(c->sort_tmp.ensure(fs::radix_temp_bytes(std::max<int64_t>(I, kcap)), "sort temp"));
  c->stats.kernel_launches += 1 + radix_launches(I, tile_bits);
  bool alt2 = false;
  int tt = -1;
  FS_TRY(stage_begin(c, FS_STAGE_TILE_SORT, stream, false, &tt));
  FS_CUDA(fs::radix_sort_pairs(c->lk_a.as<uint32_t>(), val_dst->as<uint32_t>(),
                               c->lk_b.as<uint32_t>(), c->lv_b.as<uint32_t>(), I, tile_bits,
                               c->sort_tmp.p, &alt2, stream),
          "tile sort");
  const uint32_t* lkey = alt2 ? c->lk_b.as<uint32_t>() : c->lk_a.as<uint32_t>();
  if (alt2)
    FS_CUDA(cudaMemcpyAsync(val_dst->p, c->lv_b.p, static_cast<size_t>(I) * 4,
                            cudaMemcpyDeviceToDevice, stream),
            "list copy");
  FS_CUDA(fs::launch_ranges(I, lkey, ranges_dst, stream), "ranges");
  FS_TRY(stage_end(c, tt, stream));
  return FS_OK;
}

// Front-to-back depth chunk boundaries of a batch of k_total sorted slots:
// chunk ci covers positions [chunk_begin(ci), chunk_begin(ci + 1)).
int64_t chunk_end(int64_t k_total, int chunks, int ci) {
  return (ci == chunks - 1) ? k_total : (k_total >> (chunks - 1 - ci));
}

// Layout of the main pass's tile lists kept for the near-tie re-check: per
// view batch and depth chunk, the list values and the ranges over the
// batch's tiles; per batch tile, the chunk in which it saturated; per batch
// and chunk, the last slot of the chunk.
fs_status kept_layout(fs_ctx* c, const fs_camera* cams, int32_t V, int vb, int chunks) {
  c->kl_tile_off.clear();
  int64_t tiles = 0;
  for (int32_t v0 = 0; v0 < V; v0 += vb) {
    c->kl_tile_off.push_back(tiles);
    const int nb = std::min(vb, V - v0);
    for (int k = 0; k < nb; ++k) {
      const int64_t tx = (cams[v0 + k].width + fs::kTile - 1) / fs::kTile;
      const int64_t ty = (cams[v0 + k].height + fs::kTile - 1) / fs::kTile;
      tiles += tx * ty;
    }
  }
  c->kl_tile_off.push_back(tiles);
  const size_t batches = c->kl_tile_off.size() - 1;
  c->kl_chunks = chunks;
  if (c->kl_val.size() < batches * chunks) c->kl_val.resize(batches * chunks);
  FS_TRY(c->kl_ranges.ensure(static_cast<size_t>(tiles) * chunks * 8 + 8, "kept ranges"));
  FS_TRY(c->kl_satc.ensure(static_cast<size_t>(tiles) + 8, "kept saturation chunks"));
  FS_TRY(c->kl_bound.ensure(batches * chunks * 4 + 4, "kept chunk bounds"));
  return FS_OK;
}

// The side stream of the batch overlap (created on first use, on the
// context's device, which is current here).
fs_status ensure_side_stream(fs_ctx* c) {
  if (c->side) return FS_OK;
  FS_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking), "side stream");
  return FS_OK;
}

fs_status ensure_prologue_events(fs_ctx* c) {
  for (cudaEvent_t& e : c->prologue_done)
    if (!e) FS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
  if (!c->buffers_free)
    FS_CUDA(cudaEventCreateWithFlags(&c->buffers_free, cudaEventDisableTiming), "cudaEventCreate");
  return FS_OK;
}

// The shapes of one solve, fixed for its captured replays (fs_graph_*): per
// view batch the depth-sort bits, per (batch, depth chunk) the sorted
// positions the chunk spans and its list entries, and the batches' views in
// pinned host memory (a replayed copy reads its source at replay time).
struct GraphPlan {
  std::vector<int> key_bits;      // [batch]
  std::vector<int64_t> npos;      // [batch * chunks + ci]
  std::vector<int64_t> entries;   // [batch * chunks + ci]
  int chunks = 0;
  HostBuf views;                  // [batch][kMaxViewsPerBatch]
};

// record != NULL: the solve's shapes are written to *record (a plan).
// plan != NULL: the solve is being captured: no host readback, no side
// stream, sizes from the plan and from device memory.
fs_status accumulate_impl(fs_ctx* c, const fs_scene* s, const fs_camera* cams, int32_t V,
                          const void* const* masks, int32_t mask_dtype, int32_t mask_memory,
                          int32_t E, void* table, int32_t table_dtype, bool keep,
                          cudaStream_t stream, GraphPlan* record = nullptr,
                          const GraphPlan* plan = nullptr) {
  const int64_t n = s->n;
  c->kl_valid = false;
  if (n == 0 || V == 0) return FS_OK;
  const int vb = batch_views(c, n);
  FS_TRY(ensure_free_tabs(c, cams, V, vb));
  if (vb < 1) return fail(FS_UNSUPPORTED, "fs_accumulate: scene too large");
  const int64_t kcap = static_cast<int64_t>(vb) * n;
  const int chunks = std::max(1, std::min(c->depth_chunks, fs::kMaxChunks));
  FS_TRY(ensure_window(c, n, vb, V, keep));
  FS_TRY(stage_masks(c, cams, V, masks, mask_dtype, mask_memory, stream));
  if (keep) FS_TRY(kept_layout(c, cams, V, vb, chunks));

  unsigned long long* ctr = c->counters.as<unsigned long long>();
  const int batches = static_cast<int>((V + vb - 1) / vb);
  // With every view's projection resident (keep), batch b + 1's projection
  // writes storage of its own: it is launched on a side stream as soon as
  // batch b is sorted and runs while batch b bins and blends.  Batches
  // alternate between two sets of depth-sort buffers, view arrays and
  // key-range slots (by parity).  Without the memory for the second set the
  // batches run one after another.
  bool overlap = keep && batches > 1 && !plan && !record;
  if (record) {
    record->key_bits.assign(batches, 0);
    record->npos.assign(static_cast<size_t>(batches) * chunks, 0);
    record->entries.assign(static_cast<size_t>(batches) * chunks, 0);
    record->chunks = chunks;
  }
  if (plan && (static_cast<int>(plan->key_bits.size()) != batches || plan->chunks != chunks))
    return fail(FS_INVALID_ARGUMENT, "captured solve: the plan does not match the inputs");
  // sized by the recording solve: nothing is allocated while capturing
  if (plan || record)
    FS_TRY(c->chunk_bnd.ensure(static_cast<size_t>(fs::kMaxChunks + 1) * 8, "chunk bounds"));
  if (overlap) {
    const size_t kb = static_cast<size_t>(kcap) * 4;
    overlap = ensure_side_stream(c) == FS_OK && c->key_a2.ensure(kb, "keys") == FS_OK &&
              c->val_a2.ensure(kb, "vals") == FS_OK && c->key_b2.ensure(kb, "keys") == FS_OK &&
              c->val_b2.ensure(kb, "vals") == FS_OK;
    cudaGetLastError();
  }
  FS_TRY(c->key_range.ensure(32, "depth key range"));
  struct Prologue {
    BatchLayout L;
    fs::ViewParams* vd = nullptr;  // the batch's views on the device
    uint32_t *key = nullptr, *val = nullptr, *key_alt = nullptr, *val_alt = nullptr;
    const uint32_t* krh = nullptr;  // depth-key range read back to the host
  };
  Prologue pro[2];
  // The buffer set of batch b: the two sets alternate only when the batches
  // overlap (the second set is allocated only then).
  auto parity = [overlap](int bb) { return overlap ? (bb & 1) : 0; };
  // Batch b's views go up, every Gaussian is projected into them and the
  // visible depth-key range is read back, all on `strm`;
  // prologue_done[parity(b)] marks the end.
  auto launch_prologue = [&](int bb, cudaStream_t strm) -> fs_status {
    const int q = parity(bb);
    const int32_t w0 = bb * vb;
    const int nbb = std::min(vb, V - w0);
    fs::ViewParams* vhq =
        plan ? plan->views.as<fs::ViewParams>() + static_cast<int64_t>(bb) * fs::kMaxViewsPerBatch
             : c->views_host.as<fs::ViewParams>() + q * fs::kMaxViewsPerBatch;
    Prologue& pr = pro[q];
    const ProjPtrs PP = proj_ptrs(c, keep, w0, n);
    pr.L = layout_batch(c, vhq, cams, w0, nbb, PP.cols);
    pr.vd = c->views.as<fs::ViewParams>() + q * fs::kMaxViewsPerBatch;
    pr.key = (q ? c->key_a2 : c->key_a).as<uint32_t>();
    pr.val = (q ? c->val_a2 : c->val_a).as<uint32_t>();
    pr.key_alt = (q ? c->key_b2 : c->key_b).as<uint32_t>();
    pr.val_alt = (q ? c->val_b2 : c->val_b).as<uint32_t>();
    uint32_t* krq = c->key_range.as<uint32_t>() + 4 * q;
    uint32_t* krhq = c->total_host.as<uint32_t>() + 4 + 4 * q;
    pr.krh = krhq;
    FS_CUDA(cudaMemcpyAsync(pr.vd, vhq, sizeof(fs::ViewParams) * nbb, cudaMemcpyHostToDevice,
                            strm),
            "view upload");
    // project every Gaussian into the batch's views; the depth sort then
    // takes only the bits in which the batch's visible depth keys differ
    FS_CUDA(cudaMemsetAsync(krq, 0xFF, 4, strm), "key range");
    FS_CUDA(cudaMemsetAsync(krq + 1, 0, 8, strm), "key range");
    c->stats.kernel_launches += 2;
    int tp = -1;
    FS_TRY(stage_begin(c, FS_STAGE_PROJECT, strm, plan != nullptr, &tp));
    FS_CUDA(fs::launch_project(n, nbb, pr.vd, s->pos_op.as<float4>(), s->cov.as<float4>(),
                               PP.rec, PP.rec16, PP.foot, PP.cnt, pr.key, pr.val, PP.dlo, krq,
                               strm),
            "project");
    FS_TRY(stage_end(c, tp, strm));
    if (PP.dkey)
      FS_CUDA(cudaMemcpyAsync(PP.dkey, pr.key, static_cast<size_t>(nbb) * n * 4,
                              cudaMemcpyDeviceToDevice, strm),
              "depth key copy");
    if (plan) return FS_OK;  // captured: the key range stays on the device
    FS_CUDA(cudaMemcpyAsync(krhq, krq, 12, cudaMemcpyDeviceToHost, strm), "key range readback");
    FS_CUDA(cudaEventRecord(c->prologue_done[q], strm), "prologue event");
    return FS_OK;
  };
  FS_TRY(ensure_prologue_events(c));
  if (overlap) FS_TRY(launch_prologue(0, stream));
  for (int32_t v0 = 0, b = 0; v0 < V; v0 += vb, ++b) {
    const int nb = std::min(vb, V - v0);
    const int q = parity(b);
    if (!overlap) FS_TRY(launch_prologue(b, stream));
    const Prologue& pr = pro[q];
    const BatchLayout L = pr.L;
    const int total_tiles = L.total_tiles, max_tiles = L.max_tiles;
    const int tile_bits = std::max(1, ceil_log2(total_tiles));
    const int64_t k_total = static_cast<int64_t>(nb) * n;
    FS_TRY(c->state.ensure(static_cast<size_t>(L.pixels) * 4, "pixel state"));
    const size_t sat_bytes = static_cast<size_t>((total_tiles + 63) / 64) * 8;
    FS_TRY(c->sat.ensure(sat_bytes, "tile flags"));
    const size_t subsat_bytes = static_cast<size_t>((4 * total_tiles + 63) / 64) * 8;
    FS_TRY(c->subsat.ensure(subsat_bytes, "sub-tile flags"));
    FS_TRY(c->ranges.ensure(static_cast<size_t>(total_tiles) * 8, "tile ranges"));
    fs::ViewParams* vd = pr.vd;
    float* state = c->state.as<float>();
    uint64_t* sat = c->sat.as<uint64_t>();
    const ProjPtrs P = proj_ptrs(c, keep, v0, n);
    uint8_t* satc = nullptr;
    if (keep) {
      satc = c->kl_satc.as<uint8_t>() + c->kl_tile_off[b];
      FS_CUDA(cudaMemsetAsync(satc, 0xFF, static_cast<size_t>(total_tiles), stream),
              "saturation chunks");
    }
    // the batch's projection (and its key range on the host) is complete
    if (!plan) FS_CUDA(cudaEventSynchronize(c->prologue_done[q]), "key range readback");
    if (overlap) FS_CUDA(cudaStreamWaitEvent(stream, c->prologue_done[q], 0), "prologue wait");
    const uint32_t* krh = pr.krh;
    uint32_t kmin = 0, span = 0;
    int key_bits = 0;
    int64_t k_vis = 0;  // visible slots: the first k_vis sorted positions
    const uint32_t* krd = c->key_range.as<uint32_t>() + 4 * q;  // the same on the device
    if (plan) {
      key_bits = plan->key_bits[b];
      FS_CUDA(fs::launch_graph_check(nullptr, 0u, krd, key_bits, nullptr, 0, ctr, stream),
              "plan check");
      FS_CUDA(fs::launch_chunk_bounds(krd, chunks, c->chunk_bnd.as<int64_t>(), stream),
              "chunk bounds");
    } else if (krh[0] <= krh[1]) {
      kmin = krh[0];
      span = krh[1] - krh[0] + 1;  // invisible slots map to span, after every visible one
      key_bits = std::max(1, ceil_log2(static_cast<int64_t>(span) + 1));
      k_vis = krh[2];
    }
    if (record) record->key_bits[b] = key_bits;
    c->stats.kernel_launches += radix_launches(k_total, key_bits);
    bool alt = false;
    int td = -1;
    FS_TRY(stage_begin(c, FS_STAGE_DEPTH_SORT, stream, plan != nullptr, &td));
    FS_CUDA(fs::radix_sort_pairs(pr.key, pr.val, pr.key_alt, pr.val_alt, k_total, key_bits,
                                 c->sort_tmp.p, &alt, stream, kmin, span, nullptr,
                                 plan ? krd : nullptr),
            "depth sort");
    uint32_t* sorted_key = alt ? pr.key_alt : pr.key;
    uint32_t* sorted_val = alt ? pr.val_alt : pr.val;
    FS_CUDA(fs::launch_depth_tie_fix(k_total, n, sorted_key, sorted_val, P.dlo, stream),
            "depth ties");
    FS_TRY(stage_end(c, td, stream));
    if (overlap && b + 1 < batches) {
      // batch b + 1's buffers (the other parity) were last read by batch
      // b - 1's chunks, which `stream` has passed here
      FS_CUDA(cudaEventRecord(c->buffers_free, stream), "buffers event");
      FS_CUDA(cudaStreamWaitEvent(c->side, c->buffers_free, 0), "buffers wait");
      FS_TRY(launch_prologue(b + 1, c->side));
    }
    uint64_t* subsat = c->subsat.as<uint64_t>();
    int ts = -1;
    FS_TRY(stage_begin(c, FS_STAGE_PIXEL_STATE, stream, plan != nullptr, &ts));
    FS_CUDA(cudaMemsetAsync(sat, 0, sat_bytes, stream), "tile flags clear");
    FS_CUDA(cudaMemsetAsync(subsat, 0, subsat_bytes, stream), "sub-tile flags clear");
    FS_CUDA(fs::launch_state_init(vd, nb, max_tiles, E, mask_dtype, state, sat, subsat, ctr,
                                  stream),
            "pixel state");
    FS_TRY(stage_end(c, ts, stream));
    c->stats.views += nb;
    c->stats.pixels += L.pixels;
    if (keep) {  // the last slot of every chunk but the last (0xFFFFFFFF: empty chunk)
      uint32_t* bound = c->kl_bound.as<uint32_t>() + static_cast<int64_t>(b) * chunks;
      FS_CUDA(cudaMemsetAsync(bound, 0xFF, static_cast<size_t>(chunks) * 4, stream), "bounds");
      if (plan)
        FS_CUDA(fs::launch_chunk_last(c->chunk_bnd.as<int64_t>(), chunks, sorted_val, bound,
                                      stream),
                "bounds");
      for (int ci = 0; ci + 1 < chunks && !plan; ++ci) {
        const int64_t pb = ci == 0 ? 0 : chunk_end(k_vis, chunks, ci - 1);
        const int64_t p1 = chunk_end(k_vis, chunks, ci);
        if (p1 > pb)
          FS_CUDA(cudaMemcpyAsync(bound + ci, sorted_val + (p1 - 1), 4, cudaMemcpyDeviceToDevice,
                                  stream),
                  "bounds");
      }
    }

    // front-to-back depth chunks over the visible slots: a chunk lists only
    // tiles not yet saturated
    int64_t p0 = 0;
    for (int ci = 0; ci < chunks; ++ci) {
      const size_t pi = static_cast<size_t>(b) * chunks + ci;
      const int64_t p1 = plan ? 0 : chunk_end(k_vis, chunks, ci);
      const int64_t n_pos = plan ? plan->npos[pi] : p1 - p0;
      if (record) record->npos[pi] = n_pos;
      DevBuf* val_dst = keep ? &c->kl_val[static_cast<size_t>(b) * chunks + ci] : &c->lv_a;
      uint2* ranges_dst =
          keep ? c->kl_ranges.as<uint2>() + (c->kl_tile_off[b] * chunks +
                                             static_cast<int64_t>(ci) * total_tiles)
               : c->ranges.as<uint2>();
      if (n_pos <= 0) {
        if (keep)
          FS_CUDA(cudaMemsetAsync(ranges_dst, 0, static_cast<size_t>(total_tiles) * 8, stream),
                  "ranges clear");
        if (plan)  // the plan's chunk is empty: so must the replay's be
          FS_CUDA(fs::launch_graph_check(nullptr, 0u, nullptr, 0, c->chunk_bnd.as<int64_t>() + ci,
                                         0, ctr, stream),
                  "plan check");
        continue;
      }
      int64_t I = 0;
      FS_TRY(bin_positions(c, p0, n_pos, n, vd, nb, sorted_val, P, sat, total_tiles, tile_bits, kcap,
                           !plan, val_dst, ranges_dst, stream, &I,
                           plan ? c->chunk_bnd.as<int64_t>() + ci : nullptr,
                           plan ? plan->entries[pi] : 0));
      if (record) record->entries[pi] = I;
      p0 = p1;
      if (I == 0) continue;
      int tb = -1;
      FS_TRY(stage_begin(c, FS_STAGE_BLEND, stream, plan != nullptr, &tb));
      FS_CUDA(fs::launch_blend(vd, nb, max_tiles, ranges_dst, val_dst->as<uint32_t>(), P.rec,
                               P.rec16, n, E, mask_dtype, table, table_dtype, state, sat, subsat,
                               satc, ci, ctr, c->census, stream),
              "blend");
      FS_TRY(stage_end(c, tb, stream));
    }
  }
  c->kl_valid = keep;
  return FS_OK;
}

// Dedicated binning of the tiles whose `skip` bit is clear (all depths, one
// list per tile) and the re-check compositing of them into R.
fs_status recheck_batch_rebin(fs_ctx* c, const fs_scene* s, int64_t n, int nb, int64_t kcap,
                              const BatchLayout& L, const fs::ViewParams* vd, const ProjPtrs& P,
                              const uint32_t* key_src, uint64_t* skip, int32_t mask_dtype,
                              int32_t E, const int32_t* map, double* R, cudaStream_t stream) {
  const int total_tiles = L.total_tiles;
  const int tile_bits = std::max(1, ceil_log2(total_tiles));
  const int64_t k_total = static_cast<int64_t>(nb) * n;
  unsigned long long* ctr = c->counters.as<unsigned long long>();
  c->stats.kernel_launches += 1 + scan_launches(k_total);
  FS_CUDA(fs::launch_candidates(k_total, n, vd, P.cnt, P.foot, skip, c->ccnt.as<uint32_t>(),
                                stream),
          "candidates");
  FS_CUDA(fs::exclusive_scan(c->ccnt.as<uint32_t>(), nullptr, c->offs.as<uint32_t>(), k_total,
                             c->total.as<uint32_t>(), c->scan_tmp.p, stream),
          "candidate scan");
  int64_t C = 0;
  FS_TRY(read_total(c, stream, &C));
  if (C == 0) return FS_OK;
  c->stats.kernel_launches += 2 + radix_launches(C, 32);
  FS_CUDA(fs::launch_compact(k_total, c->ccnt.as<uint32_t>(), c->offs.as<uint32_t>(), key_src,
                             c->key_b.as<uint32_t>(), c->val_b.as<uint32_t>(), stream),
          "compact");
  bool alt = false;
  FS_CUDA(fs::radix_sort_pairs(c->key_b.as<uint32_t>(), c->val_b.as<uint32_t>(),
                               c->key_a.as<uint32_t>(), c->val_a.as<uint32_t>(), C, 32,
                               c->sort_tmp.p, &alt, stream),
          "candidate sort");
  uint32_t* sorted_key = alt ? c->key_a.as<uint32_t>() : c->key_b.as<uint32_t>();
  uint32_t* sorted_val = alt ? c->val_a.as<uint32_t>() : c->val_b.as<uint32_t>();
  FS_CUDA(fs::launch_depth_tie_fix(C, n, sorted_key, sorted_val, P.dlo, stream), "depth ties");
  int64_t I = 0;
  FS_TRY(bin_positions(c, 0, C, n, vd, nb, sorted_val, P, skip, total_tiles, tile_bits, kcap, false,
                       &c->lv_a, c->ranges.as<uint2>(), stream, &I));
  if (I == 0) return FS_OK;
  fs::RecheckLists Ls{};
  Ls.val[0] = c->lv_a.as<uint32_t>();
  Ls.ranges[0] = c->ranges.as<uint2>();
  Ls.chunks = 1;
  c->stats.kernel_launches += 1;
  FS_CUDA(fs::launch_recheck_blend(vd, nb, L.max_tiles, Ls, skip, P.rec, P.rec16,
                                   s->pos_op.as<float4>(), n, E, mask_dtype, map, R, ctr, stream),
          "re-check blend");
  return FS_OK;
}

// Re-check of the Gaussians whose margin is below c->recheck_margin (see
// fs_recheck.cu): their rows of `table` and their bits / label / margin are
// replaced.  `margin` holds the FP32 decision's margins on entry.
// kept_from: another context whose resident projection and kept lists the
// re-check reads (never writes); c supplies every buffer it writes.
fs_status recheck_impl(fs_ctx* c, const fs_scene* s, const fs_camera* cams, int32_t V,
                       int32_t mask_dtype, int32_t E, float gamma, void* table,
                       int32_t table_dtype, uint64_t* bits, int32_t* label, float* margin,
                       bool keep, cudaStream_t stream, const fs_ctx* kept_from = nullptr) {
  const int64_t n = s->n;
  if (kept_from && !(keep && kept_from->kl_valid)) {
    kept_from = nullptr;  // nothing kept there: project again into c
    keep = false;
  }
  const fs_ctx* K = kept_from ? kept_from : c;  // the resident projection and lists
  if (n == 0 || V == 0) return FS_OK;
  const size_t nn = static_cast<size_t>(n);
  FS_TRY(c->rk_flag.ensure(nn * 4, "re-check flags"));
  FS_TRY(c->rk_offs.ensure(nn * 4, "re-check offsets"));
  FS_TRY(c->rk_F.ensure(nn * 4, "re-check set"));
  FS_TRY(c->rk_map.ensure(nn * 4, "re-check map"));
  FS_TRY(c->scan_tmp.ensure(fs::scan_temp_bytes(n), "scan temp"));
  uint32_t* F = c->rk_F.as<uint32_t>();
  int32_t* map = c->rk_map.as<int32_t>();
  c->stats.kernel_launches += 2 + scan_launches(n);
  FS_CUDA(fs::launch_flag_margin(n, margin, c->recheck_margin, c->rk_flag.as<uint32_t>(), stream),
          "re-check flags");
  FS_CUDA(fs::exclusive_scan(c->rk_flag.as<uint32_t>(), nullptr, c->rk_offs.as<uint32_t>(), n,
                             c->total.as<uint32_t>(), c->scan_tmp.p, stream),
          "re-check scan");
  FS_CUDA(fs::launch_scatter_flagged(n, c->rk_flag.as<uint32_t>(), c->rk_offs.as<uint32_t>(), F,
                                     map, stream),
          "re-check set");
  int64_t nF = 0;
  FS_TRY(read_total(c, stream, &nF));
  c->stats.rechecked = nF;
  if (nF == 0) return FS_OK;
  const size_t rbytes = static_cast<size_t>(nF) * E * 8;
  FS_TRY(c->rk_R.ensure(rbytes, "re-check rows"));
  double* R = c->rk_R.as<double>();
  FS_CUDA(cudaMemsetAsync(R, 0, rbytes, stream), "re-check rows clear");
  const bool kept = keep && K->kl_valid;
  double* Rb = nullptr;
  if (kept) {
    FS_TRY(c->rk_Rb.ensure(rbytes, "re-check batch rows"));
    Rb = c->rk_Rb.as<double>();
  }

  const int vb = batch_views(c, n);
  FS_TRY(ensure_free_tabs(c, cams, V, vb));
  const int64_t kcap = static_cast<int64_t>(vb) * n;
  const int chunks = K->kl_chunks;
  fs::ViewParams* vh = c->views_host.as<fs::ViewParams>();
  unsigned long long* ctr = c->counters.as<unsigned long long>();
  unsigned long long* ctr_h = c->counters_host.as<unsigned long long>();
  for (int32_t v0 = 0, b = 0; v0 < V; v0 += vb, ++b) {
    const int nb = std::min(vb, V - v0);
    const ProjPtrs P = proj_ptrs(K, keep, v0, n);
    const BatchLayout L = layout_batch(c, vh, cams, v0, nb, P.cols);
    const int total_tiles = L.total_tiles;
    const size_t sat_bytes = static_cast<size_t>((total_tiles + 63) / 64) * 8;
    FS_TRY(c->sat.ensure(sat_bytes, "tile flags"));
    FS_TRY(c->subsat.ensure(sat_bytes, "deep tile flags"));
    FS_TRY(c->ranges.ensure(static_cast<size_t>(total_tiles) * 8, "tile ranges"));
    fs::ViewParams* vd = c->views.as<fs::ViewParams>();
    uint64_t* skip = c->sat.as<uint64_t>();
    uint64_t* deep = c->subsat.as<uint64_t>();
    FS_CUDA(cudaMemcpyAsync(vd, vh, sizeof(fs::ViewParams) * nb, cudaMemcpyHostToDevice, stream),
            "view upload");
    const uint32_t* key_src = P.dkey;
    if (!keep) {
      c->stats.kernel_launches += 1;
      FS_CUDA(fs::launch_project(n, nb, vd, s->pos_op.as<float4>(), s->cov.as<float4>(), P.rec,
                                 P.rec16, P.foot, P.cnt, c->key_a.as<uint32_t>(),
                                 c->val_a.as<uint32_t>(), P.dlo, nullptr, stream),
              "project");
      key_src = c->key_a.as<uint32_t>();
    }
    // tiles to re-render: those the flagged Gaussians reach
    FS_CUDA(cudaMemsetAsync(skip, 0xFF, sat_bytes, stream), "skip bits");
    FS_CUDA(cudaMemsetAsync(deep, 0, sat_bytes, stream), "deep bits");
    FS_CUDA(cudaMemsetAsync(c->total.p, 0, sizeof(uint32_t), stream), "visible clear");
    const uint8_t* satc = kept ? K->kl_satc.as<uint8_t>() + K->kl_tile_off[b] : nullptr;
    const uint32_t* bound = kept ? K->kl_bound.as<uint32_t>() + static_cast<int64_t>(b) * chunks
                                 : nullptr;
    c->stats.kernel_launches += 1;
    FS_CUDA(fs::launch_mark_tiles(nF, nb, n, F, vd, P.cnt, P.foot, skip, c->total.as<uint32_t>(),
                                  bound, chunks, P.dkey, P.dlo, satc, deep, stream),
            "mark tiles");
    int64_t visible = 0;
    FS_TRY(read_total(c, stream, &visible));
    if (visible == 0) continue;  // no re-checked Gaussian in these views
    if (kept) {
      // walk the main pass's kept chunk lists
      fs::RecheckLists Ls{};
      for (int ci = 0; ci < chunks; ++ci) {
        Ls.val[ci] = K->kl_val[static_cast<size_t>(b) * chunks + ci].as<uint32_t>();
        Ls.ranges[ci] = K->kl_ranges.as<uint2>() +
                        (K->kl_tile_off[b] * chunks + static_cast<int64_t>(ci) * total_tiles);
      }
      Ls.chunks = chunks;
      Ls.sat_chunk = satc;
      Ls.deep = deep;
      Ls.flagged = F;
      Ls.n_flagged = static_cast<int>(std::min<int64_t>(nF, 0x7FFFFFFF));
      Ls.cnt = P.cnt;
      FS_CUDA(cudaMemsetAsync(Rb, 0, rbytes, stream), "batch rows clear");
      FS_CUDA(cudaMemsetAsync(ctr + fs::kRecheckIncomplete, 0, 8, stream), "incomplete clear");
      c->stats.kernel_launches += 1;
      FS_CUDA(fs::launch_recheck_blend(vd, nb, L.max_tiles, Ls, skip, P.rec, P.rec16,
                                       s->pos_op.as<float4>(), n, E, mask_dtype, map, Rb, ctr,
                                       stream),
              "re-check blend");
      FS_CUDA(cudaMemcpyAsync(ctr_h + fs::kRecheckIncomplete, ctr + fs::kRecheckIncomplete, 8,
                              cudaMemcpyDeviceToHost, stream),
              "incomplete readback");
      FS_CUDA(cudaStreamSynchronize(stream), "incomplete readback");
      if (ctr_h[fs::kRecheckIncomplete] == 0) {
        c->stats.kernel_launches += 1;
        FS_CUDA(fs::launch_add_rows(static_cast<int64_t>(nF) * E, Rb, R, stream), "rows add");
        continue;
      }
      c->stats.recheck_rebinned += 1;  // kept lists end too early: bin these tiles anew
    }
    FS_TRY(recheck_batch_rebin(c, s, n, nb, kcap, L, vd, P, key_src, skip, mask_dtype, E, map, R,
                               stream));
  }
  c->stats.kernel_launches += 1;
  FS_CUDA(fs::launch_assign_rows(R, F, nF, E, gamma, table, table_dtype, bits, label, margin,
                                 stream),
          "re-check assign");
  return FS_OK;
}

fs_status check_accumulate_args(fs_ctx* c, const fs_scene* s, const fs_camera* cams, int32_t V,
                                const void* const* masks, int32_t mask_dtype, int32_t mask_memory,
                                int32_t E) {
  if (!c || !s) return fail(FS_INVALID_ARGUMENT, "NULL context or scene");
  if (s->ctx->device != c->device)
    return fail(FS_INVALID_ARGUMENT, "scene lives on device %d, context on device %d",
                s->ctx->device, c->device);
  if (V < 0) return fail(FS_INVALID_ARGUMENT, "n_views = %d", V);
  if (V > 0 && (!cams || !masks)) return fail(FS_INVALID_ARGUMENT, "NULL cams or masks");
  if (mask_dtype != FS_U8 && mask_dtype != FS_I32)
    return fail(FS_INVALID_ARGUMENT, "mask dtype must be FS_U8 or FS_I32");
  if (mask_memory != FS_MEM_HOST && mask_memory != FS_MEM_DEVICE)
    return fail(FS_INVALID_ARGUMENT, "bad mask memory kind %d", mask_memory);
  if (E < 1 || E > fs::kMaxLabels) return fail(FS_INVALID_ARGUMENT, "E = %d out of [1, 4096]", E);
  for (int v = 0; v < V; ++v) {
    FS_TRY(check_camera(cams[v], v));
    if (!masks[v]) return fail(FS_INVALID_ARGUMENT, "mask %d is NULL", v);
  }
  return FS_OK;
}

// Novel-view masks (fs_render.cu): per view batch, one projection and depth
// sort; per object e = 1 .. E-1, the sorted slots of its visible members,
// binned in one list, composited and folded into the masks.
fs_status render_impl(fs_ctx* c, const fs_scene* s, const fs_camera* cams, int32_t V,
                      const uint64_t* member_bits, int32_t E, float tau,
                      void* const* masks_out, int32_t out_dtype, float* const* rho_out,
                      float* const* depth_out, cudaStream_t stream) {
  const int64_t n = s->n;
  if (V == 0) return FS_OK;
  const size_t osize = dtype_size(out_dtype);
  if (n == 0) {  // nothing to render: every mask is 0, every rho and depth 0
    for (int32_t v = 0; v < V; ++v) {
      const size_t npix = static_cast<size_t>(cams[v].width) * cams[v].height;
      FS_CUDA(cudaMemsetAsync(masks_out[v], 0, npix * osize, stream), "mask clear");
      if (rho_out && rho_out[v])
        FS_CUDA(cudaMemsetAsync(rho_out[v], 0, npix * (E - 1) * 4, stream), "rho clear");
      if (depth_out && depth_out[v])
        FS_CUDA(cudaMemsetAsync(depth_out[v], 0, npix * (E - 1) * 4, stream), "depth clear");
    }
    return FS_OK;
  }
  const int vb = batch_views(c, n);
  FS_TRY(ensure_free_tabs(c, cams, V, vb));
  if (vb < 1) return fail(FS_UNSUPPORTED, "fs_render_masks: scene too large");
  const int64_t kcap = static_cast<int64_t>(vb) * n;
  FS_TRY(ensure_window(c, n, vb, V, false));
  FS_TRY(c->key_range.ensure(32, "depth key range"));
  FS_TRY(c->rd_flag.ensure(static_cast<size_t>(kcap) * 4, "render flags"));
  FS_TRY(c->rd_offs.ensure(static_cast<size_t>(kcap) * 4, "render offsets"));
  FS_TRY(c->rd_val.ensure(static_cast<size_t>(kcap) * 4, "render slots"));
  FS_TRY(c->scan_tmp.ensure(fs::scan_temp_bytes(kcap), "scan temp"));
  const size_t ro_bytes = sizeof(fs::RenderOut) * fs::kMaxViewsPerBatch;
  FS_TRY(c->render_out.ensure(ro_bytes, "render outputs"));
  FS_TRY(c->render_out_host.ensure(ro_bytes));
  c->mask_dev.assign(V, nullptr);  // the batch views carry no input mask
  fs::ViewParams* vh = c->views_host.as<fs::ViewParams>();
  fs::ViewParams* vd = c->views.as<fs::ViewParams>();
  fs::RenderOut* roh = c->render_out_host.as<fs::RenderOut>();
  fs::RenderOut* rod = c->render_out.as<fs::RenderOut>();
  uint32_t* krq = c->key_range.as<uint32_t>();
  uint32_t* krh = c->total_host.as<uint32_t>() + 4;
  for (int32_t v0 = 0; v0 < V; v0 += vb) {
    const int nb = std::min(vb, V - v0);
    const ProjPtrs P = proj_ptrs(c, false, v0, n);
    const BatchLayout L = layout_batch(c, vh, cams, v0, nb, P.cols);
    const int total_tiles = L.total_tiles, max_tiles = L.max_tiles;
    const int tile_bits = std::max(1, ceil_log2(total_tiles));
    const int64_t k_total = static_cast<int64_t>(nb) * n;
    for (int k = 0; k < nb; ++k)
      roh[k] = {masks_out[v0 + k], rho_out ? rho_out[v0 + k] : nullptr,
                depth_out ? depth_out[v0 + k] : nullptr};
    FS_CUDA(cudaMemcpyAsync(vd, vh, sizeof(fs::ViewParams) * nb, cudaMemcpyHostToDevice, stream),
            "view upload");
    FS_CUDA(cudaMemcpyAsync(rod, roh, sizeof(fs::RenderOut) * nb, cudaMemcpyHostToDevice,
                            stream),
            "render output upload");
    // every Gaussian projected into the batch's views and depth-sorted once
    FS_CUDA(cudaMemsetAsync(krq, 0xFF, 4, stream), "key range");
    FS_CUDA(cudaMemsetAsync(krq + 1, 0, 8, stream), "key range");
    FS_CUDA(fs::launch_project(n, nb, vd, s->pos_op.as<float4>(), s->cov.as<float4>(), P.rec,
                               P.rec16, P.foot, P.cnt, c->key_a.as<uint32_t>(),
                               c->val_a.as<uint32_t>(), P.dlo, krq, stream),
            "project");
    FS_CUDA(cudaMemcpyAsync(krh, krq, 12, cudaMemcpyDeviceToHost, stream), "key range readback");
    FS_CUDA(cudaStreamSynchronize(stream), "key range readback");
    uint32_t kmin = 0, span = 0;
    int key_bits = 0;
    int64_t k_vis = 0;  // the visible slots come first after the sort
    if (krh[0] <= krh[1]) {
      kmin = krh[0];
      span = krh[1] - krh[0] + 1;
      key_bits = std::max(1, ceil_log2(static_cast<int64_t>(span) + 1));
      k_vis = krh[2];
    }
    bool alt = false;
    FS_CUDA(fs::radix_sort_pairs(c->key_a.as<uint32_t>(), c->val_a.as<uint32_t>(),
                                 c->key_b.as<uint32_t>(), c->val_b.as<uint32_t>(), k_total,
                                 key_bits, c->sort_tmp.p, &alt, stream, kmin, span),
            "depth sort");
    uint32_t* sorted_key = alt ? c->key_b.as<uint32_t>() : c->key_a.as<uint32_t>();
    uint32_t* sorted_val = alt ? c->val_b.as<uint32_t>() : c->val_a.as<uint32_t>();
    FS_CUDA(fs::launch_depth_tie_fix(k_total, n, sorted_key, sorted_val, P.dlo, stream),
            "depth ties");
    // no tile saturates: every list is complete
    const size_t sat_bytes = static_cast<size_t>((total_tiles + 63) / 64) * 8;
    FS_TRY(c->sat.ensure(sat_bytes, "tile flags"));
    FS_TRY(c->ranges.ensure(static_cast<size_t>(total_tiles) * 8, "tile ranges"));
    FS_TRY(c->state.ensure(static_cast<size_t>(L.pixels) * 4, "pixel state"));
    FS_CUDA(cudaMemsetAsync(c->sat.p, 0, sat_bytes, stream), "tile flags clear");
    for (int e = 1; e < E; ++e) {
      uint32_t* flag = c->rd_flag.as<uint32_t>();
      FS_CUDA(fs::launch_member_select(k_vis, n, sorted_val, P.cnt, member_bits, 1ull << e, flag,
                                       stream),
              "object slots");
      FS_CUDA(fs::exclusive_scan(flag, nullptr, c->rd_offs.as<uint32_t>(), k_vis,
                                 c->total.as<uint32_t>(), c->scan_tmp.p, stream),
              "object scan");
      FS_CUDA(fs::launch_member_scatter(k_vis, flag, c->rd_offs.as<uint32_t>(), sorted_val,
                                        c->rd_val.as<uint32_t>(), stream),
              "object scatter");
      int64_t count = 0;
      FS_TRY(read_total(c, stream, &count));
      int64_t I = 0;
      FS_TRY(bin_positions(c, 0, count, n, vd, nb, c->rd_val.as<uint32_t>(), P,
                           c->sat.as<uint64_t>(), total_tiles, tile_bits, kcap, false, &c->lv_a,
                           c->ranges.as<uint2>(), stream, &I));
      FS_CUDA(fs::launch_render(vd, rod, nb, max_tiles, c->ranges.as<uint2>(),
                                c->lv_a.as<uint32_t>(), P.rec, P.rec16, e, e == 1, tau,
                                c->state.as<float>(), out_dtype, stream),
              "render");
    }
    // the host staging of this batch is read by the copies above before the
    // next batch rewrites it
    FS_CUDA(cudaStreamSynchronize(stream), "render");
  }
  return FS_OK;
}

}  // namespace

extern "C" {

fs_status fs_accumulate(fs_ctx* c, const fs_scene* s, const fs_camera* cams, int32_t V,
                        const void* const* masks, int32_t mask_dtype, int32_t mask_memory,
                        int32_t E, void* table, int32_t table_dtype, void* stream) {
  FS_TRY(check_accumulate_args(c, s, cams, V, masks, mask_dtype, mask_memory, E));
  if (table_dtype != FS_F32 && table_dtype != FS_F64)
    return fail(FS_INVALID_ARGUMENT, "table dtype must be FS_F32 or FS_F64");
  if (!table && s->n > 0) return fail(FS_INVALID_ARGUMENT, "table is NULL");
  DeviceGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  c->stats = fs_stats{};
  c->events_used = 0;
  FS_CUDA(cudaMemsetAsync(c->counters.p, 0, c->counters.bytes, st), "counters clear");
  return accumulate_impl(c, s, cams, V, masks, mask_dtype, mask_memory, E, table, table_dtype,
                         false, st);
}

fs_status fs_assign(fs_ctx* c, const void* table, int32_t table_dtype, int64_t n, int32_t E,
                    float gamma, uint64_t* member_bits, int32_t* label, float* margin,
                    void* stream) {
  if (!c) return fail(FS_INVALID_ARGUMENT, "NULL context");
  if (table_dtype != FS_F32 && table_dtype != FS_F64)
    return fail(FS_INVALID_ARGUMENT, "table dtype must be FS_F32 or FS_F64");
  if (n < 0 || (n > 0 && !table)) return fail(FS_INVALID_ARGUMENT, "bad table or n");
  if (E < 1 || E > fs::kMaxLabels) return fail(FS_INVALID_ARGUMENT, "E = %d out of [1, 4096]", E);
  if (!(gamma >= -1.f && gamma <= 1.f))
    return fail(FS_INVALID_ARGUMENT, "gamma = %g outside [-1, 1]", (double)gamma);
  if (member_bits && E > 64)
    return fail(FS_UNSUPPORTED, "member_bits needs E <= 64 (E = %d)", E);
  DeviceGuard g(c->device);
  FS_CUDA(fs::launch_assign(table, table_dtype, n, E, gamma, member_bits, label, margin,
                            static_cast<cudaStream_t>(stream)),
          "assign");
  if (n > 0) c->stats.kernel_launches += 1;
  return FS_OK;
}

// Whether every view's projection can stay resident for the near-tie
// re-check: it must fit in half of the free device memory (108 B per
// Gaussian and view; 76 B with reduced-precision records), and the context
// must not be set to project again.
bool keep_fits(const fs_ctx* c, int64_t n, int32_t V) {
  if (c->recheck_reproject) return false;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const double need = (c->compact ? 76.0 : 108.0) * static_cast<double>(n) * V;
  const double have = static_cast<double>(c->rec.bytes + c->foot.bytes + c->cnt.bytes +
                                          c->dlo.bytes + c->dkey.bytes);
  return need <= have + 0.5 * static_cast<double>(free_b);
}

fs_status fs_solve(fs_ctx* c, const fs_scene* s, const fs_camera* cams, int32_t V,
                   const void* const* masks, int32_t mask_dtype, int32_t mask_memory, int32_t E,
                   float gamma, const fs_result* out, void* stream) {
  FS_TRY(check_accumulate_args(c, s, cams, V, masks, mask_dtype, mask_memory, E));
  if (!out) return fail(FS_INVALID_ARGUMENT, "fs_solve: out is NULL");
  if (out->memory != FS_MEM_HOST && out->memory != FS_MEM_DEVICE)
    return fail(FS_INVALID_ARGUMENT, "fs_solve: bad output memory kind");
  const int tdt = out->table_dtype;
  if (tdt != FS_F32 && tdt != FS_F64)
    return fail(FS_INVALID_ARGUMENT, "table dtype must be FS_F32 or FS_F64");
  if (!(gamma >= -1.f && gamma <= 1.f))
    return fail(FS_INVALID_ARGUMENT, "gamma = %g outside [-1, 1]", (double)gamma);
  if (out->member_bits && E > 64) return fail(FS_UNSUPPORTED, "member_bits needs E <= 64");
  DeviceGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = s->n;
  // The cross-view reduction always runs in FP64: a Gaussian seen in many
  // views collects up to ~1e5 atomic adds, whose FP32 rounding alone would
  // exceed 1e-5 relative.  An FP32 result is rounded once at the end.
  const size_t tbytes = static_cast<size_t>(n) * E * 8;
  const bool dev_out = out->memory == FS_MEM_DEVICE;
  void* table = (dev_out && out->table && tdt == FS_F64) ? out->table : nullptr;
  if (!table) {
    FS_TRY(c->table_tmp.ensure(tbytes > 0 ? tbytes : 8, "table"));
    table = c->table_tmp.p;
  }
  c->stats = fs_stats{};
  c->events_used = 0;
  FS_CUDA(cudaMemsetAsync(c->counters.p, 0, c->counters.bytes, st), "counters clear");
  if (tbytes) FS_CUDA(cudaMemsetAsync(table, 0, tbytes, st), "table clear");
  const bool recheck = c->recheck_margin > 0.f && n > 0 && V > 0;
  // keep every view's projection resident for the re-check when it fits in
  // half of the free device memory (108 B per Gaussian and view; 76 B with
  // reduced-precision records)
  const bool keep = recheck && keep_fits(c, n, V);
  FS_TRY(accumulate_impl(c, s, cams, V, masks, mask_dtype, mask_memory, E, table, FS_F64, keep,
                         st));
  uint64_t* bits = out->member_bits;
  int32_t* label = out->label;
  float* margin = out->margin;
  const size_t nn = static_cast<size_t>(n > 0 ? n : 1);
  if (!dev_out) {
    if (bits) { FS_TRY(c->bits_tmp.ensure(nn * 8, "bits")); bits = c->bits_tmp.as<uint64_t>(); }
    if (label) { FS_TRY(c->label_tmp.ensure(nn * 4, "labels")); label = c->label_tmp.as<int32_t>(); }
    if (margin) { FS_TRY(c->margin_tmp.ensure(nn * 4, "margins")); margin = c->margin_tmp.as<float>(); }
  }
  if (recheck && !margin) {  // the re-check needs the margins
    FS_TRY(c->margin_tmp.ensure(nn * 4, "margins"));
    margin = c->margin_tmp.as<float>();
  }
  int ta = -1;
  FS_TRY(stage_begin(c, FS_STAGE_ASSIGN, st, false, &ta));
  if (bits || label || margin) {
    FS_CUDA(fs::launch_assign(table, FS_F64, n, E, gamma, bits, label, margin, st), "assign");
    if (n > 0) c->stats.kernel_launches += 1;
  }
  FS_TRY(stage_end(c, ta, st));
  if (recheck) {
    int tr = -1;
    FS_TRY(stage_begin(c, FS_STAGE_RECHECK, st, false, &tr));
    c->stage_outer = tr >= 0;  // its binning and sorts count as re-check time
    const fs_status rs = recheck_impl(c, s, cams, V, mask_dtype, E, gamma, table, FS_F64, bits,
                                      label, margin, keep, st);
    c->stage_outer = false;
    FS_TRY(rs);
    FS_TRY(stage_end(c, tr, st));
  }
  // the caller's table: rounded once to FP32, or the FP64 sums themselves
  const int64_t count = n * static_cast<int64_t>(E);
  const void* result = table;
  if (out->table && tdt == FS_F32) {
    float* dst = static_cast<float*>(out->table);
    if (!dev_out) {
      FS_TRY(c->table32_tmp.ensure(static_cast<size_t>(count > 0 ? count : 1) * 4, "table"));
      dst = c->table32_tmp.as<float>();
    }
    c->stats.kernel_launches += count > 0 ? 1 : 0;
    int tr = -1;
    FS_TRY(stage_begin(c, FS_STAGE_ASSIGN, st, false, &tr));
    FS_CUDA(fs::launch_round_table(count, static_cast<const double*>(table), dst, st),
            "table rounding");
    FS_TRY(stage_end(c, tr, st));
    result = dst;
  } else if (out->table && dev_out && table != out->table) {
    FS_CUDA(cudaMemcpyAsync(out->table, table, tbytes, cudaMemcpyDeviceToDevice, st),
            "table copy");
  }
  if (!dev_out && n > 0) {
    if (out->table)
      FS_CUDA(cudaMemcpyAsync(out->table, result, static_cast<size_t>(count) * dtype_size(tdt),
                              cudaMemcpyDeviceToHost, st),
              "table D2H");
    if (out->member_bits)
      FS_CUDA(cudaMemcpyAsync(out->member_bits, bits, n * 8, cudaMemcpyDeviceToHost, st), "D2H");
    if (out->label)
      FS_CUDA(cudaMemcpyAsync(out->label, label, n * 4, cudaMemcpyDeviceToHost, st), "D2H");
    if (out->margin)
      FS_CUDA(cudaMemcpyAsync(out->margin, margin, n * 4, cudaMemcpyDeviceToHost, st), "D2H");
  }
  return FS_OK;
}

fs_status fs_keep_after_removal(fs_ctx* c, const uint64_t* member_bits, int64_t n,
                                uint64_t remove, int32_t* keep_index, int64_t* n_keep,
                                void* stream) {
  if (!c || !n_keep) return fail(FS_INVALID_ARGUMENT, "fs_keep_after_removal: NULL argument");
  *n_keep = 0;
  if (n < 0 || n >= (static_cast<int64_t>(1) << 31) || (n > 0 && (!member_bits || !keep_index)))
    return fail(FS_INVALID_ARGUMENT, "fs_keep_after_removal: bad n or NULL array");
  if (n == 0) return FS_OK;
  DeviceGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nn = static_cast<size_t>(n);
  FS_TRY(c->rk_flag.ensure(nn * 4, "removal flags"));
  FS_TRY(c->rk_offs.ensure(nn * 4, "removal offsets"));
  FS_TRY(c->scan_tmp.ensure(fs::scan_temp_bytes(n), "scan temp"));
  FS_CUDA(fs::launch_keep_flags(n, member_bits, remove, c->rk_flag.as<uint32_t>(), st),
          "removal flags");
  FS_CUDA(fs::exclusive_scan(c->rk_flag.as<uint32_t>(), nullptr, c->rk_offs.as<uint32_t>(), n,
                             c->total.as<uint32_t>(), c->scan_tmp.p, st),
          "removal scan");
  FS_CUDA(fs::launch_keep_scatter(n, c->rk_flag.as<uint32_t>(), c->rk_offs.as<uint32_t>(),
                                  keep_index, st),
          "removal scatter");
  c->stats.kernel_launches += 2 + scan_launches(n);
  int64_t kept = 0;
  FS_TRY(read_total(c, st, &kept));
  *n_keep = kept;
  return FS_OK;
}

}  // extern "C"

// A solve captured into a CUDA graph (fs_graph_* in flashsplat.h).
struct fs_graph {
  fs_ctx* c = nullptr;  // the graph's own context: the capture holds its buffers
  // the near-tie re-check after a replay runs on a context of its own: its
  // buffers may grow, and nothing may move the captured ones
  fs_ctx* rc = nullptr;
  const fs_scene* s = nullptr;
  std::vector<fs_camera> cams;
  std::vector<const void*> masks;
  int32_t mask_dtype = 0, E = 0;
  float gamma = 0.f;
  fs_result out{};
  void* table = nullptr;  // the FP64 table the graph accumulates into
  uint64_t* bits = nullptr;
  int32_t* label = nullptr;
  float* margin = nullptr;
  bool keep = false, recheck = false;
  GraphPlan plan;
  cudaStream_t stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

void graph_free(fs_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->stream) cudaStreamDestroy(g->stream);
  g->plan.views.release();
  if (g->rc) fs_destroy(g->rc);
  if (g->c) fs_destroy(g->c);
  delete g;
}

// The captured part of a solve: counters and table cleared, every view
// accumulated into the FP64 table with device-side sizes, the assignment.
fs_status graph_body(fs_graph* g, cudaStream_t st) {
  fs_ctx* c = g->c;
  const int64_t n = g->s->n;
  FS_CUDA(cudaMemsetAsync(c->counters.p, 0, c->counters.bytes, st), "counters clear");
  FS_CUDA(cudaMemsetAsync(g->table, 0, static_cast<size_t>(n) * g->E * 8, st), "table clear");
  FS_TRY(accumulate_impl(c, g->s, g->cams.data(), static_cast<int32_t>(g->cams.size()),
                         g->masks.data(), g->mask_dtype, FS_MEM_DEVICE, g->E, g->table, FS_F64,
                         g->keep, st, nullptr, &g->plan));
  if (g->bits || g->label || g->margin)
    FS_CUDA(fs::launch_assign(g->table, FS_F64, n, g->E, g->gamma, g->bits, g->label, g->margin,
                              st),
            "assign");
  return FS_OK;
}

}  // namespace

extern "C" {

fs_status fs_graph_create(fs_ctx* tmpl, const fs_scene* s, const fs_camera* cams, int32_t V,
                          const void* const* masks, int32_t mask_dtype, int32_t E, float gamma,
                          const fs_result* out, fs_graph** graph) {
  if (!graph) return fail(FS_INVALID_ARGUMENT, "fs_graph_create: graph is NULL");
  *graph = nullptr;
  FS_TRY(check_accumulate_args(tmpl, s, cams, V, masks, mask_dtype, FS_MEM_DEVICE, E));
  if (!out || out->memory != FS_MEM_DEVICE)
    return fail(FS_INVALID_ARGUMENT, "fs_graph_create: outputs must be in device memory");
  if (out->table_dtype != FS_F32 && out->table_dtype != FS_F64)
    return fail(FS_INVALID_ARGUMENT, "table dtype must be FS_F32 or FS_F64");
  if (!(gamma >= -1.f && gamma <= 1.f))
    return fail(FS_INVALID_ARGUMENT, "gamma = %g outside [-1, 1]", (double)gamma);
  if (out->member_bits && E > 64) return fail(FS_UNSUPPORTED, "member_bits needs E <= 64");
  if (s->n == 0 || V == 0) return fail(FS_INVALID_ARGUMENT, "fs_graph_create: nothing to solve");
  fs_options o{};
  o.views_per_batch = tmpl->views_per_batch;
  o.depth_chunks = tmpl->depth_chunks;
  o.recheck_margin = tmpl->recheck_margin > 0.f ? tmpl->recheck_margin : -1.f;
  o.recheck_reproject = tmpl->recheck_reproject ? 1 : 0;
  o.record_precision = tmpl->compact ? FS_F16 : 0;
  o.coverage = tmpl->sigma3 ? FS_COVERAGE_3SIGMA : FS_COVERAGE_EXACT;
  fs_graph* g = new (std::nothrow) fs_graph();
  if (!g) return fail(FS_OUT_OF_MEMORY, "fs_graph_create: host allocation failed");
  fs_status st = fs_create(&g->c, tmpl->device, &o);
  if (st != FS_OK) {
    graph_free(g);
    return st;
  }
  fs_ctx* c = g->c;
  DeviceGuard dg(c->device);
  g->s = s;
  g->cams.assign(cams, cams + V);
  g->masks.assign(masks, masks + V);
  g->mask_dtype = mask_dtype;
  g->E = E;
  g->gamma = gamma;
  g->out = *out;
  const int64_t n = s->n;
  const size_t nn = static_cast<size_t>(n);
  auto bail = [&](fs_status e) {
    graph_free(g);
    return e;
  };
  g->table = (out->table && out->table_dtype == FS_F64) ? out->table : nullptr;
  if (!g->table) {
    if ((st = c->table_tmp.ensure(nn * E * 8, "table")) != FS_OK) return bail(st);
    g->table = c->table_tmp.p;
  }
  g->bits = out->member_bits;
  g->label = out->label;
  g->margin = out->margin;
  g->recheck = c->recheck_margin > 0.f;
  if (g->recheck && !g->margin) {
    if ((st = c->margin_tmp.ensure(nn * 4, "margins")) != FS_OK) return bail(st);
    g->margin = c->margin_tmp.as<float>();
  }
  // the re-check runs on a context of its own, which reads the captured
  // solve's resident projection and kept lists when they fit (g->keep) and
  // writes only its own buffers, so nothing the graph holds is ever resized
  g->keep = g->recheck && keep_fits(c, n, V);
  if (g->recheck) {
    if ((st = fs_create(&g->rc, tmpl->device, &o)) != FS_OK) return bail(st);
    const int vbr = batch_views(g->rc, n);
    if ((st = ensure_window(g->rc, n, vbr, V, false)) != FS_OK) return bail(st);
    if ((st = stage_masks(g->rc, cams, V, masks, mask_dtype, FS_MEM_DEVICE, nullptr)) != FS_OK)
      return bail(st);
  }
  cudaError_t ce = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaStreamCreate"));
  // 1. a solve that records the shapes and sizes every buffer
  c->stats = fs_stats{};
  ce = cudaMemsetAsync(c->counters.p, 0, c->counters.bytes, g->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(g->table, 0, nn * E * 8, g->stream);
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "fs_graph_create"));
  if ((st = accumulate_impl(c, s, cams, V, masks, mask_dtype, FS_MEM_DEVICE, E, g->table, FS_F64,
                            g->keep, g->stream, &g->plan, nullptr)) != FS_OK)
    return bail(st);
  if ((ce = cudaStreamSynchronize(g->stream)) != cudaSuccess)
    return bail(cuda_fail(ce, "fs_graph_create"));
  const int vb = batch_views(c, n);
  const size_t batches = static_cast<size_t>((V + vb - 1) / vb);
  if ((st = g->plan.views.ensure(batches * fs::kMaxViewsPerBatch * sizeof(fs::ViewParams))) !=
      FS_OK)
    return bail(st);
  // 2. the capture: the same solve with device-side sizes
  if ((ce = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return bail(cuda_fail(ce, "cudaStreamBeginCapture"));
  st = graph_body(g, g->stream);
  ce = cudaStreamEndCapture(g->stream, &g->graph);
  if (st != FS_OK) return bail(st);
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaStreamEndCapture"));
  if ((ce = cudaGraphInstantiate(&g->exec, g->graph, 0)) != cudaSuccess)
    return bail(cuda_fail(ce, "cudaGraphInstantiate"));
  *graph = g;
  return FS_OK;
}

fs_status fs_graph_launch(fs_graph* g, void* stream) {
  if (!g) return fail(FS_INVALID_ARGUMENT, "fs_graph_launch: graph is NULL");
  fs_ctx* c = g->c;
  DeviceGuard dg(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  c->stats = fs_stats{};
  c->events_used = 0;
  FS_CUDA(cudaGraphLaunch(g->exec, st), "cudaGraphLaunch");
  const int32_t V = static_cast<int32_t>(g->cams.size());
  if (g->recheck) {
    fs_ctx* rc = g->rc;
    rc->stats = fs_stats{};
    rc->events_used = 0;
    FS_CUDA(cudaMemsetAsync(rc->counters.p, 0, rc->counters.bytes, st), "counters clear");
    FS_TRY(recheck_impl(rc, g->s, g->cams.data(), V, g->mask_dtype, g->E, g->gamma, g->table,
                        FS_F64, g->bits, g->label, g->margin, g->keep, st,
                        g->keep ? g->c : nullptr));
  }
  const int64_t count = g->s->n * static_cast<int64_t>(g->E);
  if (g->out.table && g->out.table_dtype == FS_F32)
    FS_CUDA(fs::launch_round_table(count, static_cast<const double*>(g->table),
                                   static_cast<float*>(g->out.table), st),
            "table rounding");
  return FS_OK;
}

fs_status fs_graph_synchronize(fs_graph* g, void* stream, fs_stats* stats) {
  if (!g) return fail(FS_INVALID_ARGUMENT, "fs_graph_synchronize: graph is NULL");
  fs_stats rs{};
  if (g->rc) FS_TRY(fs_synchronize(g->rc, stream, &rs));
  FS_TRY(fs_synchronize(g->c, stream, stats));
  if (stats) {
    stats->rechecked = rs.rechecked;
    stats->recheck_pairs = rs.recheck_pairs;
    stats->recheck_rebinned = rs.recheck_rebinned;
  }
  return FS_OK;
}

fs_status fs_graph_destroy(fs_graph* g) {
  if (!g) return FS_OK;
  DeviceGuard dg(g->c ? g->c->device : 0);
  if (g->stream) cudaStreamSynchronize(g->stream);
  graph_free(g);
  return FS_OK;
}

fs_status fs_render_masks(fs_ctx* c, const fs_scene* s, const fs_camera* cams, int32_t V,
                          const uint64_t* member_bits, int32_t E, float tau,
                          void* const* masks_out, int32_t out_dtype, float* const* rho_out,
                          float* const* depth_out, void* stream) {
  FS_TRY(check_accumulate_args(c, s, cams, V, masks_out, out_dtype, FS_MEM_DEVICE, E));
  if (E < 2 || E > 64) return fail(FS_INVALID_ARGUMENT, "fs_render_masks: E = %d out of [2, 64]", E);
  if (!(tau == tau)) return fail(FS_INVALID_ARGUMENT, "fs_render_masks: tau is NaN");
  if (s->n > 0 && V > 0 && !member_bits)
    return fail(FS_INVALID_ARGUMENT, "fs_render_masks: member_bits is NULL");
  DeviceGuard g(c->device);
  return render_impl(c, s, cams, V, member_bits, E, tau, masks_out, out_dtype, rho_out,
                     depth_out, static_cast<cudaStream_t>(stream));
}

fs_status fs_check_wait_timeout(int32_t device, int32_t spins) {
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= count)
    return fail(FS_INVALID_ARGUMENT, "fs_check_wait_timeout: bad device %d", device);
  if (spins < 1) return fail(FS_INVALID_ARGUMENT, "fs_check_wait_timeout: spins < 1");
  DeviceGuard g(device);
  // lookback (512) | total (4) | counters | one view | one footprint | tiny arrays
  const size_t bytes = 512 + 256 + 8 * fs::kNumCounters + 1024 + 256 + 256;
  DevBuf ws;
  FS_TRY(ws.ensure(bytes, "wait check"));
  char* base = ws.as<char>();
  FS_CUDA(cudaMemset(base, 0, bytes), "wait check");
  auto* counters = reinterpret_cast<unsigned long long*>(base + 768);
  const size_t o_view = 768 + 8 * fs::kNumCounters;
  cudaError_t le = fs::launch_lookback_probe(
      base, reinterpret_cast<uint32_t*>(base + 512), counters,
      reinterpret_cast<const fs::ViewParams*>(base + ((o_view + 255) & ~size_t(255))),
      reinterpret_cast<const uint32_t*>(base + bytes - 256),
      reinterpret_cast<const fs::Footprint*>(base + bytes - 512),
      reinterpret_cast<const uint64_t*>(base + bytes - 256),
      reinterpret_cast<uint32_t*>(base + bytes - 128), reinterpret_cast<uint32_t*>(base + bytes - 64),
      spins, nullptr);
  unsigned long long h[fs::kNumCounters] = {};
  if (le == cudaSuccess) le = cudaMemcpy(h, counters, sizeof(h), cudaMemcpyDeviceToHost);
  ws.release();
  if (le != cudaSuccess) return cuda_fail(le, "fs_check_wait_timeout");
  if (h[fs::kLookbackTimeout])
    return fail(FS_TIMEOUT, "the binning's bounded wait gave up after %d polls, as it must",
                spins);
  return FS_OK;
}

namespace {

fs_status test_device(int32_t device, const char* what) {
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= count) return fail(FS_INVALID_ARGUMENT, "%s: bad device %d", what, device);
  return FS_OK;
}

}  // namespace

fs_status fs_test_sort_pairs(int32_t device, uint32_t* keys, uint32_t* vals, int64_t n,
                             int32_t bits) {
  FS_TRY(test_device(device, "fs_test_sort_pairs"));
  if (n < 0 || n >= (static_cast<int64_t>(1) << 31) || bits < 1 || bits > 32 ||
      (n > 0 && (!keys || !vals)))
    return fail(FS_INVALID_ARGUMENT, "fs_test_sort_pairs: bad arrays, n or bits");
  if (n == 0) return FS_OK;
  DeviceGuard g(device);
  DevBuf ak, av, tmp;
  FS_TRY(ak.ensure(static_cast<size_t>(n) * 4, "sort keys"));
  FS_TRY(av.ensure(static_cast<size_t>(n) * 4, "sort vals"));
  FS_TRY(tmp.ensure(fs::radix_temp_bytes(n), "sort temp"));
  bool alt = false;
  cudaError_t e = fs::radix_sort_pairs(keys, vals, ak.as<uint32_t>(), av.as<uint32_t>(), n, bits,
                                       tmp.p, &alt, nullptr);
  if (e == cudaSuccess && alt) {
    e = cudaMemcpy(keys, ak.p, static_cast<size_t>(n) * 4, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(vals, av.p, static_cast<size_t>(n) * 4, cudaMemcpyDeviceToDevice);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  ak.release();
  av.release();
  tmp.release();
  if (e != cudaSuccess) return cuda_fail(e, "fs_test_sort_pairs");
  return FS_OK;
}

fs_status fs_test_exclusive_scan(int32_t device, const uint32_t* in, uint32_t* out, int64_t n,
                                 uint32_t* total) {
  FS_TRY(test_device(device, "fs_test_exclusive_scan"));
  if (n < 0 || n >= (static_cast<int64_t>(1) << 31) || !total || (n > 0 && (!in || !out)))
    return fail(FS_INVALID_ARGUMENT, "fs_test_exclusive_scan: bad arrays or n");
  *total = 0;
  if (n == 0) return FS_OK;
  DeviceGuard g(device);
  DevBuf tmp, tot;
  FS_TRY(tmp.ensure(fs::scan_temp_bytes(n), "scan temp"));
  FS_TRY(tot.ensure(4, "scan total"));
  cudaError_t e = fs::exclusive_scan(in, nullptr, out, n, tot.as<uint32_t>(), tmp.p, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(total, tot.p, 4, cudaMemcpyDeviceToHost);
  tmp.release();
  tot.release();
  if (e != cudaSuccess) return cuda_fail(e, "fs_test_exclusive_scan");
  return FS_OK;
}

fs_status fs_test_tile_ranges(int32_t device, const uint32_t* keys, int64_t n, int32_t n_tiles,
                              uint32_t* ranges) {
  FS_TRY(test_device(device, "fs_test_tile_ranges"));
  if (n < 0 || n >= (static_cast<int64_t>(1) << 31) || n_tiles < 1 || !ranges ||
      (n > 0 && !keys))
    return fail(FS_INVALID_ARGUMENT, "fs_test_tile_ranges: bad arrays, n or n_tiles");
  DeviceGuard g(device);
  // every key must name a tile: the kernel writes ranges[key]
  std::vector<uint32_t> hk(static_cast<size_t>(n));
  cudaError_t e = n > 0 ? cudaMemcpy(hk.data(), keys, static_cast<size_t>(n) * 4,
                                     cudaMemcpyDeviceToHost)
                        : cudaSuccess;
  if (e != cudaSuccess) return cuda_fail(e, "fs_test_tile_ranges");
  for (int64_t k = 0; k < n; ++k)
    if (hk[k] >= static_cast<uint32_t>(n_tiles) || (k > 0 && hk[k] < hk[k - 1]))
      return fail(FS_INVALID_ARGUMENT, "fs_test_tile_ranges: key %lld out of range or order",
                  (long long)k);
  e = cudaMemset(ranges, 0, static_cast<size_t>(n_tiles) * 8);
  if (e == cudaSuccess && n > 0)
    e = fs::launch_ranges(n, keys, reinterpret_cast<uint2*>(ranges), nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "fs_test_tile_ranges");
  return FS_OK;
}

fs_status fs_synchronize(fs_ctx* c, void* stream, fs_stats* stats) {
  if (!c) return fail(FS_INVALID_ARGUMENT, "NULL context");
  DeviceGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned long long* ch = c->counters_host.as<unsigned long long>();
  FS_CUDA(cudaMemcpyAsync(ch, c->counters.p, sizeof(unsigned long long) * fs::kNumCounters,
                          cudaMemcpyDeviceToHost, st),
          "counters readback");
  FS_CUDA(cudaStreamSynchronize(st), "fs_synchronize");
  FS_CUDA(cudaGetLastError(), "fs_synchronize");
  c->stats.bad_labels = static_cast<int64_t>(ch[fs::kBadLabels]);
  c->stats.pairs = static_cast<int64_t>(ch[fs::kPairs]);
  c->stats.staged_entries = static_cast<int64_t>(ch[fs::kStaged]);
  c->stats.census_pairs = static_cast<int64_t>(ch[fs::kCensusPairs]);
  c->stats.census_rounds = static_cast<int64_t>(ch[fs::kRounds]);
  c->stats.census_steps = static_cast<int64_t>(ch[fs::kSteps]);
  c->stats.census_rounds_mixed = static_cast<int64_t>(ch[fs::kRoundsMixed]);
  c->stats.recheck_pairs = static_cast<int64_t>(ch[fs::kRecheckPairs]);
  if (ch[fs::kLookbackTimeout])
    return fail(FS_TIMEOUT, "tile binning: %llu bounded wait(s) for a preceding block's offset "
                "gave up; the lists of that solve are incomplete", ch[fs::kLookbackTimeout]);
  if (ch[fs::kBinningMismatch])
    return fail(FS_CUDA_ERROR, "internal error: tile binning count and emission disagreed for "
                "%llu Gaussian(s)", ch[fs::kBinningMismatch]);
  if (ch[fs::kGraphOverflow] || ch[fs::kGraphKeyRange])
    return fail(FS_UNSUPPORTED, "captured solve: the inputs outgrew the capture's plan (%llu "
                "list(s) over capacity, %llu depth sort(s) short of bits); capture again",
                ch[fs::kGraphOverflow], ch[fs::kGraphKeyRange]);
  int64_t blends = 0;
  for (int k = 0; k < FS_NUM_STAGES; ++k) c->stats.stage_ms[k] = 0.0;
  for (size_t k = 0; k + 1 < c->events_used; k += 2) {
    float t = 0.f;
    FS_CUDA(cudaEventElapsedTime(&t, c->events[k], c->events[k + 1]), "cudaEventElapsedTime");
    const int stage = c->event_stage[k / 2];
    c->stats.stage_ms[stage] += t;
    if (stage == FS_STAGE_BLEND) ++blends;
  }
  c->stats.blend_ms = c->stats.stage_ms[FS_STAGE_BLEND];
  c->stats.blend_launches = blends;
  if (stats) *stats = c->stats;
  return FS_OK;
}

}  // extern "C"
