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
    if (p) {
      cudaFree(p);
      p = nullptr;
      bytes = 0;
    }
    size_t want = std::max(need, static_cast<size_t>(bytes + bytes / 4));
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
  return static_cast<int64_t>((bits + 7) / 8) * (2 + scan_launches(nb * 256));
}

}  // namespace

void fs::set_last_error(const char* msg) {
  snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
}

struct fs_ctx {
  int device = 0;
  int views_per_batch = 16;
  int depth_chunks = 4;  // front-to-back chunks per batch (sizes 1/8, 1/8, 1/4, 1/2)
  int n_sm = 0;
  bool time_stages = false;
  std::vector<cudaEvent_t> events;  // (start, stop) pairs around blend launches
  size_t events_used = 0;
  // workspace
  DevBuf views, rec, foot, cnt, key_a, val_a, key_b, val_b, offs, ccnt, dlo, state, sat, subsat;
  DevBuf lk_a, lv_a, lk_b, lv_b, ranges, sort_tmp, scan_tmp, total, counters;
  DevBuf mask_stage, table_tmp, bits_tmp, label_tmp, margin_tmp;
  HostBuf views_host, total_host, counters_host;
  fs_stats stats{};
  int scenes = 0;
};

struct fs_scene {
  fs_ctx* ctx = nullptr;
  int64_t n = 0;
  DevBuf pos_op, cov;  // (m, o) and Sigma3D as float pairs
};

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
  DeviceGuard g(device);
  fs_status st;
  if ((st = c->views.ensure(sizeof(fs::ViewParams) * fs::kMaxViewsPerBatch, "views")) != FS_OK ||
      (st = c->views_host.ensure(sizeof(fs::ViewParams) * fs::kMaxViewsPerBatch)) != FS_OK ||
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
                    &c->table_tmp, &c->bits_tmp, &c->label_tmp, &c->margin_tmp};
  for (DevBuf* b : bufs) b->release();
  c->views_host.release();
  c->total_host.release();
  c->counters_host.release();
  for (cudaEvent_t e : c->events) cudaEventDestroy(e);
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

void fill_view(const fs_camera& cam, fs::ViewParams* vp) {
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

fs_status accumulate_impl(fs_ctx* c, const fs_scene* s, const fs_camera* cams, int32_t V,
                          const void* const* masks, int32_t mask_dtype, int32_t mask_memory,
                          int32_t E, void* table, int32_t table_dtype, cudaStream_t stream) {
  const int64_t n = s->n;
  if (n == 0 || V == 0) return FS_OK;
  int vb = c->views_per_batch;
  // (view, Gaussian) slots of one batch must fit in 31 bits
  const int64_t max_vb = ((static_cast<int64_t>(1) << 31) - 1) / n;
  if (max_vb < 1) return fail(FS_UNSUPPORTED, "fs_accumulate: scene too large");
  vb = static_cast<int>(std::min<int64_t>(vb, max_vb));
  const size_t msize = dtype_size(mask_dtype);
  const int64_t kcap = static_cast<int64_t>(vb) * n;
  FS_TRY(c->rec.ensure(static_cast<size_t>(kcap) * sizeof(fs::ProjRecord), "records"));
  FS_TRY(c->foot.ensure(static_cast<size_t>(kcap) * sizeof(fs::Footprint), "footprints"));
  FS_TRY(c->cnt.ensure(static_cast<size_t>(kcap) * 4, "counts"));
  FS_TRY(c->key_a.ensure(static_cast<size_t>(kcap) * 4, "keys"));
  FS_TRY(c->val_a.ensure(static_cast<size_t>(kcap) * 4, "vals"));
  FS_TRY(c->key_b.ensure(static_cast<size_t>(kcap) * 4, "keys"));
  FS_TRY(c->val_b.ensure(static_cast<size_t>(kcap) * 4, "vals"));
  FS_TRY(c->offs.ensure(static_cast<size_t>(kcap) * 4, "offsets"));
  FS_TRY(c->scan_tmp.ensure(fs::scan_temp_bytes(kcap), "scan temp"));
  FS_TRY(c->sort_tmp.ensure(fs::radix_temp_bytes(kcap), "sort temp"));

  FS_TRY(c->ccnt.ensure(static_cast<size_t>(kcap) * 4, "chunk counts"));
  FS_TRY(c->dlo.ensure(static_cast<size_t>(kcap) * 4, "depth low words"));

  fs::ViewParams* vh = c->views_host.as<fs::ViewParams>();
  uint32_t* total_h = c->total_host.as<uint32_t>();
  unsigned long long* ctr = c->counters.as<unsigned long long>();
  for (int32_t v0 = 0; v0 < V; v0 += vb) {
    const int nb = std::min(vb, V - v0);
    int tile_base = 0, max_tiles = 0;
    int64_t state_off = 0;
    size_t stage_bytes = 0;
    for (int k = 0; k < nb; ++k) {
      const fs_camera& cam = cams[v0 + k];
      stage_bytes += ((static_cast<size_t>(cam.width) * cam.height * msize) + 255) & ~size_t(255);
    }
    if (mask_memory == FS_MEM_HOST) FS_TRY(c->mask_stage.ensure(stage_bytes, "mask staging"));
    size_t stage_off = 0;
    for (int k = 0; k < nb; ++k) {
      const fs_camera& cam = cams[v0 + k];
      fill_view(cam, &vh[k]);
      vh[k].tile_base = tile_base;
      vh[k].state_off = state_off;
      const int nt = vh[k].tiles_x * vh[k].tiles_y;
      tile_base += nt;
      max_tiles = std::max(max_tiles, nt);
      const size_t npix = static_cast<size_t>(cam.width) * cam.height;
      state_off += static_cast<int64_t>(npix);
      const size_t mbytes = npix * msize;
      if (mask_memory == FS_MEM_DEVICE) {
        vh[k].mask = masks[v0 + k];
      } else {
        char* dst = c->mask_stage.as<char>() + stage_off;
        FS_CUDA(cudaMemcpyAsync(dst, masks[v0 + k], mbytes, cudaMemcpyHostToDevice, stream),
                "mask upload");
        vh[k].mask = dst;
        stage_off += (mbytes + 255) & ~size_t(255);
      }
    }
    const int total_tiles = tile_base;
    const int tile_bits = std::max(1, ceil_log2(total_tiles));
    const int64_t k_total = static_cast<int64_t>(nb) * n;
    FS_TRY(c->state.ensure(static_cast<size_t>(state_off) * 4, "pixel state"));
    const size_t sat_bytes = static_cast<size_t>((total_tiles + 63) / 64) * 8;
    FS_TRY(c->sat.ensure(sat_bytes, "tile flags"));
    const size_t subsat_bytes = static_cast<size_t>((4 * total_tiles + 63) / 64) * 8;
    FS_TRY(c->subsat.ensure(subsat_bytes, "sub-tile flags"));
    FS_TRY(c->ranges.ensure(static_cast<size_t>(total_tiles) * 8, "tile ranges"));
    fs::ViewParams* vd = c->views.as<fs::ViewParams>();
    float* state = c->state.as<float>();
    uint64_t* sat = c->sat.as<uint64_t>();
    FS_CUDA(cudaMemcpyAsync(vd, vh, sizeof(fs::ViewParams) * nb, cudaMemcpyHostToDevice, stream),
            "view upload");

    // project every Gaussian into the batch's views, sort by depth
    c->stats.kernel_launches += 3 + radix_launches(k_total, 32);
    FS_CUDA(fs::launch_project(n, nb, vd, s->pos_op.as<float4>(), s->cov.as<float4>(),
                               c->rec.as<fs::ProjRecord>(), c->foot.as<fs::Footprint>(),
                               c->cnt.as<uint32_t>(), c->key_a.as<uint32_t>(),
                               c->val_a.as<uint32_t>(), c->dlo.as<uint32_t>(), stream),
            "project");
    bool alt = false;
    FS_CUDA(fs::radix_sort_pairs(c->key_a.as<uint32_t>(), c->val_a.as<uint32_t>(),
                                 c->key_b.as<uint32_t>(), c->val_b.as<uint32_t>(), k_total, 32,
                                 c->sort_tmp.p, &alt, stream),
            "depth sort");
    uint32_t* sorted_key = alt ? c->key_b.as<uint32_t>() : c->key_a.as<uint32_t>();
    uint32_t* sorted_val = alt ? c->val_b.as<uint32_t>() : c->val_a.as<uint32_t>();
    FS_CUDA(fs::launch_depth_tie_fix(k_total, n, sorted_key, sorted_val, c->dlo.as<uint32_t>(),
                                     stream),
            "depth ties");
    uint64_t* subsat = c->subsat.as<uint64_t>();
    FS_CUDA(cudaMemsetAsync(sat, 0, sat_bytes, stream), "tile flags clear");
    FS_CUDA(cudaMemsetAsync(subsat, 0, subsat_bytes, stream), "sub-tile flags clear");
    FS_CUDA(fs::launch_state_init(vd, nb, max_tiles, E, mask_dtype, state, sat, subsat, ctr,
                                  stream),
            "pixel state");
    c->stats.views += nb;
    c->stats.pixels += state_off;

    // front-to-back depth chunks: a chunk lists only tiles not yet saturated
    const int chunks = std::max(1, c->depth_chunks);
    int64_t p0 = 0;
    for (int ci = 0; ci < chunks; ++ci) {
      const int64_t p1 = (ci == chunks - 1) ? k_total : (k_total >> (chunks - 1 - ci));
      const int64_t n_pos = p1 - p0;
      if (n_pos <= 0) continue;
      uint32_t* total_d = c->total.as<uint32_t>();
      c->stats.kernel_launches += 1 + scan_launches(n_pos);
      FS_CUDA(fs::launch_chunk_count(p0, n_pos, n, vd, sorted_val, c->cnt.as<uint32_t>(),
                                     c->foot.as<fs::Footprint>(), sat, c->ccnt.as<uint32_t>(),
                                     stream),
              "chunk count");
      FS_CUDA(fs::exclusive_scan(c->ccnt.as<uint32_t>(), nullptr, c->offs.as<uint32_t>(), n_pos,
                                 total_d, c->scan_tmp.p, stream),
              "count scan");
      FS_CUDA(cudaMemcpyAsync(total_h, total_d, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream),
              "count readback");
      FS_CUDA(cudaStreamSynchronize(stream), "count readback");
      const int64_t I = *total_h;
      if (I >= (static_cast<int64_t>(1) << 31))
        return fail(FS_UNSUPPORTED, "fs_accumulate: %lld list entries in one chunk; use fewer "
                    "views per batch", (long long)I);
      c->stats.list_entries += I;
      if (I == 0) {
        p0 = p1;
        continue;
      }
      FS_TRY(c->lk_a.ensure(static_cast<size_t>(I) * 4, "list keys"));
      FS_TRY(c->lv_a.ensure(static_cast<size_t>(I) * 4, "list values"));
      FS_TRY(c->lk_b.ensure(static_cast<size_t>(I) * 4, "list keys"));
      FS_TRY(c->lv_b.ensure(static_cast<size_t>(I) * 4, "list values"));
      FS_TRY(c->sort_tmp.ensure(fs::radix_temp_bytes(std::max<int64_t>(I, kcap)), "sort temp"));
      c->stats.kernel_launches += 3 + radix_launches(I, tile_bits);
      FS_CUDA(fs::launch_emit(p0, n_pos, n, vd, sorted_val, c->offs.as<uint32_t>(),
                              c->ccnt.as<uint32_t>(), c->cnt.as<uint32_t>(),
                              c->foot.as<fs::Footprint>(), sat,
                              c->lk_a.as<uint32_t>(), c->lv_a.as<uint32_t>(), ctr, stream),
              "emit");
      bool alt2 = false;
      FS_CUDA(fs::radix_sort_pairs(c->lk_a.as<uint32_t>(), c->lv_a.as<uint32_t>(),
                                   c->lk_b.as<uint32_t>(), c->lv_b.as<uint32_t>(), I, tile_bits,
                                   c->sort_tmp.p, &alt2, stream),
              "tile sort");
      const uint32_t* lkey = alt2 ? c->lk_b.as<uint32_t>() : c->lk_a.as<uint32_t>();
      const uint32_t* lval = alt2 ? c->lv_b.as<uint32_t>() : c->lv_a.as<uint32_t>();
      FS_CUDA(cudaMemsetAsync(c->ranges.p, 0, static_cast<size_t>(total_tiles) * 8, stream),
              "ranges clear");
      FS_CUDA(fs::launch_ranges(I, lkey, c->ranges.as<uint2>(), stream), "ranges");
      cudaEvent_t ev0 = nullptr, ev1 = nullptr;
      if (c->time_stages) {
        while (c->events.size() < c->events_used + 2) {
          cudaEvent_t e;
          FS_CUDA(cudaEventCreate(&e), "cudaEventCreate");
          c->events.push_back(e);
        }
        ev0 = c->events[c->events_used];
        ev1 = c->events[c->events_used + 1];
        c->events_used += 2;
        FS_CUDA(cudaEventRecord(ev0, stream), "cudaEventRecord");
      }
      FS_CUDA(fs::launch_blend(vd, nb, max_tiles, c->ranges.as<uint2>(), lval,
                               c->rec.as<fs::ProjRecord>(), n, E, mask_dtype, table, table_dtype,
                               state, sat, subsat, ctr, stream),
              "blend");
      if (ev1) FS_CUDA(cudaEventRecord(ev1, stream), "cudaEventRecord");
      p0 = p1;
    }
  }
  return FS_OK;
}

fs_status check_accumulate_args(fs_ctx* c, const fs_scene* s, const fs_camera* cams, int32_t V,
                                const void* const* masks, int32_t mask_dtype, int32_t mask_memory,
                                int32_t E) {
  if (!c || !s) return fail(FS_INVALID_ARGUMENT, "NULL context or scene");
  if (s->ctx != c) return fail(FS_INVALID_ARGUMENT, "scene belongs to another context");
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
  return accumulate_impl(c, s, cams, V, masks, mask_dtype, mask_memory, E, table, table_dtype, st);
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
  const size_t tbytes = static_cast<size_t>(n) * E * dtype_size(tdt);
  const bool dev_out = out->memory == FS_MEM_DEVICE;
  void* table = (dev_out && out->table) ? out->table : nullptr;
  if (!table) {
    FS_TRY(c->table_tmp.ensure(tbytes > 0 ? tbytes : 8, "table"));
    table = c->table_tmp.p;
  }
  c->stats = fs_stats{};
  c->events_used = 0;
  FS_CUDA(cudaMemsetAsync(c->counters.p, 0, c->counters.bytes, st), "counters clear");
  if (tbytes) FS_CUDA(cudaMemsetAsync(table, 0, tbytes, st), "table clear");
  FS_TRY(accumulate_impl(c, s, cams, V, masks, mask_dtype, mask_memory, E, table, tdt, st));
  uint64_t* bits = out->member_bits;
  int32_t* label = out->label;
  float* margin = out->margin;
  if (!dev_out) {
    const size_t nn = static_cast<size_t>(n > 0 ? n : 1);
    if (bits) { FS_TRY(c->bits_tmp.ensure(nn * 8, "bits")); bits = c->bits_tmp.as<uint64_t>(); }
    if (label) { FS_TRY(c->label_tmp.ensure(nn * 4, "labels")); label = c->label_tmp.as<int32_t>(); }
    if (margin) { FS_TRY(c->margin_tmp.ensure(nn * 4, "margins")); margin = c->margin_tmp.as<float>(); }
  }
  if (bits || label || margin) {
    FS_CUDA(fs::launch_assign(table, tdt, n, E, gamma, bits, label, margin, st), "assign");
    if (n > 0) c->stats.kernel_launches += 1;
  }
  if (!dev_out && n > 0) {
    if (out->table)
      FS_CUDA(cudaMemcpyAsync(out->table, table, tbytes, cudaMemcpyDeviceToHost, st), "table D2H");
    if (bits)
      FS_CUDA(cudaMemcpyAsync(out->member_bits, bits, n * 8, cudaMemcpyDeviceToHost, st), "D2H");
    if (label)
      FS_CUDA(cudaMemcpyAsync(out->label, label, n * 4, cudaMemcpyDeviceToHost, st), "D2H");
    if (margin)
      FS_CUDA(cudaMemcpyAsync(out->margin, margin, n * 4, cudaMemcpyDeviceToHost, st), "D2H");
  }
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
  if (ch[fs::kBinningMismatch])
    return fail(FS_CUDA_ERROR, "internal error: tile binning count and emission disagreed for "
                "%llu Gaussian(s)", ch[fs::kBinningMismatch]);
  double ms = 0.0;
  for (size_t k = 0; k + 1 < c->events_used; k += 2) {
    float t = 0.f;
    FS_CUDA(cudaEventElapsedTime(&t, c->events[k], c->events[k + 1]), "cudaEventElapsedTime");
    ms += t;
  }
  c->stats.blend_ms = ms;
  c->stats.blend_launches = static_cast<int64_t>(c->events_used / 2);
  if (stats) *stats = c->stats;
  return FS_OK;
}

}  // extern "C"
