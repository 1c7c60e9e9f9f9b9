// Request server: continuous batching of segmentation requests against
// resident scenes (the C ABI's fs_server_* calls).
//
// Each of `slots` worker threads owns a context and a CUDA stream.  Requests
// wait in one FIFO queue; a worker that is free admits the oldest queued
// request whose estimated device footprint fits beside the running ones
// (a request that fits nowhere runs alone once the device is idle), runs its
// fs_solve on its own stream and leaves the results in host memory for
// fs_server_fetch.  Requests therefore start as soon as a slot and memory
// free up, and several requests' kernels overlap on the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/flashsplat.h"
#include "fs_internal.h"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  int64_t ticket = 0;
  int32_t scene = 0;
  std::vector<fs_camera> cams;
  std::vector<std::vector<uint8_t>> masks;  // host copies, row-major H x W
  int32_t mask_dtype = FS_U8;
  int32_t E = 2;
  float gamma = 0.f;
  int64_t est = 0;  // estimated device bytes while running
  bool running = false, done = false;
  std::string error;
  std::vector<uint64_t> bits;
  std::vector<int32_t> label;
  std::vector<float> margin;
  fs_server_info info{};
};

struct SceneEntry {
  fs_scene* scene = nullptr;
  int64_t n = 0;
  bool tuned = false;
  int views_per_batch = 50, depth_chunks = 6;
  std::mutex tune_mu;
  // graphs on: a captured solve of the scene's last (cameras, E, gamma, mask
  // dtype), its device mask buffers and outputs; one replay at a time
  std::mutex graph_mu;
  fs_graph* graph = nullptr;
  std::vector<fs_camera> g_cams;
  int32_t g_E = 0, g_dtype = 0;
  float g_gamma = 0.f;
  std::vector<void*> g_masks;
  void* g_out = nullptr;  // bits [n] | label [n] | margin [n]
  double last_use = 0.0;
};

// Device bytes a request needs while it runs: the context's per-batch
// window (records, footprints, keys, list entries), the FP64 table and its
// rounding, the staged masks and the per-pixel state of one batch.
int64_t footprint(int64_t n, int vb, const std::vector<fs_camera>& cams, int32_t mask_dtype,
                  int32_t E) {
  const int64_t nb = std::min<int64_t>(vb, static_cast<int64_t>(cams.size()));
  const int64_t window = nb * n * (64 + 32 + 4 * 9) + nb * n * 2 * 16;
  int64_t pixels = 0, batch_pixels = 0;
  for (size_t v = 0; v < cams.size(); ++v) {
    const int64_t p = static_cast<int64_t>(cams[v].width) * cams[v].height;
    pixels += p;
    if (static_cast<int64_t>(v) < nb) batch_pixels += p;
  }
  const int64_t msize = mask_dtype == FS_I32 ? 4 : 1;
  return window + n * E * 12 + n * 16 + pixels * msize + batch_pixels * 4 + (64 << 20);
}

}  // namespace

struct fs_server {
  int device = 0;
  int n_slots = 4;
  int64_t budget = 0;
  bool autotune = false;
  int max_graphs = 0;  // scenes whose captured solve is kept (0: no graphs)
  std::mutex graphs_mu;
  int live_graphs = 0;
  fs_ctx* scene_ctx = nullptr;
  std::vector<fs_ctx*> ctx;
  std::vector<cudaStream_t> streams;
  std::mutex scenes_mu;
  std::vector<std::unique_ptr<SceneEntry>> scenes;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
  int64_t next_ticket = 1;
  int64_t reserved = 0;
  int running = 0;
  bool stopping = false;
  std::vector<std::thread> threads;
};

namespace {

// Index of the first queued request that fits the budget now, or -1.
int admissible(const fs_server* s) {
  for (size_t k = 0; k < s->queue.size(); ++k) {
    const Request* r = s->queue[k];
    if (s->reserved + r->est <= s->budget || s->running == 0) return static_cast<int>(k);
  }
  return -1;
}

fs_status solve_request(fs_server* s, int slot, const SceneEntry& se, Request* r, int32_t V,
                        fs_stats* stats) {
  std::vector<const void*> mp(static_cast<size_t>(V));
  for (int32_t v = 0; v < V; ++v) mp[v] = r->masks[v].data();
  fs_result out{};
  out.memory = FS_MEM_HOST;
  out.table_dtype = FS_F32;
  out.table = nullptr;
  out.member_bits = r->E <= 64 ? r->bits.data() : nullptr;
  out.label = r->label.data();
  out.margin = r->margin.data();
  fs_status st = fs_solve(s->ctx[slot], se.scene, r->cams.data(), V, mp.data(), r->mask_dtype,
                          FS_MEM_HOST, r->E, r->gamma, &out, s->streams[slot]);
  if (st == FS_OK) st = fs_synchronize(s->ctx[slot], s->streams[slot], stats);
  return st;
}

fs_status fail(fs_status st, const std::string& msg) {
  fs::set_last_error(msg.c_str());
  return st;
}

// Frees a scene's captured solve (its graph_mu held).
void drop_graph(SceneEntry& se) {
  if (se.graph) fs_graph_destroy(se.graph);
  se.graph = nullptr;
  for (void* m : se.g_masks) cudaFree(m);
  se.g_masks.clear();
  if (se.g_out) cudaFree(se.g_out);
  se.g_out = nullptr;
}

// Room for one more captured solve: under the cap, or after dropping the
// least recently used graph of another scene that is not replaying.
void make_room(fs_server* s, SceneEntry* self) {
  std::lock_guard<std::mutex> lk(s->graphs_mu);
  while (s->live_graphs >= s->max_graphs) {
    SceneEntry* lru = nullptr;
    {
      std::lock_guard<std::mutex> g(s->scenes_mu);
      for (auto& e : s->scenes)
        if (e.get() != self && e->graph && (!lru || e->last_use < lru->last_use)) lru = e.get();
    }
    if (!lru || !lru->graph_mu.try_lock()) break;  // nothing to drop now: go over the cap
    drop_graph(*lru);
    lru->graph_mu.unlock();
    --s->live_graphs;
  }
  ++s->live_graphs;
}

// A request through its scene's captured solve: the masks are copied into
// the graph's buffers and the graph replayed; a request with other cameras,
// E, gamma or mask dtype captures the scene anew.
fs_status solve_with_graph(fs_server* s, int slot, SceneEntry& se, Request* r,
                           fs_stats* stats) {
  std::lock_guard<std::mutex> gl(se.graph_mu);
  const int32_t V = static_cast<int32_t>(r->cams.size());
  const size_t msize = r->mask_dtype == FS_I32 ? 4 : 1;
  const size_t n = static_cast<size_t>(se.n);
  cudaStream_t st = s->streams[slot];
  const bool same = se.graph && se.g_cams.size() == r->cams.size() &&
                    std::equal(reinterpret_cast<const char*>(se.g_cams.data()),
                               reinterpret_cast<const char*>(se.g_cams.data() + V),
                               reinterpret_cast<const char*>(r->cams.data())) &&
                    se.g_E == r->E && se.g_gamma == r->gamma && se.g_dtype == r->mask_dtype;
  if (!same) {
    if (se.graph) {
      drop_graph(se);
      std::lock_guard<std::mutex> lk(s->graphs_mu);
      --s->live_graphs;
    }
    make_room(s, &se);
    cudaError_t e = cudaMalloc(&se.g_out, n * 16);
    for (int32_t v = 0; v < V && e == cudaSuccess; ++v) {
      void* m = nullptr;
      e = cudaMalloc(&m, r->masks[v].size());
      if (e == cudaSuccess) se.g_masks.push_back(m);
      if (e == cudaSuccess) e = cudaMemcpy(m, r->masks[v].data(), r->masks[v].size(),
                                           cudaMemcpyHostToDevice);
    }
    fs_status status = FS_OK;
    if (e != cudaSuccess) {
      status = fail(FS_OUT_OF_MEMORY, std::string("captured solve buffers: ") +
                                          cudaGetErrorString(e));
    } else {
      char* o = static_cast<char*>(se.g_out);
      fs_result out{};
      out.memory = FS_MEM_DEVICE;
      out.table_dtype = FS_F32;
      out.table = nullptr;
      out.member_bits = r->E <= 64 ? reinterpret_cast<uint64_t*>(o) : nullptr;
      out.label = reinterpret_cast<int32_t*>(o + n * 8);
      out.margin = reinterpret_cast<float*>(o + n * 12);
      std::vector<const void*> mp(se.g_masks.begin(), se.g_masks.end());
      status = fs_graph_create(s->ctx[slot], se.scene, r->cams.data(), V, mp.data(),
                               r->mask_dtype, r->E, r->gamma, &out, &se.graph);
    }
    if (status != FS_OK) {
      drop_graph(se);
      std::lock_guard<std::mutex> lk(s->graphs_mu);
      --s->live_graphs;
      return status;
    }
    se.g_cams = r->cams;
    se.g_E = r->E;
    se.g_gamma = r->gamma;
    se.g_dtype = r->mask_dtype;
  } else {
    for (int32_t v = 0; v < V; ++v)
      if (cudaMemcpyAsync(se.g_masks[v], r->masks[v].data(), r->masks[v].size(),
                          cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail(FS_CUDA_ERROR, "captured solve: mask upload failed");
  }
  se.last_use = now_s();
  fs_status status = fs_graph_launch(se.graph, st);
  const char* o = static_cast<const char*>(se.g_out);
  if (status == FS_OK && r->E <= 64 &&
      cudaMemcpyAsync(r->bits.data(), o, n * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    status = fail(FS_CUDA_ERROR, "captured solve: result copy failed");
  if (status == FS_OK &&
      (cudaMemcpyAsync(r->label.data(), o + n * 8, n * 4, cudaMemcpyDeviceToHost, st) !=
           cudaSuccess ||
       cudaMemcpyAsync(r->margin.data(), o + n * 12, n * 4, cudaMemcpyDeviceToHost, st) !=
           cudaSuccess))
    status = fail(FS_CUDA_ERROR, "captured solve: result copy failed");
  if (status == FS_OK) status = fs_graph_synchronize(se.graph, st, stats);
  (void)msize;
  return status;
}

// The first request of a scene (autotune on): time a few batching settings
// on a sample of its views and keep the fastest for the scene.
void tune_scene(fs_server* s, int slot, SceneEntry& se, Request* r) {
  static const int cand[][2] = {{50, 6}, {32, 5}, {64, 6}, {16, 4}, {50, 4}};
  const int32_t V = static_cast<int32_t>(std::min<size_t>(r->cams.size(), 32));
  double best = 1e300;
  fs_stats st{};
  for (const auto& c : cand) {
    fs::ctx_set_batching(s->ctx[slot], c[0], c[1]);
    const double t0 = now_s();
    if (solve_request(s, slot, se, r, V, &st) != FS_OK) continue;
    const double dt = now_s() - t0;
    if (dt < best) {
      best = dt;
      se.views_per_batch = c[0];
      se.depth_chunks = c[1];
    }
  }
}

void worker(fs_server* s, int slot) {
  cudaSetDevice(s->device);
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      int k = -1;
      s->cv_work.wait(lk, [&] { return s->stopping || (k = admissible(s)) >= 0; });
      if (s->stopping) return;
      r = s->queue[static_cast<size_t>(k)];
      s->queue.erase(s->queue.begin() + k);
      r->running = true;
      s->reserved += r->est;
      s->running += 1;
      r->info.start_s = now_s();
      r->info.slot = slot;
    }
    SceneEntry* se;
    {
      std::lock_guard<std::mutex> g(s->scenes_mu);
      se = s->scenes[static_cast<size_t>(r->scene)].get();
    }
    if (s->autotune) {
      std::lock_guard<std::mutex> g(se->tune_mu);
      if (!se->tuned) {
        tune_scene(s, slot, *se, r);
        se->tuned = true;
      }
    }
    fs::ctx_set_batching(s->ctx[slot], se->views_per_batch, se->depth_chunks);
    r->info.views_per_batch = se->views_per_batch;
    r->info.depth_chunks = se->depth_chunks;
    const fs_status st =
        s->max_graphs > 0
            ? solve_with_graph(s, slot, *se, r, &r->info.stats)
            : solve_request(s, slot, *se, r, static_cast<int32_t>(r->cams.size()),
                            &r->info.stats);
    if (st != FS_OK) r->error = fs_last_error();
    // keep the slot's retained workspace within its share of the budget
    if (static_cast<int64_t>(fs::ctx_workspace_bytes(s->ctx[slot])) > s->budget / s->n_slots) {
      cudaStreamSynchronize(s->streams[slot]);
      fs::ctx_release_workspace(s->ctx[slot]);
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r->info.status = st;
      r->info.done = 1;
      r->info.done_s = now_s();
      r->running = false;
      r->done = true;
      r->masks.clear();
      r->masks.shrink_to_fit();
      s->reserved -= r->est;
      s->running -= 1;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

fs_status fs_server_create(const fs_server_options* opt, fs_server** out) {
  if (!out) return fail(FS_INVALID_ARGUMENT, "fs_server_create: out is NULL");
  *out = nullptr;
  std::unique_ptr<fs_server> s(new (std::nothrow) fs_server());
  if (!s) return fail(FS_OUT_OF_MEMORY, "fs_server_create: host allocation failed");
  s->device = opt ? opt->device : 0;
  s->n_slots = (opt && opt->slots > 0) ? std::min(opt->slots, 64) : 4;
  s->autotune = opt && opt->autotune;
  s->max_graphs = (opt && opt->graphs > 0) ? opt->graphs : 0;
  fs_options o{};
  o.recheck_reproject = 1;  // bounded per-request memory: no per-view record store
  fs_status st = fs_create(&s->scene_ctx, s->device, &o);
  if (st != FS_OK) return st;
  if (cudaSetDevice(s->device) != cudaSuccess)
    return fail(FS_CUDA_ERROR, "fs_server_create: cudaSetDevice failed");
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  s->budget = (opt && opt->budget_bytes > 0) ? opt->budget_bytes
                                             : static_cast<int64_t>(free_b / 2);
  for (int k = 0; k < s->n_slots; ++k) {
    fs_ctx* c = nullptr;
    if ((st = fs_create(&c, s->device, &o)) != FS_OK) {
      fs_server_destroy(s.release());
      return st;
    }
    s->ctx.push_back(c);
    cudaStream_t str = nullptr;
    if (cudaStreamCreateWithFlags(&str, cudaStreamNonBlocking) != cudaSuccess) {
      fs_server_destroy(s.release());
      return fail(FS_CUDA_ERROR, "fs_server_create: cudaStreamCreate failed");
    }
    s->streams.push_back(str);
  }
  fs_server* raw = s.get();
  for (int k = 0; k < raw->n_slots; ++k) raw->threads.emplace_back(worker, raw, k);
  *out = s.release();
  return FS_OK;
}

fs_status fs_server_add_scene(fs_server* s, const fs_gaussians* g, int32_t* scene_id) {
  if (!s || !scene_id) return fail(FS_INVALID_ARGUMENT, "fs_server_add_scene: NULL argument");
  std::lock_guard<std::mutex> lk(s->scenes_mu);
  std::unique_ptr<SceneEntry> e(new SceneEntry());
  fs_status st = fs_scene_create(s->scene_ctx, g, &e->scene);
  if (st != FS_OK) return st;
  e->n = fs_scene_size(e->scene);
  *scene_id = static_cast<int32_t>(s->scenes.size());
  s->scenes.push_back(std::move(e));
  return FS_OK;
}

fs_status fs_server_submit(fs_server* s, int32_t scene_id, const fs_camera* cams,
                           int32_t n_views, const void* const* masks, int32_t mask_dtype,
                           int32_t E, float gamma, int64_t* ticket) {
  if (!s || !ticket) return fail(FS_INVALID_ARGUMENT, "fs_server_submit: NULL argument");
  if (n_views < 1 || !cams || !masks)
    return fail(FS_INVALID_ARGUMENT, "fs_server_submit: no views");
  if (mask_dtype != FS_U8 && mask_dtype != FS_I32)
    return fail(FS_INVALID_ARGUMENT, "fs_server_submit: mask dtype must be FS_U8 or FS_I32");
  if (E < 1 || E > 4096) return fail(FS_INVALID_ARGUMENT, "fs_server_submit: E out of range");
  if (!(gamma >= -1.f && gamma <= 1.f))
    return fail(FS_INVALID_ARGUMENT, "fs_server_submit: gamma outside [-1, 1]");
  int64_t n = 0;
  int vb = 16;
  {
    std::lock_guard<std::mutex> lk(s->scenes_mu);
    if (scene_id < 0 || scene_id >= static_cast<int32_t>(s->scenes.size()))
      return fail(FS_INVALID_ARGUMENT, "fs_server_submit: unknown scene id");
    const SceneEntry& e = *s->scenes[static_cast<size_t>(scene_id)];
    n = e.n;
    // before its scene is tuned a request may run with the largest batch
    vb = (s->autotune && !e.tuned) ? 64 : e.views_per_batch;
  }
  std::unique_ptr<Request> r(new Request());
  r->scene = scene_id;
  r->cams.assign(cams, cams + n_views);
  const size_t msize = mask_dtype == FS_I32 ? 4 : 1;
  r->masks.resize(static_cast<size_t>(n_views));
  for (int32_t v = 0; v < n_views; ++v) {
    if (!masks[v] || cams[v].width < 1 || cams[v].height < 1)
      return fail(FS_INVALID_ARGUMENT, "fs_server_submit: bad mask or camera size");
    const size_t bytes = static_cast<size_t>(cams[v].width) * cams[v].height * msize;
    const uint8_t* src = static_cast<const uint8_t*>(masks[v]);
    r->masks[v].assign(src, src + bytes);
  }
  r->mask_dtype = mask_dtype;
  r->E = E;
  r->gamma = gamma;
  r->bits.resize(static_cast<size_t>(n > 0 ? n : 1));
  r->label.resize(static_cast<size_t>(n > 0 ? n : 1));
  r->margin.resize(static_cast<size_t>(n > 0 ? n : 1));
  r->est = footprint(n, vb, r->cams, mask_dtype, E);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return fail(FS_CANCELLED, "fs_server_submit: server is stopping");
    r->ticket = s->next_ticket++;
    r->info.submit_s = now_s();
    r->info.bytes_estimate = r->est;
    *ticket = r->ticket;
    s->queue.push_back(r.get());
    s->reqs[r->ticket] = std::move(r);
  }
  s->cv_work.notify_one();
  return FS_OK;
}

fs_status fs_server_fetch(fs_server* s, int64_t ticket, int32_t wait, uint64_t* member_bits,
                          int32_t* label, float* margin, fs_server_info* info) {
  return fs_server_fetch_for(s, ticket, wait ? -1 : 0, member_bits, label, margin, info);
}

fs_status fs_server_fetch_for(fs_server* s, int64_t ticket, int32_t timeout_ms,
                              uint64_t* member_bits, int32_t* label, float* margin,
                              fs_server_info* info) {
  if (!s) return fail(FS_INVALID_ARGUMENT, "fs_server_fetch: NULL server");
  std::unique_ptr<Request> r;
  int64_t n = 0;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(FS_INVALID_ARGUMENT, "fs_server_fetch: unknown ticket");
    Request* rp = it->second.get();
    if (!rp->done) {
      if (timeout_ms == 0) return fail(FS_TIMEOUT, "fs_server_fetch: request not finished");
      if (timeout_ms < 0) {
        s->cv_done.wait(lk, [&] { return rp->done; });
      } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                      [&] { return rp->done; })) {
        return fail(FS_TIMEOUT, "fs_server_fetch: request not finished within the limit");
      }
    }
    r = std::move(s->reqs[ticket]);
    s->reqs.erase(ticket);
  }
  {
    std::lock_guard<std::mutex> lk(s->scenes_mu);
    n = s->scenes[static_cast<size_t>(r->scene)]->n;
  }
  const fs_status st = static_cast<fs_status>(r->info.status);
  if (st == FS_OK) {
    if (member_bits && r->E <= 64) std::copy(r->bits.begin(), r->bits.begin() + n, member_bits);
    if (label) std::copy(r->label.begin(), r->label.begin() + n, label);
    if (margin) std::copy(r->margin.begin(), r->margin.begin() + n, margin);
  }
  if (info) *info = r->info;
  if (st != FS_OK) return fail(st, r->error.empty() ? "request failed" : r->error);
  return FS_OK;
}

fs_status fs_server_cancel(fs_server* s, int64_t ticket) {
  if (!s) return fail(FS_INVALID_ARGUMENT, "fs_server_cancel: NULL server");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(FS_INVALID_ARGUMENT, "fs_server_cancel: unknown ticket");
    Request* r = it->second.get();
    if (r->running || r->done)
      return fail(FS_UNSUPPORTED, "fs_server_cancel: request already started");
    s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
    r->done = true;
    r->info.done = 1;
    r->info.status = FS_CANCELLED;
    r->info.done_s = now_s();
    r->error = "cancelled";
  }
  s->cv_done.notify_all();
  return FS_OK;
}

fs_status fs_server_destroy(fs_server* s) {
  if (!s) return FS_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    for (Request* r : s->queue) {
      r->done = true;
      r->info.done = 1;
      r->info.status = FS_CANCELLED;
    }
    s->queue.clear();
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  for (std::thread& t : s->threads) t.join();
  for (size_t k = 0; k < s->ctx.size(); ++k) {
    if (k < s->streams.size() && s->streams[k]) {
      cudaStreamSynchronize(s->streams[k]);
      cudaStreamDestroy(s->streams[k]);
    }
    fs_destroy(s->ctx[k]);
  }
  for (auto& e : s->scenes) {
    drop_graph(*e);
    fs_scene_destroy(e->scene);
  }
  if (s->scene_ctx) fs_destroy(s->scene_ctx);
  delete s;
  return FS_OK;
}

}  // extern "C"
