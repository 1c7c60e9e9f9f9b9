// fs_solve_noalloc: the whole solve for small scenes without allocating any
// memory.  Its working memory is one file-scope __device__ array of fixed size
// that every GPU loading the library keeps until the process exits.
//
// Who needs it: code that runs where allocating device memory is not an
// option -- for instance a plugin living inside a host application that owns
// every byte of device memory through its own pool, or a latency-critical
// loop that must not pay for cudaMalloc/cudaFree (which can synchronise the
// whole device).  Such callers pass their inputs and outputs; nothing else is
// allocated, neither by this code nor by any library routine it calls.
//
// The array's host-side name is only a stand-in for the device symbol: the
// address the kernels receive is obtained with cudaGetSymbolAddress, once per
// device, with that device current, the first time the device is used here.
// Every call shares the array and finds the previous call's contents in it;
// everything that must start at zero is cleared on each call.  Two calls whose
// work overlaps on the GPU (other streams, other host threads) race on the
// array and must not be issued.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "../../include/flashsplat.h"
#include "fs_common.cuh"
#include "fs_internal.h"

namespace fs {
namespace {

// ---- fixed capacity ------------------------------------------------------
constexpr int64_t kNA_N = FS_NOALLOC_MAX_GAUSSIANS;
constexpr int kNA_Side = FS_NOALLOC_MAX_SIDE;
constexpr int64_t kNA_Entries = FS_NOALLOC_MAX_LIST_ENTRIES;
constexpr int kNA_Tiles = (kNA_Side / kTile) * (kNA_Side / kTile);
constexpr size_t kNA_SortTmp = 512 * 1024;  // >= radix_temp_bytes(kNA_Entries), checked at run time
constexpr size_t kNA_ScanTmp = 4 * 1024;    // >= scan_temp_bytes(kNA_N), checked at run time

constexpr size_t al(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// region offsets in the scratch array
constexpr size_t oPos = 0;
constexpr size_t oCov = oPos + al(kNA_N * 16);
constexpr size_t oViews = oCov + al(kNA_N * 48);
constexpr size_t oRec = oViews + al(sizeof(ViewParams));
constexpr size_t oFoot = oRec + al(kNA_N * sizeof(ProjRecord));
constexpr size_t oCnt = oFoot + al(kNA_N * sizeof(Footprint));
constexpr size_t oKeyA = oCnt + al(kNA_N * 4);
constexpr size_t oValA = oKeyA + al(kNA_N * 4);
constexpr size_t oKeyB = oValA + al(kNA_N * 4);
constexpr size_t oValB = oKeyB + al(kNA_N * 4);
constexpr size_t oOffs = oValB + al(kNA_N * 4);
constexpr size_t oCcnt = oOffs + al(kNA_N * 4);
constexpr size_t oDlo = oCcnt + al(kNA_N * 4);
constexpr size_t oLkA = oDlo + al(kNA_N * 4);
constexpr size_t oLvA = oLkA + al(kNA_Entries * 4);
constexpr size_t oLkB = oLvA + al(kNA_Entries * 4);
constexpr size_t oLvB = oLkB + al(kNA_Entries * 4);
constexpr size_t oRanges = oLvB + al(kNA_Entries * 4);
constexpr size_t oState = oRanges + al(kNA_Tiles * 8);
constexpr size_t oSat = oState + al(static_cast<size_t>(kNA_Side) * kNA_Side * 4);
constexpr size_t oSubsat = oSat + al(kNA_Tiles);
constexpr size_t oSortTmp = oSubsat + al(4 * kNA_Tiles);
constexpr size_t oScanTmp = oSortTmp + al(kNA_SortTmp);
constexpr size_t oWords = oScanTmp + al(kNA_ScanTmp);  // total (u32), error word (u32)
constexpr size_t oCounters = oWords + 256;
constexpr size_t kNA_Bytes = oCounters + al(kNumCounters * 8);

}  // namespace
}  // namespace fs

// The shared working memory (see the top of this file).
static __device__ __align__(256) unsigned char g_noalloc_scratch[fs::kNA_Bytes];

namespace {

fs_status na_fail(fs_status st, const char* msg) {
  fs::set_last_error(msg);
  return st;
}

fs_status na_cuda(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof(buf), "fs_solve_noalloc: %s: %s", what, cudaGetErrorString(e));
  fs::set_last_error(buf);
  return FS_CUDA_ERROR;
}

#define NA_CUDA(expr, what)                                  \
  do {                                                       \
    cudaError_t e_ = (expr);                                 \
    if (e_ != cudaSuccess) return na_cuda(e_, what);         \
  } while (0)

constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
unsigned char* g_na_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device` (current), looked up once.
fs_status scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return na_fail(FS_UNSUPPORTED, "device index too large");
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return na_cuda(e, "cudaGetSymbolAddress");
    g_na_ptr[device] = static_cast<unsigned char*>(p);
  }
  *out = g_na_ptr[device];
  return FS_OK;
}

int bits_for(int64_t x) {
  int b = 0;
  while ((static_cast<int64_t>(1) << b) < x) ++b;
  return std::max(1, b);
}

}  // namespace

extern "C" fs_status fs_solve_noalloc(int32_t device, const fs_gaussians* g, const fs_camera* cams,
                                      int32_t n_views, const void* const* masks,
                                      int32_t mask_dtype, int32_t E, float gamma, float* table,
                                      uint64_t* member_bits, int32_t* label, float* margin,
                                      void* stream) {
  using namespace fs;
  if (!g || !table) return na_fail(FS_INVALID_ARGUMENT, "fs_solve_noalloc: NULL scene or table");
  const int64_t n = g->n;
  if (n < 1 || n > kNA_N)
    return na_fail(FS_INVALID_ARGUMENT,
                   "fs_solve_noalloc: the scene must hold 1..FS_NOALLOC_MAX_GAUSSIANS Gaussians");
  if (g->memory != FS_MEM_DEVICE || g->quat_dtype != FS_F32 || g->scale_dtype != FS_F32 ||
      g->opacity_dtype != FS_F32 || !g->mean || !g->quat || !g->scale || !g->opacity)
    return na_fail(FS_INVALID_ARGUMENT,
                   "fs_solve_noalloc: Gaussian attributes must be FS_F32 device arrays");
  if (n_views < 0 || (n_views > 0 && (!cams || !masks)))
    return na_fail(FS_INVALID_ARGUMENT, "fs_solve_noalloc: bad cameras or masks");
  if (mask_dtype != FS_U8 && mask_dtype != FS_I32)
    return na_fail(FS_INVALID_ARGUMENT, "fs_solve_noalloc: mask dtype must be FS_U8 or FS_I32");
  if (E < 1 || E > kMaxLabels)
    return na_fail(FS_INVALID_ARGUMENT, "fs_solve_noalloc: E out of [1, 4096]");
  if (!(gamma >= -1.f && gamma <= 1.f))
    return na_fail(FS_INVALID_ARGUMENT, "fs_solve_noalloc: gamma outside [-1, 1]");
  if (member_bits && E > 64)
    return na_fail(FS_UNSUPPORTED, "fs_solve_noalloc: member_bits needs E <= 64");
  for (int v = 0; v < n_views; ++v) {
    const fs_camera& c = cams[v];
    if (c.width < 1 || c.height < 1 || c.width > kNA_Side || c.height > kNA_Side)
      return na_fail(FS_INVALID_ARGUMENT,
                     "fs_solve_noalloc: every view must be at most FS_NOALLOC_MAX_SIDE pixels wide "
                     "and high");
    if (!(c.fx > 0 && c.fy > 0) || !masks[v])
      return na_fail(FS_INVALID_ARGUMENT, "fs_solve_noalloc: bad camera or NULL mask");
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double d = 0;
        for (int k = 0; k < 3; ++k) d += c.R[3 * a + k] * c.R[3 * b + k];
        if (!(fabs(d - (a == b ? 1.0 : 0.0)) <= 1e-5))
          return na_fail(FS_INVALID_ARGUMENT, "fs_solve_noalloc: camera R is not a rotation");
      }
  }
  if (radix_temp_bytes(kNA_Entries) > kNA_SortTmp || scan_temp_bytes(kNA_N) > kNA_ScanTmp)
    return na_fail(FS_UNSUPPORTED, "fs_solve_noalloc: internal scratch layout too small");

  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return na_fail(FS_CUDA_ERROR, "cudaGetDevice failed");
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return na_fail(FS_INVALID_ARGUMENT, "fs_solve_noalloc: bad device");
  }
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};

  unsigned char* S = nullptr;
  if (fs_status st = scratch_address(device, &S)) return st;
  cudaStream_t strm = static_cast<cudaStream_t>(stream);
  float4* pos = reinterpret_cast<float4*>(S + oPos);
  float4* cov = reinterpret_cast<float4*>(S + oCov);
  ViewParams* vd = reinterpret_cast<ViewParams*>(S + oViews);
  ProjRecord* rec = reinterpret_cast<ProjRecord*>(S + oRec);
  Footprint* foot = reinterpret_cast<Footprint*>(S + oFoot);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(S + oCnt);
  uint32_t* key_a = reinterpret_cast<uint32_t*>(S + oKeyA);
  uint32_t* val_a = reinterpret_cast<uint32_t*>(S + oValA);
  uint32_t* key_b = reinterpret_cast<uint32_t*>(S + oKeyB);
  uint32_t* val_b = reinterpret_cast<uint32_t*>(S + oValB);
  uint32_t* offs = reinterpret_cast<uint32_t*>(S + oOffs);
  uint32_t* ccnt = reinterpret_cast<uint32_t*>(S + oCcnt);
  uint32_t* dlo = reinterpret_cast<uint32_t*>(S + oDlo);
  uint32_t* lk_a = reinterpret_cast<uint32_t*>(S + oLkA);
  uint32_t* lv_a = reinterpret_cast<uint32_t*>(S + oLvA);
  uint32_t* lk_b = reinterpret_cast<uint32_t*>(S + oLkB);
  uint32_t* lv_b = reinterpret_cast<uint32_t*>(S + oLvB);
  uint2* ranges = reinterpret_cast<uint2*>(S + oRanges);
  float* state = reinterpret_cast<float*>(S + oState);
  uint64_t* sat = reinterpret_cast<uint64_t*>(S + oSat);
  uint64_t* subsat = reinterpret_cast<uint64_t*>(S + oSubsat);
  void* sort_tmp = S + oSortTmp;
  void* scan_tmp = S + oScanTmp;
  uint32_t* total_d = reinterpret_cast<uint32_t*>(S + oWords);
  unsigned int* err_d = reinterpret_cast<unsigned int*>(S + oWords + 4);
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(S + oCounters);

  // everything that must start at zero
  NA_CUDA(cudaMemsetAsync(S + oWords, 0, 256, strm), "clear");
  NA_CUDA(cudaMemsetAsync(ctr, 0, kNumCounters * 8, strm), "clear");
  NA_CUDA(cudaMemsetAsync(table, 0, static_cast<size_t>(n) * E * sizeof(float), strm), "clear");

  NA_CUDA(launch_scene_prep(n, static_cast<const float*>(g->mean), g->quat, FS_F32, g->scale,
                            FS_F32, g->opacity, FS_F32, pos, cov, err_d, strm),
          "scene");
  unsigned int h_err = 0;
  NA_CUDA(cudaMemcpyAsync(&h_err, err_d, 4, cudaMemcpyDeviceToHost, strm), "readback");
  NA_CUDA(cudaStreamSynchronize(strm), "readback");
  if (h_err)
    return na_fail(FS_INVALID_ARGUMENT,
                   "fs_solve_noalloc: a Gaussian has a zero quaternion or a non-finite attribute");

  for (int v = 0; v < n_views; ++v) {
    ViewParams vp;
    fill_view(cams[v], &vp);  // the same view set-up as fs_solve
    vp.tile_base = 0;
    vp.state_off = 0;
    vp.mask = masks[v];
    const int tiles = vp.tiles_x * vp.tiles_y;
    // pageable source: the copy has taken the bytes when the call returns
    NA_CUDA(cudaMemcpyAsync(vd, &vp, sizeof(vp), cudaMemcpyHostToDevice, strm), "view upload");
    NA_CUDA(launch_project(n, 1, vd, pos, cov, rec, nullptr, foot, cnt, key_a, val_a, dlo, nullptr,
                           strm),
            "project");
    bool alt = false;
    NA_CUDA(radix_sort_pairs(key_a, val_a, key_b, val_b, n, 32, sort_tmp, &alt, strm), "sort");
    uint32_t* skey = alt ? key_b : key_a;
    uint32_t* sval = alt ? val_b : val_a;
    NA_CUDA(launch_depth_tie_fix(n, n, skey, sval, dlo, strm), "ties");
    NA_CUDA(cudaMemsetAsync(sat, 0, static_cast<size_t>((tiles + 63) / 64) * 8, strm), "clear");
    NA_CUDA(cudaMemsetAsync(subsat, 0, static_cast<size_t>((4 * tiles + 63) / 64) * 8, strm),
            "clear");
    NA_CUDA(launch_state_init(vd, 1, tiles, E, mask_dtype, state, sat, subsat, ctr, strm), "state");
    const int chunks = 6;
    int64_t p0 = 0;
    for (int ci = 0; ci < chunks; ++ci) {
      const int64_t p1 = (ci == chunks - 1) ? n : (n >> (chunks - 1 - ci));
      const int64_t n_pos = p1 - p0;
      if (n_pos <= 0) continue;
      NA_CUDA(launch_chunk_count(p0, n_pos, n, vd, sval, foot, sat, ccnt, strm), "count");
      NA_CUDA(exclusive_scan(ccnt, nullptr, offs, n_pos, total_d, scan_tmp, strm), "scan");
      uint32_t I = 0;
      NA_CUDA(cudaMemcpyAsync(&I, total_d, 4, cudaMemcpyDeviceToHost, strm), "readback");
      NA_CUDA(cudaStreamSynchronize(strm), "readback");
      if (I > static_cast<uint32_t>(kNA_Entries))
        return na_fail(FS_UNSUPPORTED,
                       "fs_solve_noalloc: a view needs more than FS_NOALLOC_MAX_LIST_ENTRIES "
                       "(tile, Gaussian) pairs in one depth chunk; the table is incomplete");
      if (I > 0) {
        NA_CUDA(launch_emit(p0, n_pos, n, vd, sval, offs, ccnt, foot, sat, lk_a, lv_a, ctr,
                            strm),
                "emit");
        bool alt2 = false;
        NA_CUDA(radix_sort_pairs(lk_a, lv_a, lk_b, lv_b, I, bits_for(tiles), sort_tmp, &alt2, strm),
                "tile sort");
        const uint32_t* lkey = alt2 ? lk_b : lk_a;
        const uint32_t* lval = alt2 ? lv_b : lv_a;
        NA_CUDA(cudaMemsetAsync(ranges, 0, static_cast<size_t>(tiles) * 8, strm), "clear");
        NA_CUDA(launch_ranges(I, lkey, ranges, strm), "ranges");
        NA_CUDA(launch_blend(vd, 1, tiles, ranges, lval, rec, nullptr, n, E, mask_dtype, table,
                             FS_F32, state, sat, subsat, nullptr, 0, ctr, false, strm),
                "blend");
      }
      p0 = p1;
    }
  }
  if (member_bits || label || margin)
    NA_CUDA(launch_assign(table, FS_F32, n, E, gamma, member_bits, label, margin, strm), "assign");
  unsigned long long h_ctr[kNumCounters];
  NA_CUDA(cudaMemcpyAsync(h_ctr, ctr, sizeof(h_ctr), cudaMemcpyDeviceToHost, strm), "readback");
  NA_CUDA(cudaStreamSynchronize(strm), "readback");
  if (h_ctr[kBinningMismatch])
    return na_fail(FS_CUDA_ERROR, "fs_solve_noalloc: internal binning mismatch");
  return FS_OK;
}
