"""Thin Python binding of libflashsplat (include/flashsplat.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  The ``fs_*`` functions mirror the C ABI one to one; ``Solver`` is a
convenience wrapper that takes numpy / torch inputs, keeps device buffers in
torch tensors and returns torch tensors.  PyTorch provides device memory and
streams only.

The library must have been built (``paper_2409_08270_gb300.build.build()``);
loading fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

FS_OK, FS_INVALID_ARGUMENT, FS_OUT_OF_MEMORY, FS_CUDA_ERROR, FS_TIMEOUT, FS_UNSUPPORTED, \
    FS_CANCELLED = range(7)
FS_F32, FS_F64, FS_BF16, FS_F16, FS_U8, FS_I32 = range(6)
FS_MEM_HOST, FS_MEM_DEVICE = 0, 1
FS_COVERAGE_EXACT, FS_COVERAGE_3SIGMA = 0, 1

STATUS_NAMES = {0: "FS_OK", 1: "FS_INVALID_ARGUMENT", 2: "FS_OUT_OF_MEMORY", 3: "FS_CUDA_ERROR",
                4: "FS_TIMEOUT", 5: "FS_UNSUPPORTED", 6: "FS_CANCELLED"}

# every entry point declared in include/flashsplat.h
EXPORTS = ["fs_version", "fs_last_error", "fs_create", "fs_destroy", "fs_scene_create",
           "fs_scene_destroy", "fs_scene_size", "fs_accumulate", "fs_assign", "fs_solve",
           "fs_synchronize", "fs_keep_after_removal", "fs_check_wait_timeout", "fs_render_masks",
           "fs_test_sort_pairs", "fs_test_exclusive_scan", "fs_test_tile_ranges",
           "fs_graph_create", "fs_graph_launch", "fs_graph_synchronize", "fs_graph_destroy",
           "fs_solve_noalloc", "fs_server_create", "fs_server_add_scene",
           "fs_server_submit", "fs_server_fetch", "fs_server_fetch_for", "fs_server_cancel",
           "fs_server_destroy"]


class fs_options(ctypes.Structure):
    _fields_ = [("views_per_batch", ctypes.c_int32), ("time_stages", ctypes.c_int32),
                ("depth_chunks", ctypes.c_int32), ("recheck_margin", ctypes.c_float),
                ("recheck_reproject", ctypes.c_int32), ("record_precision", ctypes.c_int32),
                ("census", ctypes.c_int32), ("coverage", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 8)]


class fs_gaussians(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("mean", ctypes.c_void_p), ("quat", ctypes.c_void_p),
                ("scale", ctypes.c_void_p), ("opacity", ctypes.c_void_p),
                ("quat_dtype", ctypes.c_int32), ("scale_dtype", ctypes.c_int32),
                ("opacity_dtype", ctypes.c_int32), ("memory", ctypes.c_int32)]


class fs_camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3), ("fx", ctypes.c_double),
                ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class fs_stats(ctypes.Structure):
    _fields_ = [("views", ctypes.c_int64), ("pixels", ctypes.c_int64),
                ("list_entries", ctypes.c_int64), ("bad_labels", ctypes.c_int64),
                ("pairs", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("blend_ms", ctypes.c_double), ("blend_launches", ctypes.c_int64),
                ("staged_entries", ctypes.c_int64), ("rechecked", ctypes.c_int64),
                ("recheck_pairs", ctypes.c_int64), ("recheck_rebinned", ctypes.c_int64),
                ("census_pairs", ctypes.c_int64), ("census_rounds", ctypes.c_int64),
                ("census_steps", ctypes.c_int64), ("census_rounds_mixed", ctypes.c_int64),
                ("stage_ms", ctypes.c_double * 8)]


# indices of fs_stats.stage_ms (FS_STAGE_*)
STAGES = ("project", "depth_sort", "pixel_state", "binning", "tile_sort", "blend", "recheck",
          "assign")


class fs_result(ctypes.Structure):
    _fields_ = [("memory", ctypes.c_int32), ("table_dtype", ctypes.c_int32),
                ("table", ctypes.c_void_p), ("member_bits", ctypes.c_void_p),
                ("label", ctypes.c_void_p), ("margin", ctypes.c_void_p)]


class fs_server_options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("slots", ctypes.c_int32),
                ("budget_bytes", ctypes.c_int64), ("autotune", ctypes.c_int32),
                ("graphs", ctypes.c_int32), ("reserved", ctypes.c_int32 * 8)]


class fs_server_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("done", ctypes.c_int32),
                ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("slot", ctypes.c_int32),
                ("views_per_batch", ctypes.c_int32), ("depth_chunks", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("bytes_estimate", ctypes.c_int64),
                ("stats", fs_stats)]


class FlashSplatError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libflashsplat.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libflashsplat.so not found at {path}: build it with "
                           "paper_2409_08270_gb300.build.build() (needs nvcc)")
    lib = ctypes.CDLL(path)
    vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    sig = {
        "fs_version": (i32, []),
        "fs_last_error": (ctypes.c_char_p, []),
        "fs_create": (i32, [ctypes.POINTER(vp), i32, ctypes.POINTER(fs_options)]),
        "fs_destroy": (i32, [vp]),
        "fs_scene_create": (i32, [vp, ctypes.POINTER(fs_gaussians), ctypes.POINTER(vp)]),
        "fs_scene_destroy": (i32, [vp]),
        "fs_scene_size": (i64, [vp]),
        "fs_accumulate": (i32, [vp, vp, ctypes.POINTER(fs_camera), i32, ctypes.POINTER(vp), i32,
                                i32, i32, vp, i32, vp]),
        "fs_assign": (i32, [vp, vp, i32, i64, i32, f32, vp, vp, vp, vp]),
        "fs_solve": (i32, [vp, vp, ctypes.POINTER(fs_camera), i32, ctypes.POINTER(vp), i32, i32,
                           i32, f32, ctypes.POINTER(fs_result), vp]),
        "fs_synchronize": (i32, [vp, vp, ctypes.POINTER(fs_stats)]),
        "fs_check_wait_timeout": (i32, [i32, i32]),
        "fs_test_sort_pairs": (i32, [i32, vp, vp, i64, i32]),
        "fs_test_exclusive_scan": (i32, [i32, vp, vp, i64, ctypes.POINTER(ctypes.c_uint32)]),
        "fs_test_tile_ranges": (i32, [i32, vp, i64, i32, vp]),
        "fs_keep_after_removal": (i32, [vp, vp, i64, ctypes.c_uint64, vp, ctypes.POINTER(i64), vp]),
        "fs_graph_create": (i32, [vp, vp, ctypes.POINTER(fs_camera), i32, ctypes.POINTER(vp), i32,
                                  i32, f32, ctypes.POINTER(fs_result), ctypes.POINTER(vp)]),
        "fs_graph_launch": (i32, [vp, vp]),
        "fs_graph_synchronize": (i32, [vp, vp, ctypes.POINTER(fs_stats)]),
        "fs_graph_destroy": (i32, [vp]),
        "fs_render_masks": (i32, [vp, vp, ctypes.POINTER(fs_camera), i32, vp, i32, f32,
                                  ctypes.POINTER(vp), i32, ctypes.POINTER(vp),
                                  ctypes.POINTER(vp), vp]),
        "fs_solve_noalloc": (i32, [i32, ctypes.POINTER(fs_gaussians), ctypes.POINTER(fs_camera),
                                   i32, ctypes.POINTER(vp), i32, i32, f32, vp, vp, vp, vp, vp]),
        "fs_server_create": (i32, [ctypes.POINTER(fs_server_options), ctypes.POINTER(vp)]),
        "fs_server_add_scene": (i32, [vp, ctypes.POINTER(fs_gaussians), ctypes.POINTER(i32)]),
        "fs_server_submit": (i32, [vp, i32, ctypes.POINTER(fs_camera), i32, ctypes.POINTER(vp),
                                   i32, i32, f32, ctypes.POINTER(i64)]),
        "fs_server_fetch": (i32, [vp, i64, i32, vp, vp, vp, ctypes.POINTER(fs_server_info)]),
        "fs_server_fetch_for": (i32, [vp, i64, i32, vp, vp, vp, ctypes.POINTER(fs_server_info)]),
        "fs_server_cancel": (i32, [vp, i64]),
        "fs_server_destroy": (i32, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int):
    if status != FS_OK:
        msg = load().fs_last_error().decode(errors="replace")
        raise FlashSplatError(status, msg)


# ---- one-to-one wrappers of the C ABI ------------------------------------

def fs_version() -> int:
    return load().fs_version()


def fs_last_error() -> str:
    return load().fs_last_error().decode(errors="replace")


def fs_create(device: int = 0, views_per_batch: int = 0, time_stages: bool = False,
              depth_chunks: int = 0, recheck_margin: float = 0.0,
              recheck_reproject: bool = False, record_precision: int = 0,
              census: bool = False, coverage: int = 0) -> int:
    ctx = ctypes.c_void_p()
    opt = fs_options()
    opt.views_per_batch = views_per_batch
    opt.time_stages = 1 if time_stages else 0
    opt.depth_chunks = depth_chunks
    opt.recheck_margin = recheck_margin
    opt.recheck_reproject = 1 if recheck_reproject else 0
    opt.record_precision = record_precision
    opt.census = 1 if census else 0
    opt.coverage = coverage
    check(load().fs_create(ctypes.byref(ctx), device, ctypes.byref(opt)))
    return ctx.value


def fs_destroy(ctx: int):
    check(load().fs_destroy(ctx))


def fs_scene_create(ctx: int, g: fs_gaussians) -> int:
    sc = ctypes.c_void_p()
    check(load().fs_scene_create(ctx, ctypes.byref(g), ctypes.byref(sc)))
    return sc.value


def fs_scene_destroy(scene: int):
    check(load().fs_scene_destroy(scene))


def fs_accumulate(ctx, scene, cams, masks, mask_dtype, mask_memory, E, table, table_dtype,
                  stream=0):
    V = len(masks)
    mp = (ctypes.c_void_p * max(V, 1))(*masks)
    check(load().fs_accumulate(ctx, scene, cams, V, mp, mask_dtype, mask_memory, E, table,
                               table_dtype, stream))


def fs_assign(ctx, table, table_dtype, n, E, gamma, bits=None, label=None, margin=None, stream=0):
    check(load().fs_assign(ctx, table, table_dtype, n, E, gamma, bits, label, margin, stream))


def fs_solve(ctx, scene, cams, masks, mask_dtype, mask_memory, E, gamma, result: fs_result,
             stream=0):
    V = len(masks)
    mp = (ctypes.c_void_p * max(V, 1))(*masks)
    check(load().fs_solve(ctx, scene, cams, V, mp, mask_dtype, mask_memory, E, gamma,
                          ctypes.byref(result), stream))


def fs_synchronize(ctx, stream=0) -> fs_stats:
    st = fs_stats()
    check(load().fs_synchronize(ctx, stream, ctypes.byref(st)))
    return st


def fs_check_wait_timeout(device: int, spins: int) -> int:
    """Status of the bounded-wait diagnostic (FS_TIMEOUT expected)."""
    return load().fs_check_wait_timeout(device, spins)


def fs_test_sort_pairs(device: int, keys, vals, bits: int) -> None:
    """Stable in-place sort of two uint32 device arrays by key, for keys
    below 2^bits (the library's radix sort, for isolated tests)."""
    check(load().fs_test_sort_pairs(device, keys.data_ptr(), vals.data_ptr(), keys.numel(),
                                    bits))


def fs_test_exclusive_scan(device: int, inp, out) -> int:
    """Exclusive prefix sum (mod 2^32) of a uint32 device array into `out`;
    returns the total."""
    tot = ctypes.c_uint32(0)
    check(load().fs_test_exclusive_scan(device, inp.data_ptr(), out.data_ptr(), inp.numel(),
                                        ctypes.byref(tot)))
    return int(tot.value)


def fs_test_tile_ranges(device: int, keys, n_tiles: int, ranges) -> None:
    """Per tile, the [first, last + 1) run of its key in a sorted uint32
    device array, into `ranges` (n_tiles x 2 uint32 on the device)."""
    check(load().fs_test_tile_ranges(device, keys.data_ptr(), keys.numel(), n_tiles,
                                     ranges.data_ptr()))


def fs_solve_noalloc(device, g: fs_gaussians, cams, masks, mask_dtype, E, gamma, table,
                     bits=None, label=None, margin=None, stream=0):
    """Allocation-free small-scene solve (see include/flashsplat.h)."""
    V = len(masks)
    mp = (ctypes.c_void_p * max(V, 1))(*masks)
    check(load().fs_solve_noalloc(device, ctypes.byref(g), cams, V, mp, mask_dtype, E, gamma,
                                  table, bits, label, margin, stream))


# ---- helpers ---------------------------------------------------------------

def make_cameras(cams) -> ctypes.Array:
    cams = list(cams)
    arr = (fs_camera * max(len(cams), 1))()
    for k, c in enumerate(cams):
        arr[k].R[:] = [float(x) for x in np.asarray(c["R"], dtype=np.float64).reshape(9)]
        arr[k].t[:] = [float(x) for x in np.asarray(c["t"], dtype=np.float64).reshape(3)]
        arr[k].fx, arr[k].fy = float(c["fx"]), float(c["fy"])
        arr[k].cx, arr[k].cy = float(c["cx"]), float(c["cy"])
        arr[k].width, arr[k].height = int(c["width"]), int(c["height"])
    return arr


def _torch():
    import torch
    return torch


class Solver:
    """A context on one GPU with one resident scene.

    gaussians: dict of arrays mean [N,3] f32, quat [N,4], scale [N,3], opacity [N]
    (numpy or torch; float32, or bfloat16 quat/scale and float16 opacity for
    the reduced-precision storage form).
    """

    _DT = {"float32": FS_F32, "bfloat16": FS_BF16, "float16": FS_F16}

    def __init__(self, gaussians, device: int = 0, views_per_batch: int = 0,
                 time_stages: bool = False, depth_chunks: int = 0, recheck_margin: float = 0.0,
                 recheck_reproject: bool = False, record_precision: int = 0,
                 census: bool = False, coverage: int = 0):
        torch = _torch()
        self.device = torch.device("cuda", device)
        self.ctx = fs_create(device, views_per_batch, time_stages, depth_chunks, recheck_margin,
                             recheck_reproject, record_precision, census, coverage)
        self.scene = None
        dev = {}
        for k in ("mean", "quat", "scale", "opacity"):
            a = gaussians[k]
            if not torch.is_tensor(a):
                a = torch.from_numpy(np.ascontiguousarray(a))
            dev[k] = a.to(self.device).contiguous()
        self.n = int(dev["mean"].shape[0])
        g = fs_gaussians()
        g.n = self.n
        g.mean, g.quat = dev["mean"].data_ptr(), dev["quat"].data_ptr()
        g.scale, g.opacity = dev["scale"].data_ptr(), dev["opacity"].data_ptr()
        g.quat_dtype = self._DT[str(dev["quat"].dtype).replace("torch.", "")]
        g.scale_dtype = self._DT[str(dev["scale"].dtype).replace("torch.", "")]
        g.opacity_dtype = self._DT[str(dev["opacity"].dtype).replace("torch.", "")]
        g.memory = FS_MEM_DEVICE
        self.scene = fs_scene_create(self.ctx, g)
        torch.cuda.synchronize(self.device)

    def close(self):
        if self.scene:
            fs_scene_destroy(self.scene)
            self.scene = None
        if self.ctx:
            fs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _stream(stream):
        torch = _torch()
        s = stream if stream is not None else torch.cuda.current_stream()
        return s.cuda_stream

    def upload_masks(self, masks):
        """Device copies of the masks (uint8 or int32), one tensor per view."""
        torch = _torch()
        out = []
        for m in masks:
            t = m if torch.is_tensor(m) else torch.from_numpy(np.ascontiguousarray(m))
            out.append(t.to(self.device).contiguous())
        return out

    @staticmethod
    def _mask_dtype(t):
        s = str(t.dtype)
        if "uint8" in s:
            return FS_U8
        if "int32" in s:
            return FS_I32
        raise ValueError(f"mask dtype {t.dtype} (want uint8 or int32)")

    def accumulate(self, cams, masks, E, table, stream=None):
        """table (torch, device, [N, E] float32/float64) += contributions."""
        torch = _torch()
        dm = self.upload_masks(masks)
        tdt = FS_F64 if table.dtype == torch.float64 else FS_F32
        fs_accumulate(self.ctx, self.scene, make_cameras(cams), [m.data_ptr() for m in dm],
                      self._mask_dtype(dm[0]), FS_MEM_DEVICE, E, table.data_ptr(), tdt,
                      self._stream(stream))
        return dm

    def assign(self, table, gamma, stream=None):
        torch = _torch()
        n, E = table.shape
        bits = torch.empty(n, dtype=torch.int64, device=self.device) if E <= 64 else None
        label = torch.empty(n, dtype=torch.int32, device=self.device)
        margin = torch.empty(n, dtype=torch.float32, device=self.device)
        tdt = FS_F64 if table.dtype == torch.float64 else FS_F32
        fs_assign(self.ctx, table.data_ptr(), tdt, n, E, float(gamma),
                  bits.data_ptr() if bits is not None else None, label.data_ptr(),
                  margin.data_ptr(), self._stream(stream))
        return bits, label, margin

    def keep_after_removal(self, bits, remove_labels, stream=None):
        """Indices (int32, device) of the Gaussians outside every removed
        object's subset; bits: device int64 [n] membership bits."""
        torch = _torch()
        n = int(bits.shape[0])
        keep = torch.empty(max(n, 1), dtype=torch.int32, device=self.device)
        mask = 0
        for e in remove_labels:
            mask |= 1 << int(e)
        n_keep = ctypes.c_int64(0)
        check(load().fs_keep_after_removal(self.ctx, bits.data_ptr(), n, ctypes.c_uint64(mask),
                                           keep.data_ptr(), ctypes.byref(n_keep),
                                           self._stream(stream)))
        return keep[:n_keep.value]

    def render_masks(self, cams, bits, E, tau=0.1, out_dtype="uint8", want_planes=False,
                     stream=None):
        """Masks for the views `cams` from membership bits (device int64 [n],
        e.g. solve()["bits"]): object e = 1 .. E-1 rendered alone, rho^e > tau,
        the nearest passing object wins (fs_render_masks).  Returns the per-view
        masks (device tensors [H, W]) and, with want_planes, per view rho and
        depth [E-1, H, W]."""
        torch = _torch()
        dt = torch.uint8 if out_dtype == "uint8" else torch.int32
        masks, rhos, depths = [], [], []
        for c in cams:
            H, W = int(c["height"]), int(c["width"])
            masks.append(torch.empty((H, W), dtype=dt, device=self.device))
            if want_planes:
                rhos.append(torch.empty((E - 1, H, W), dtype=torch.float32, device=self.device))
                depths.append(torch.empty((E - 1, H, W), dtype=torch.float32, device=self.device))
        V = len(cams)
        mp = (ctypes.c_void_p * max(V, 1))(*[m.data_ptr() for m in masks])
        rp = (ctypes.c_void_p * max(V, 1))(*[r.data_ptr() for r in rhos]) if want_planes else None
        dp = (ctypes.c_void_p * max(V, 1))(*[d.data_ptr() for d in depths]) if want_planes else None
        check(load().fs_render_masks(self.ctx, self.scene, make_cameras(cams), V, bits.data_ptr(),
                                     E, float(tau), mp, FS_U8 if dt == torch.uint8 else FS_I32,
                                     rp, dp, self._stream(stream)))
        torch.cuda.synchronize(self.device)
        out = {"masks": masks}
        if want_planes:
            out["rho"], out["depth"] = rhos, depths
        return out

    def capture(self, cams, masks, E, gamma, table_dtype="float32"):
        """A captured solve (fs_graph_create) over device masks: returns a
        CapturedSolve whose launch() replays it into fixed output tensors."""
        return CapturedSolve(self, cams, masks, E, gamma, table_dtype)

    def solve(self, cams, masks, E, gamma, table_dtype="float32", stream=None, sync=True):
        """Whole path on device-resident masks: returns dict of device tensors."""
        torch = _torch()
        dm = masks if (masks and torch.is_tensor(masks[0]) and masks[0].is_cuda) \
            else self.upload_masks(masks)
        tdt = FS_F64 if table_dtype == "float64" else FS_F32
        table = torch.empty((self.n, E), dtype=torch.float64 if tdt == FS_F64 else torch.float32,
                            device=self.device)
        bits = torch.empty(self.n, dtype=torch.int64, device=self.device) if E <= 64 else None
        label = torch.empty(self.n, dtype=torch.int32, device=self.device)
        margin = torch.empty(self.n, dtype=torch.float32, device=self.device)
        res = fs_result()
        res.memory, res.table_dtype = FS_MEM_DEVICE, tdt
        res.table = table.data_ptr()
        res.member_bits = bits.data_ptr() if bits is not None else None
        res.label, res.margin = label.data_ptr(), margin.data_ptr()
        st = self._stream(stream)
        fs_solve(self.ctx, self.scene, make_cameras(cams), [m.data_ptr() for m in dm],
                 self._mask_dtype(dm[0]), FS_MEM_DEVICE, E, float(gamma), res, st)
        out = {"table": table, "bits": bits, "label": label, "margin": margin}
        if sync:
            out["stats"] = fs_synchronize(self.ctx, st)
        return out


# ---- request server ---------------------------------------------------------

def fs_server_create(device: int = 0, slots: int = 4, budget_bytes: int = 0,
                     autotune: bool = False, graphs: int = 0) -> int:
    opt = fs_server_options()
    opt.device, opt.slots, opt.budget_bytes = device, slots, budget_bytes
    opt.autotune = 1 if autotune else 0
    opt.graphs = int(graphs)
    out = ctypes.c_void_p()
    check(load().fs_server_create(ctypes.byref(opt), ctypes.byref(out)))
    return out.value


def fs_server_add_scene(srv: int, g: fs_gaussians) -> int:
    sid = ctypes.c_int32()
    check(load().fs_server_add_scene(srv, ctypes.byref(g), ctypes.byref(sid)))
    return sid.value


def fs_server_submit(srv: int, scene_id: int, cams, mask_ptrs, mask_dtype: int, E: int,
                     gamma: float) -> int:
    arr = (ctypes.c_void_p * max(len(mask_ptrs), 1))(*mask_ptrs)
    ticket = ctypes.c_int64()
    check(load().fs_server_submit(srv, scene_id, cams, len(mask_ptrs), arr, mask_dtype, E,
                                  ctypes.c_float(gamma), ctypes.byref(ticket)))
    return ticket.value


def fs_server_fetch(srv: int, ticket: int, wait: bool, bits_ptr, label_ptr, margin_ptr,
                    timeout_ms: int | None = None):
    info = fs_server_info()
    if timeout_ms is None:
        st = load().fs_server_fetch(srv, ticket, 1 if wait else 0, bits_ptr, label_ptr,
                                    margin_ptr, ctypes.byref(info))
    else:
        st = load().fs_server_fetch_for(srv, ticket, int(timeout_ms), bits_ptr, label_ptr,
                                        margin_ptr, ctypes.byref(info))
    return st, info


def fs_server_cancel(srv: int, ticket: int):
    check(load().fs_server_cancel(srv, ticket))


def fs_server_destroy(srv: int):
    check(load().fs_server_destroy(srv))


class Server:
    """Request server over resident scenes (continuous batching; see
    fs_server_create in flashsplat.h).  Scenes and masks are numpy arrays in
    host memory; results come back as numpy arrays."""

    def __init__(self, device: int = 0, slots: int = 4, budget_bytes: int = 0,
                 autotune: bool = False, graphs: int = 0):
        self.srv = fs_server_create(device, slots, budget_bytes, autotune, graphs)
        self.sizes = []
        self._keep = {}

    def add_scene(self, gaussians) -> int:
        arrs = {k: np.ascontiguousarray(np.asarray(gaussians[k], dtype=np.float32))
                for k in ("mean", "quat", "scale", "opacity")}
        g = fs_gaussians()
        g.n = int(arrs["mean"].shape[0])
        g.mean, g.quat = arrs["mean"].ctypes.data, arrs["quat"].ctypes.data
        g.scale, g.opacity = arrs["scale"].ctypes.data, arrs["opacity"].ctypes.data
        g.quat_dtype = g.scale_dtype = g.opacity_dtype = FS_F32
        g.memory = FS_MEM_HOST
        sid = fs_server_add_scene(self.srv, g)
        self.sizes.append(g.n)
        return sid

    def submit(self, scene_id: int, cams, masks, E: int, gamma: float) -> int:
        ms = [np.ascontiguousarray(m) for m in masks]
        dt = FS_I32 if ms[0].dtype == np.int32 else FS_U8
        ms = [m.astype(np.int32 if dt == FS_I32 else np.uint8, copy=False) for m in ms]
        t = fs_server_submit(self.srv, scene_id, make_cameras(cams), [m.ctypes.data for m in ms],
                             dt, E, gamma)
        self._keep[t] = (scene_id, E)
        return t

    def fetch(self, ticket: int, wait: bool = True, timeout_ms: int | None = None):
        """Results of a request; None while it runs when wait is False or the
        bounded wait of timeout_ms milliseconds runs out (FS_TIMEOUT)."""
        sid, E = self._keep[ticket]
        n = self.sizes[sid]
        bits = np.empty(n, np.uint64) if E <= 64 else None
        label = np.empty(n, np.int32)
        margin = np.empty(n, np.float32)
        st, info = fs_server_fetch(self.srv, ticket, wait,
                                   bits.ctypes.data if bits is not None else None,
                                   label.ctypes.data, margin.ctypes.data, timeout_ms)
        if st == FS_TIMEOUT and (not wait or timeout_ms is not None):
            return None
        del self._keep[ticket]
        if st != FS_OK:
            raise FlashSplatError(st, load().fs_last_error().decode(errors="replace"))
        return {"bits": bits, "label": label, "margin": margin, "info": info}

    def cancel(self, ticket: int):
        fs_server_cancel(self.srv, ticket)

    def close(self):
        if self.srv:
            fs_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CapturedSolve:
    """One solve captured into a CUDA graph (fs_graph_*): `masks` are device
    tensors read at every replay (write new labels into them in place);
    `outputs` holds the table, bits, label and margin tensors every replay
    writes."""

    def __init__(self, solver, cams, masks, E, gamma, table_dtype="float32"):
        torch = _torch()
        self.solver = solver
        self.masks = masks if (masks and torch.is_tensor(masks[0]) and masks[0].is_cuda) \
            else solver.upload_masks(masks)
        dev, n = solver.device, solver.n
        f64 = table_dtype == "float64"
        self.outputs = {
            "table": torch.empty((n, E), dtype=torch.float64 if f64 else torch.float32, device=dev),
            "bits": torch.empty(n, dtype=torch.int64, device=dev) if E <= 64 else None,
            "label": torch.empty(n, dtype=torch.int32, device=dev),
            "margin": torch.empty(n, dtype=torch.float32, device=dev)}
        res = fs_result()
        res.memory, res.table_dtype = FS_MEM_DEVICE, FS_F64 if f64 else FS_F32
        res.table = self.outputs["table"].data_ptr()
        res.member_bits = self.outputs["bits"].data_ptr() if self.outputs["bits"] is not None else None
        res.label = self.outputs["label"].data_ptr()
        res.margin = self.outputs["margin"].data_ptr()
        self._cams = make_cameras(cams)
        V = len(cams)
        mp = (ctypes.c_void_p * max(V, 1))(*[m.data_ptr() for m in self.masks])
        g = ctypes.c_void_p()
        check(load().fs_graph_create(solver.ctx, solver.scene, self._cams, V, mp,
                                     solver._mask_dtype(self.masks[0]), E, float(gamma),
                                     ctypes.byref(res), ctypes.byref(g)))
        self.graph = g.value

    def launch(self, stream=None):
        check(load().fs_graph_launch(self.graph, self.solver._stream(stream)))

    def synchronize(self, stream=None):
        st = fs_stats()
        check(load().fs_graph_synchronize(self.graph, self.solver._stream(stream), ctypes.byref(st)))
        return st

    def close(self):
        if self.graph:
            load().fs_graph_destroy(self.graph)
            self.graph = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
