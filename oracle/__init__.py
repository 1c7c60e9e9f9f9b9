"""FlashSplat FP64 CPU oracle -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path:
the renderer/accumulator is plain C (``fs_oracle.c``), the assignment step is
numpy (``assign.py``).

Paper: FlashSplat (arXiv 2409.08270).  Sec. 3.1 Eq. 1 (alpha blending),
Sec. 3.2 Eq. 2-6 (binary ILP and its closed form), Sec. 3.2 "Regularized ILP"
(background bias), Sec. 3.3 Eq. 7 (multi-instance), Supp. Sec. 6 (contribution
table A in R^{E x N} and segmentation matrix S), Sec. 3.4 and Supp. Sec. 8.2
(novel-view mask rendering, ``render_masks``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

from .assign import assign, assign_margin  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libfs_oracle.so")
_lib = None

FLAG_ALPHA_EDGE = 1
FLAG_T_EDGE = 2
FLAG_DEPTH_TIE = 4
FLAG_DOWNSTREAM = 8
COVERAGE_EXACT = 0
COVERAGE_3SIGMA = 1


class Camera(ctypes.Structure):
    """Mirror of ``fso_camera``: world->camera R (row-major), t, intrinsics."""

    _fields_ = [
        ("R", ctypes.c_double * 9),
        ("t", ctypes.c_double * 3),
        ("fx", ctypes.c_double),
        ("fy", ctypes.c_double),
        ("cx", ctypes.c_double),
        ("cy", ctypes.c_double),
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("pad", ctypes.c_int32 * 2),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libfs_oracle.so`` (gcc, -O2,
    no floating-point contraction, so every step rounds as written on every
    host)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", "-o",
           tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    i64, i32, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
    lib.fso_accumulate.restype = ctypes.c_int
    lib.fso_accumulate.argtypes = [i64, vp, vp, vp, vp, i32, vp, vp, vp, i32, vp, i64, i32, i32,
                                   vp, vp, vp, vp, vp, ctypes.c_double, i32, ctypes.c_double,
                                   ctypes.c_double, i32, i32]
    lib.fso_pixel_lists.restype = ctypes.c_int64
    lib.fso_pixel_lists.argtypes = [i64, vp, vp, vp, vp, i32, vp, i32, i64, vp, vp, vp, vp]
    lib.fso_render_masks.restype = ctypes.c_int
    lib.fso_render_masks.argtypes = [i64, vp, vp, vp, vp, vp, i32, vp, i32, ctypes.c_double, i32,
                                     i32, vp, vp, vp, vp, vp]
    lib.fso_project_view.restype = ctypes.c_int
    lib.fso_project_view.argtypes = [i64, vp, vp, vp, vp, vp, vp]
    _lib = lib
    return lib


def _f32(a, shape_last=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if shape_last is not None and a.ndim != 2:
        a = a.reshape(-1, shape_last)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def make_cameras(cams) -> ctypes.Array:
    """cams: iterable of dicts with R (3x3), t (3), fx, fy, cx, cy, width, height."""
    cams = list(cams)
    arr = (Camera * max(len(cams), 1))()
    for k, c in enumerate(cams):
        R = np.asarray(c["R"], dtype=np.float64).reshape(9)
        t = np.asarray(c["t"], dtype=np.float64).reshape(3)
        arr[k].R[:] = list(R)
        arr[k].t[:] = list(t)
        arr[k].fx, arr[k].fy = float(c["fx"]), float(c["fy"])
        arr[k].cx, arr[k].cy = float(c["cx"]), float(c["cy"])
        arr[k].width, arr[k].height = int(c["width"]), int(c["height"])
    return arr


@dataclass
class Accumulation:
    table: np.ndarray   # [rows, E] float64
    risk: np.ndarray    # [rows, E] float64: bound on |change| if marginal decisions flip
    flags: np.ndarray   # [rows] uint8, FLAG_* bits
    t_final: np.ndarray | None
    n_eval: int         # evaluated (pixel, Gaussian) pairs
    n_hit: int          # contributing pairs (alpha*T > 0) on tracked rows
    n_bad_label: int    # pixels whose label is outside [0, E)
    n_unseen: int       # tracked Gaussians valid in no view
    n_part: int = 0     # pairs taking part: alpha >= 1/255 up to and including the stop (no sel)


def accumulate(gaussians, cams, masks, E: int, sel=None, cull_mode: int = 0,
               nthreads: int | None = None, want_t_final: bool = False,
               event_rel: float = 1e-5, record_f16: bool = False, alpha_min: float = 0.0,
               t_min: float = 0.0, tie_reverse: bool = False,
               coverage: int = 0) -> Accumulation:
    """Contribution table of Eq. 6 / Eq. 7 in FP64.

    gaussians: dict with mean [N,3], quat [N,4] (w,x,y,z), scale [N,3] (linear),
    opacity [N] (activated).  cams: list of camera dicts.  masks: list of V
    integer arrays [H, W].  sel: optional sorted Gaussian indices to track.
    event_rel: the relative precision assumed for alpha in the implementation
    compared with; it sets the windows inside which a decision counts as
    marginal in `risk`: alpha within event_rel of 1/255, and T(1 - alpha)
    within event_rel * (1 + sum alpha/(1 - alpha)) + 2^-23 per factor of 1e-4
    (1e-5 suits an FP32 implementation; an FP64-level one is compared with a
    far narrower window).
    alpha_min, t_min (0: 1/255 and 1e-4) and tie_reverse (equal depths by
    higher index first) move the rule's decisions, for tests of the bound.
    coverage: 0 = every pixel the alpha >= 1/255 ellipse reaches; 1 = only
    pixels in the 16x16 tiles of the 3-sigma square (the standard 3D-GS
    rasteriser's coverage, COVERAGE_3SIGMA).
    record_f16: alpha from the reduced-precision record of each (view,
    Gaussian) -- the whitening matrix rounded to FP16 and the mean to FP32 --
    evaluated in FP64 (the oracle of the reduced-precision form).
    """
    lib = _load()
    mean = _f32(gaussians["mean"], 3)
    quat = _f32(gaussians["quat"], 4)
    scale = _f32(gaussians["scale"], 3)
    opac = np.ascontiguousarray(np.asarray(gaussians["opacity"], dtype=np.float32).reshape(-1))
    N = mean.shape[0]
    cams = list(cams)
    V = len(cams)
    carr = make_cameras(cams)
    flat = [np.ascontiguousarray(np.asarray(m).reshape(-1).astype(np.int32)) for m in masks]
    offs = np.zeros(max(V, 1), dtype=np.int64)
    acc = 0
    for v in range(V):
        c = cams[v]
        if flat[v].size != int(c["width"]) * int(c["height"]):
            raise ValueError(f"mask {v} has {flat[v].size} pixels, camera wants "
                             f"{int(c['width'])}x{int(c['height'])}")
        offs[v] = acc
        acc += flat[v].size
    allm = np.concatenate(flat) if flat else np.zeros(1, np.int32)
    if sel is not None:
        sel = np.ascontiguousarray(np.asarray(sel, dtype=np.int64))
        if sel.size and np.any(np.diff(sel) <= 0):
            raise ValueError("sel must be strictly increasing")
        rows = sel.size
    else:
        rows = N
    table = np.zeros((rows, E), dtype=np.float64)
    risk = np.zeros((rows, E), dtype=np.float64)
    flags = np.zeros(max(rows, 1), dtype=np.uint8)
    tf = np.zeros(max(acc, 1), dtype=np.float64) if want_t_final else None
    stats = np.zeros(5, dtype=np.int64)
    if nthreads is None:
        nthreads = max(1, len(os.sched_getaffinity(0)))
    rc = lib.fso_accumulate(N, _ptr(mean), _ptr(quat), _ptr(scale), _ptr(opac), V, carr,
                            _ptr(allm), _ptr(offs), E, _ptr(sel),
                            0 if sel is None else sel.size, cull_mode, nthreads,
                            _ptr(table), _ptr(risk), _ptr(flags), _ptr(tf), _ptr(stats),
                            float(event_rel), 1 if record_f16 else 0, float(alpha_min),
                            float(t_min), 1 if tie_reverse else 0, int(coverage))
    if rc != 0:
        raise ValueError(f"fso_accumulate failed with code {rc}")
    return Accumulation(table, risk, flags[:rows], None if tf is None else tf[:acc],
                        int(stats[0]), int(stats[1]), int(stats[2]), int(stats[3]), int(stats[4]))


def pixel_lists(gaussians, cams, cull_mode: int = 0):
    """Per-pixel ordered (Gaussian, alpha*T) terms of Eq. 1, CSR over all pixels.

    Returns (offsets [P+1], gidx, contrib, t_final [P]); pixels are listed view
    by view, row-major.
    """
    lib = _load()
    mean = _f32(gaussians["mean"], 3)
    quat = _f32(gaussians["quat"], 4)
    scale = _f32(gaussians["scale"], 3)
    opac = np.ascontiguousarray(np.asarray(gaussians["opacity"], dtype=np.float32).reshape(-1))
    N = mean.shape[0]
    cams = list(cams)
    carr = make_cameras(cams)
    P = sum(int(c["width"]) * int(c["height"]) for c in cams)
    offs = np.zeros(P + 1, dtype=np.int64)
    tf = np.zeros(max(P, 1), dtype=np.float64)
    cap = 1 << 16
    while True:
        gidx = np.zeros(cap, dtype=np.int32)
        con = np.zeros(cap, dtype=np.float64)
        n = lib.fso_pixel_lists(N, _ptr(mean), _ptr(quat), _ptr(scale), _ptr(opac), len(cams),
                                carr, cull_mode, cap, _ptr(offs), _ptr(gidx), _ptr(con), _ptr(tf))
        if n < 0:
            raise ValueError("fso_pixel_lists failed")
        if n <= cap:
            return offs, gidx[:n], con[:n], tf[:P]
        cap = int(n)


def project_view(gaussians, cam):
    """Projected quantities of one view: [N, 10] = valid, depth, mx, my,
    conic a, b, c, opacity, bbox width, bbox height."""
    lib = _load()
    mean = _f32(gaussians["mean"], 3)
    quat = _f32(gaussians["quat"], 4)
    scale = _f32(gaussians["scale"], 3)
    opac = np.ascontiguousarray(np.asarray(gaussians["opacity"], dtype=np.float32).reshape(-1))
    N = mean.shape[0]
    out = np.zeros((max(N, 1), 10), dtype=np.float64)
    rc = lib.fso_project_view(N, _ptr(mean), _ptr(quat), _ptr(scale), _ptr(opac),
                              make_cameras([cam]), _ptr(out))
    if rc != 0:
        raise ValueError("fso_project_view failed (zero quaternion?)")
    return out[:N]


@dataclass
class MaskRender:
    label: list         # per view [H, W] int32: the mask value (0: no object passes)
    rho: list           # per view [E-1, H, W]: rho^e, the accumulated alpha of object e
    depth: list         # per view [E-1, H, W]: D^e = sum alpha T z / rho^e (0 where rho^e = 0)
    rho_risk: list      # per view [E-1, H, W]: bound on |change of rho^e| (marginal decisions)
    z_sum: list         # per view [E-1, H, W]: sum alpha T z
    z_risk: list        # per view [E-1, H, W]: bound on |change of sum alpha T z|


def render_masks(gaussians, cams, member_bits, E: int, tau: float = 0.1, coverage: int = 0,
                 nthreads: int | None = None) -> MaskRender:
    """Masks for (novel) views from a segmentation (Sec. 3.4; Supp. Sec. 8.2):
    object e = 1 .. E-1 (the Gaussians with bit e of member_bits set) is
    rendered alone; rho^e > tau passes, and among the objects that pass the
    smallest depth D^e wins (E = 2: the binary mask [rho^1 > tau]).  tau = 0.1
    is the paper's choice (Sec. 4.6).  FP64, the accumulation's rules."""
    lib = _load()
    mean = _f32(gaussians["mean"], 3)
    quat = _f32(gaussians["quat"], 4)
    scale = _f32(gaussians["scale"], 3)
    opac = np.ascontiguousarray(np.asarray(gaussians["opacity"], dtype=np.float32).reshape(-1))
    N = mean.shape[0]
    bits = np.ascontiguousarray(np.asarray(member_bits).astype(np.uint64).reshape(-1))
    if bits.size != N:
        raise ValueError("member_bits needs one word per Gaussian")
    if not 2 <= E <= 64:
        raise ValueError("E must be in [2, 64]")
    cams = list(cams)
    npix = [int(c["width"]) * int(c["height"]) for c in cams]
    total = sum(npix)
    K = E - 1
    label = np.zeros(max(total, 1), dtype=np.int32)
    planes = [np.zeros(max(total * K, 1), dtype=np.float64) for _ in range(4)]
    if nthreads is None:
        nthreads = max(1, len(os.sched_getaffinity(0)))
    rc = lib.fso_render_masks(N, _ptr(mean), _ptr(quat), _ptr(scale), _ptr(opac), _ptr(bits),
                              len(cams), make_cameras(cams), E, float(tau), int(coverage),
                              nthreads, _ptr(label), *[_ptr(a) for a in planes])
    if rc != 0:
        raise ValueError(f"fso_render_masks failed with code {rc}")
    out = MaskRender([], [], [], [], [], [])
    off = 0
    for c, n in zip(cams, npix):
        H, W = int(c["height"]), int(c["width"])
        out.label.append(label[off:off + n].reshape(H, W).copy())
        rho, z, rr, zr = (a[off * K:(off + n) * K].reshape(K, H, W).copy() for a in planes)
        out.rho.append(rho)
        out.z_sum.append(z)
        out.rho_risk.append(rr)
        out.z_risk.append(zr)
        with np.errstate(divide="ignore", invalid="ignore"):
            out.depth.append(np.where(rho > 0, z / np.where(rho > 0, rho, 1.0), 0.0))
        off += n
    return out
