"""Seeded synthetic workloads shaped like the paper's scenes.

The paper evaluates on reconstructed 3D-GS scenes of MIP-360, T&T, LLFF,
Instruct-NeRF2NeRF and LERF with SAM masks (Sec. 4.1).  None of that data is
used here; these generators stand in for it with the same structure:

* a scene of N Gaussians {m, q, s, o} (Sec. 3.1; colour is not needed),
* V pinhole cameras (forward-facing arc or 360-degree orbit),
* one label mask per view: the silhouette of the ground-truth object(s),
  found by casting the pixel-centre ray against each object's bounding
  ellipsoid (nearest hit wins), then corrupted with the kind of noise SAM
  masks show (random flips, eroded/dilated borders, id swaps at boundaries).

This module is the only code the CUDA path and the FP64 oracle share.  It
holds none of the method's arithmetic (no EWA projection, no alpha
compositing, no accumulation): masks are pure ray/ellipsoid geometry.

All randomness comes from numpy's PCG64 with the seeds below, so the same
call gives bit-identical inputs on every machine.
"""
from __future__ import annotations

import math
import zlib
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 240908270


@dataclass
class Workload:
    name: str
    gaussians: dict            # mean [N,3], quat [N,4] (w,x,y,z), scale [N,3], opacity [N]; float32
    cams: list                 # dicts: R (3x3, world->camera), t (3), fx, fy, cx, cy, width, height
    masks: list                # V arrays [H, W] (uint8 or int32 labels)
    E: int                     # number of labels, background 0 included
    gamma: float               # background bias
    gt: np.ndarray             # ground-truth object id per Gaussian (0 = background)
    info: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.gaussians["mean"].shape[0])

    @property
    def pixels(self) -> int:
        return int(sum(int(c["width"]) * int(c["height"]) for c in self.cams))


# ---------------------------------------------------------------------------
# building blocks
# ---------------------------------------------------------------------------

def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _quat_to_rot(q):
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def look_at(position, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)):
    """World->camera (R, t) for a camera at `position` looking at `target`.

    Camera axes: x right, y down, z forward (OpenCV).  R is a proper rotation.
    """
    pos = np.asarray(position, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - pos
    f /= np.linalg.norm(f)
    r = np.cross(np.asarray(up, dtype=np.float64), f)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ pos
    return R, t


def camera(position, width, height, fx, fy=None, cx=None, cy=None, target=(0, 0, 0)):
    R, t = look_at(position, target)
    return {"R": R, "t": t, "fx": float(fx), "fy": float(fx if fy is None else fy),
            "cx": float(width / 2 if cx is None else cx),
            "cy": float(height / 2 if cy is None else cy),
            "width": int(width), "height": int(height)}


def fx_from_hfov(width, hfov_deg):
    return (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)


def _pixel_rays(cam, y0=0, y1=None, x0=0, x1=None):
    """World-space ray directions (not normalised) through the pixel centres of
    rows [y0, y1) and columns [x0, x1), shape [h, w, 3]."""
    W, H = cam["width"], cam["height"]
    y1 = H if y1 is None else y1
    x1 = W if x1 is None else x1
    u = (np.arange(x0, x1) + 0.5 - cam["cx"]) / cam["fx"]
    v = (np.arange(y0, y1) + 0.5 - cam["cy"]) / cam["fy"]
    dc = np.empty((y1 - y0, x1 - x0, 3))
    dc[..., 0] = u[None, :]
    dc[..., 1] = v[:, None]
    dc[..., 2] = 1.0
    R = np.asarray(cam["R"])
    return dc @ R            # row-vector form of R^T d


def _camera_origin(cam):
    R = np.asarray(cam["R"])
    return -R.T @ np.asarray(cam["t"])


def _sphere_box(cam, centre, radius):
    """Pixel rectangle [y0, y1) x [x0, x1) that holds the image of a ball
    (the ball lies inside a camera-aligned cube whose corners bound x/z, y/z)."""
    W, H = cam["width"], cam["height"]
    p = np.asarray(cam["R"]) @ np.asarray(centre) + np.asarray(cam["t"])
    if p[2] - radius <= 1e-3:
        return 0, H, 0, W
    zs = (p[2] - radius, p[2] + radius)
    xs = [cam["fx"] * (p[0] + sx * radius) / z + cam["cx"] for sx in (-1, 1) for z in zs]
    ys = [cam["fy"] * (p[1] + sy * radius) / z + cam["cy"] for sy in (-1, 1) for z in zs]
    x0, x1 = int(max(0, math.floor(min(xs)) - 1)), int(min(W, math.ceil(max(xs)) + 1))
    y0, y1 = int(max(0, math.floor(min(ys)) - 1)), int(min(H, math.ceil(max(ys)) + 1))
    if x0 >= x1 or y0 >= y1:
        return 0, 0, 0, 0
    return y0, y1, x0, x1


def ellipsoid_hits(cam, centre, axes_rot, radii, box=None):
    """Ray entry distance into the ellipsoid {c + Rot diag(radii) u : |u| <= 1}
    for the pixels of `box` = (y0, y1, x0, x1) (default: the whole image):
    +inf where the ray misses, 0 when the camera is inside."""
    y0, y1, x0, x1 = box if box is not None else (0, cam["height"], 0, cam["width"])
    rays = _pixel_rays(cam, y0, y1, x0, x1)
    o = _camera_origin(cam) - np.asarray(centre)
    inv = np.asarray(axes_rot).T / np.asarray(radii)[:, None]     # D^-1 Rot^T
    o2 = inv @ o
    d2 = rays @ inv.T
    a = np.einsum("hwk,hwk->hw", d2, d2)
    b = 2.0 * (d2 @ o2)
    c = float(o2 @ o2) - 1.0
    disc = b * b - 4.0 * a * c
    hit = disc >= 0.0
    sq = np.sqrt(np.where(hit, disc, 0.0))
    s0 = (-b - sq) / (2.0 * a)
    s1 = (-b + sq) / (2.0 * a)
    s = np.where(s0 > 0.0, s0, np.where(s1 > 0.0, 0.0, np.inf))
    return np.where(hit, s, np.inf)


def label_map(cam, objects):
    """Nearest-hit object id per pixel; objects = [(id, centre, Rot, radii)]."""
    H, W = cam["height"], cam["width"]
    best = np.full((H, W), np.inf)
    lab = np.zeros((H, W), dtype=np.int32)
    for oid, c, rot, rad in objects:
        y0, y1, x0, x1 = _sphere_box(cam, c, float(np.max(rad)))
        if y0 >= y1:
            continue
        s = ellipsoid_hits(cam, c, rot, rad, (y0, y1, x0, x1))
        sub_b = best[y0:y1, x0:x1]
        closer = s < sub_b
        best[y0:y1, x0:x1] = np.where(closer, s, sub_b)
        lab[y0:y1, x0:x1] = np.where(closer, oid, lab[y0:y1, x0:x1])
    return lab


def _shift(a, dy, dx, fill):
    out = np.full_like(a, fill)
    H, W = a.shape
    ys, yd = (slice(0, H - dy), slice(dy, H)) if dy >= 0 else (slice(-dy, H), slice(0, H + dy))
    xs, xd = (slice(0, W - dx), slice(dx, W)) if dx >= 0 else (slice(-dx, W), slice(0, W + dx))
    out[yd, xd] = a[ys, xs]
    return out


def morph(mask, radius, dilate):
    """Binary dilation (max) or erosion (min) with a (2r+1)^2 square."""
    if radius <= 0:
        return mask.copy()
    m = mask.astype(bool)
    out = m.copy()
    for dy in range(-radius, radius + 1):
        for dx in range(-radius, radius + 1):
            s = _shift(m, dy, dx, fill=not dilate)
            out = (out | s) if dilate else (out & s)
    return out


def boundary_swaps(lab, frac, rng):
    """Give `frac` of the boundary pixels a random differing 4-neighbour's id."""
    H, W = lab.shape
    nbrs = [_shift(lab, dy, dx, fill=-1) for dy, dx in ((1, 0), (-1, 0), (0, 1), (0, -1))]
    diff = np.stack([(n != lab) & (n >= 0) for n in nbrs])          # [4, H, W]
    bnd = diff.any(axis=0)
    ys, xs = np.nonzero(bnd)
    pick = rng.random(ys.size) < frac
    ys, xs = ys[pick], xs[pick]
    out = lab.copy()
    for k in range(ys.size):
        y, x = ys[k], xs[k]
        choices = [j for j in range(4) if diff[j, y, x]]
        j = choices[rng.integers(len(choices))]
        out[y, x] = nbrs[j][y, x]
    return out


def _clustered_scene(rng, n, n_clusters, centre_lo, centre_hi, std_lo, std_hi,
                     logscale_mu, logscale_sd, opac_sd):
    centres = rng.uniform(centre_lo, centre_hi, size=(n_clusters, 3))
    rots = [_quat_to_rot(q) for q in _unit_quats(rng, n_clusters)]
    stds = rng.uniform(std_lo, std_hi, size=(n_clusters, 3))
    w = rng.uniform(0.5, 1.5, size=n_clusters)
    counts = rng.multinomial(n, w / w.sum())
    means = np.empty((n, 3))
    gt = np.empty(n, dtype=np.int32)
    k0 = 0
    for k in range(n_clusters):
        c = counts[k]
        z = rng.standard_normal((c, 3)) * stds[k]
        means[k0:k0 + c] = centres[k] + z @ rots[k].T
        gt[k0:k0 + c] = k
        k0 += c
    g = {
        "mean": means.astype(np.float32),
        "quat": _unit_quats(rng, n).astype(np.float32),
        "scale": np.exp(rng.normal(logscale_mu, logscale_sd, size=(n, 3))).astype(np.float32),
        "opacity": _sigmoid(rng.normal(0.0, opac_sd, size=n)).astype(np.float32),
    }
    objects = [(k, centres[k], rots[k], 2.0 * stds[k]) for k in range(n_clusters)]
    return g, gt, objects


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------

def tiny_scene(seed=SEED_BASE + 1, n=2000, views=8, width=128, height=128, fx=150.0,
               flip=0.02, gamma=0.5):
    """Plain FP32 tiny scene: N Gaussians uniform in [-1,1]^3, log-scales
    N(-3, 0.5), random unit quaternions, opacity sigmoid(N(0,1)); views on a
    horizontal ring of radius 3; binary masks = silhouette of the ball of
    radius 0.4 that holds the ground-truth foreground, with `flip` i.i.d. flips."""
    rng = np.random.default_rng(seed)
    mean = rng.uniform(-1.0, 1.0, size=(n, 3))
    g = {
        "mean": mean.astype(np.float32),
        "quat": _unit_quats(rng, n).astype(np.float32),
        "scale": np.exp(rng.normal(-3.0, 0.5, size=(n, 3))).astype(np.float32),
        "opacity": _sigmoid(rng.normal(0.0, 1.0, size=n)).astype(np.float32),
    }
    gt = (np.linalg.norm(mean, axis=1) < 0.4).astype(np.int32)
    cams, masks = [], []
    ball = [(1, np.zeros(3), np.eye(3), np.full(3, 0.4))]
    for v in range(views):
        az = 2.0 * math.pi * v / views
        cam = camera((3.0 * math.sin(az), 0.0, -3.0 * math.cos(az)), width, height, fx)
        lab = label_map(cam, ball)
        flips = rng.random(lab.shape) < flip
        masks.append(np.where(flips, 1 - lab, lab).astype(np.uint8))
        cams.append(cam)
    return Workload("tiny", g, cams, masks, 2, gamma, gt,
                    {"P": sum(m.size for m in masks)})


def binary_scene(seed=SEED_BASE + 2, n=1_000_000, views=100, width=1008, height=756,
                 hfov=60.0, n_clusters=20, flip=0.045, max_morph=3, gamma=0.5):
    """Binary segmentation at real-scene scale (LLFF-like forward-facing):
    N Gaussians from `n_clusters` anisotropic clusters (centres in
    [-1,1]^2 x [-0.5,0.5], per-axis std U[0.05,0.3]), log-scales N(-4,1),
    opacity sigmoid(N(0,1.5)); views on an arc of radius 4, azimuth
    U[-30,30] deg; mask = visible silhouette of the cluster nearest the
    origin, eroded or dilated by 0..max_morph px, plus `flip` i.i.d. flips."""
    rng = np.random.default_rng(seed)
    g, cl, objects = _clustered_scene(rng, n, n_clusters, [-1, -1, -0.5], [1, 1, 0.5],
                                      0.05, 0.3, -4.0, 1.0, 1.5)
    target = int(np.argmin([np.linalg.norm(o[1]) for o in objects]))
    gt = (cl == target).astype(np.int32)
    fx = fx_from_hfov(width, hfov)
    cams, masks = [], []
    changed = 0
    for v in range(views):
        az = math.radians(rng.uniform(-30.0, 30.0))
        cam = camera((4.0 * math.sin(az), 0.0, -4.0 * math.cos(az)), width, height, fx)
        lab = label_map(cam, [(k + 1, c, r, s) for k, c, r, s in objects])
        clean = lab == target + 1
        r = int(rng.integers(0, max_morph + 1))
        m = morph(clean, r, dilate=bool(rng.random() < 0.5))
        flips = rng.random(m.shape) < flip
        m = np.where(flips, ~m, m)
        changed += int(np.count_nonzero(m != clean))
        masks.append(m.astype(np.uint8))
        cams.append(cam)
    P = sum(x.size for x in masks)
    return Workload("binary", g, cams, masks, 2, gamma, gt,
                    {"P": P, "noise_fraction": changed / max(P, 1), "target_cluster": target})


def multi_scene(seed=SEED_BASE + 3, n=3_000_000, views=200, width=1256, height=828,
                hfov=60.0, n_clusters=32, swap=0.03, gamma=0.5, elevations=(15.0, 40.0)):
    """Multi-instance (MIP-360-like 360-degree orbit): N Gaussians in
    `n_clusters` clusters (centres in [-1.5,1.5]^3), cluster k -> label k+1;
    views split over two elevations, azimuth step 360/(views/2) deg, radius 5;
    int32 id masks = nearest visible cluster silhouette (0 = background), with
    `swap` of the boundary pixels taking a differing 4-neighbour's id."""
    rng = np.random.default_rng(seed)
    g, cl, objects = _clustered_scene(rng, n, n_clusters, [-1.5] * 3, [1.5] * 3,
                                      0.05, 0.3, -4.0, 1.0, 1.5)
    gt = (cl + 1).astype(np.int32)
    fx = fx_from_hfov(width, hfov)
    cams, masks = [], []
    per_ring = max(1, views // len(elevations))
    for v in range(views):
        ring = min(v // per_ring, len(elevations) - 1)
        el = math.radians(elevations[ring])
        az = math.radians((v % per_ring) * 360.0 / per_ring)
        pos = (5.0 * math.cos(el) * math.sin(az), 5.0 * math.sin(el), -5.0 * math.cos(el) * math.cos(az))
        cam = camera(pos, width, height, fx)
        lab = label_map(cam, [(k + 1, c, r, s) for k, c, r, s in objects])
        masks.append(boundary_swaps(lab, swap, rng).astype(np.int32))
        cams.append(cam)
    return Workload("multi", g, cams, masks, n_clusters + 1, gamma, gt,
                    {"P": sum(m.size for m in masks)})


def round_bf16(x):
    """Round float32 values to bfloat16 (round-to-nearest-even), kept as float32."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).reshape(a.shape)


def round_fp16(x):
    """Round float32 values to IEEE half (round-to-nearest-even), kept as float32."""
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float32)


def rounded_gaussians(g):
    """The reduced-precision storage of a scene's attributes: positions stay
    FP32, quaternions and scales are rounded to bfloat16 and opacities to
    FP16 (values kept as float32, so any consumer sees the rounded values)."""
    return {"mean": np.asarray(g["mean"], np.float32),
            "quat": round_bf16(g["quat"]), "scale": round_bf16(g["scale"]),
            "opacity": round_fp16(g["opacity"])}


SERVE_RESOLUTIONS = ((512, 512), (800, 600), (1008, 756), (1256, 828), (1600, 1200))


def serving_scenes(seed=SEED_BASE + 5, count=16, n_lo=200_000, n_hi=2_000_000, v_lo=20,
                   v_hi=150, labels_hi=16, scale=1.0):
    """Scenes of uneven size for the request server: N log-uniform in
    [n_lo, n_hi], V uniform in {v_lo..v_hi}, a resolution from
    SERVE_RESOLUTIONS, 1..labels_hi object labels (clusters grouped into
    labels), a 360-degree orbit at two elevations like multi_scene, uint8
    clean label masks (E = labels + 1).  `scale` shrinks N, V and the
    resolution together (for quick tests).  Returns a list of Workloads."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))) * scale)
        v = max(2, int(rng.integers(v_lo, v_hi + 1) * scale))
        wd, ht = SERVE_RESOLUTIONS[int(rng.integers(0, len(SERVE_RESOLUTIONS)))]
        wd, ht = max(16, int(wd * scale)), max(16, int(ht * scale))
        labels = int(rng.integers(1, labels_hi + 1))
        n_clusters = max(labels, int(rng.integers(labels, 33)))
        sub = np.random.default_rng(int(rng.integers(1 << 62)))
        g, cl, objects = _clustered_scene(sub, n, n_clusters, [-1.5] * 3, [1.5] * 3,
                                          0.05, 0.3, -4.0, 1.0, 1.5)
        group = sub.integers(0, labels, size=n_clusters) + 1   # cluster -> label
        fx = fx_from_hfov(wd, 60.0)
        cams, masks = [], []
        per_ring = max(1, v // 2)
        for i in range(v):
            el = math.radians(15.0 if i < per_ring else 40.0)
            az = math.radians((i % per_ring) * 360.0 / per_ring)
            pos = (5.0 * math.cos(el) * math.sin(az), 5.0 * math.sin(el),
                   -5.0 * math.cos(el) * math.cos(az))
            cam = camera(pos, wd, ht, fx)
            lab = label_map(cam, [(int(group[c]), objects[c][1], objects[c][2], objects[c][3])
                                  for c in range(n_clusters)])
            masks.append(lab.astype(np.uint8))
            cams.append(cam)
        out.append(Workload(f"serve{k}", g, cams, masks, labels + 1, 0.5,
                            group[cl].astype(np.int32), {"P": sum(m.size for m in masks)}))
    return out


def request_masks(w, seed, flip=0.02):
    """A request's masks: the scene's clean masks with fresh seeded noise --
    every pixel flipped to a random other label with probability `flip`,
    drawn as one noise field per view shifted by a seeded offset (cheap
    enough to make per request)."""
    rng = np.random.default_rng(seed)
    out = []
    for v, m in enumerate(w.masks):
        field = _noise_field(w.name, v, m.shape, flip, w.E)
        dy, dx = int(rng.integers(0, m.shape[0])), int(rng.integers(0, m.shape[1]))
        f = np.roll(field, (dy, dx), axis=(0, 1))
        out.append(np.where(f > 0, (m.astype(np.int64) + f) % w.E, m).astype(m.dtype))
    return out


_NOISE = {}


def _noise_field(name, v, shape, flip, E):
    key = (name, v, shape, flip, E)
    if key not in _NOISE:
        rng = np.random.default_rng(zlib.crc32(repr(key).encode()))
        f = np.where(rng.random(shape) < flip, rng.integers(1, max(E, 2), size=shape), 0)
        _NOISE[key] = f.astype(np.int16)
    return _NOISE[key]
