"""Novel-view mask rendering on the GPU against the FP64 oracle (Sec. 3.4;
Supp. Sec. 8.2; tau = 0.1 as in Sec. 4.6).

The masks must agree exactly wherever the decision is not within rounding of
a tie: every object's rho^e clear of tau, and the nearest passing object's
depth clear of the next one.  rho^e and D^e agree within 1e-5 relative plus
the oracle's bound on near-threshold alpha and stop decisions.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2409_08270_gb300 import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-5
TAU = 0.1


@pytest.fixture(scope="module")
def fsb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_08270_gb300 import build, flashsplat
    build.build()
    flashsplat.load()
    return flashsplat


@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_scene()


def _novel_cams():
    """Views off the training ring (raised, at other azimuths and distances),
    with sizes that leave ragged tiles."""
    cams = []
    for k, (w, h) in enumerate([(100, 75), (37, 53), (128, 96), (17, 16)]):
        az = 0.7 + 1.3 * k
        r = 2.6 + 0.3 * k
        cams.append(synth.camera((r * math.sin(az), 0.9, -r * math.cos(az)), w, h,
                                 1.1 * w, target=(0.05 * k, -0.05, 0.0)))
    return cams


def _objects(tiny, rng):
    """Four objects split by the octant of the mean, and 15% of the Gaussians
    also in a second object (memberships may overlap, as at gamma < 0)."""
    m = tiny.gaussians["mean"]
    obj = 1 + (m[:, 0] > 0).astype(np.int64) + 2 * (m[:, 1] > 0).astype(np.int64)
    bits = np.left_shift(np.uint64(1), obj.astype(np.uint64))
    extra = rng.random(len(obj)) < 0.15
    second = 1 + rng.integers(0, 4, len(obj))
    bits = bits | np.where(extra, np.left_shift(np.uint64(1), second.astype(np.uint64)),
                           np.uint64(0))
    return bits


def _gpu_render(fsb, g, cams, bits, E, coverage=0, out_dtype="uint8"):
    import torch
    s = fsb.Solver(g, coverage=coverage)
    try:
        dbits = torch.from_numpy(bits.astype(np.int64)).to(s.device)
        out = s.render_masks(cams, dbits, E, tau=TAU, out_dtype=out_dtype, want_planes=True)
        return ([m.cpu().numpy().astype(np.int32) for m in out["masks"]],
                [r.cpu().numpy().astype(np.float64) for r in out["rho"]],
                [d.cpu().numpy().astype(np.float64) for d in out["depth"]])
    finally:
        s.close()


def _compare(gpu, ora):
    masks, rho_g, dep_g = gpu
    n_amb = n_pix = n_rho = 0
    for v in range(len(masks)):
        ro, rr = ora.rho[v], ora.rho_risk[v]
        zo, zr = ora.z_sum[v], ora.z_risk[v]
        do = ora.depth[v]
        # rho^e within 1e-5 relative plus the oracle's bound
        err = np.abs(rho_g[v] - ro)
        bound = RTOL * ro + 1.01 * rr + 1e-7
        assert np.all(err <= bound), (v, float((err - bound).max()))
        n_rho += int((ro > 0).sum())
        # D^e where the object is seen: the relative error of sum alpha T z and
        # of rho^e, plus their bounds carried through the quotient
        seen = ro >= 1e-3
        dtol = 3 * RTOL * do + (zr + do * rr) / np.maximum(ro, 1e-30)
        assert np.all(np.abs(dep_g[v] - do)[seen] <= dtol[seen] + 1e-6)
        # masks: exact unless a decision sits within its tolerance
        near_tau = (np.abs(ro - TAU) <= RTOL * TAU + 1.01 * rr + 1e-7).any(0)
        passing = ro > TAU
        d_pass = np.where(passing, do, np.inf)
        d_sorted = np.sort(d_pass, axis=0)
        if d_sorted.shape[0] > 1:
            two = np.isfinite(d_sorted[1])         # at least two objects pass
            with np.errstate(invalid="ignore"):
                gap = np.where(two, d_sorted[1] - d_sorted[0], np.inf)
        else:
            two = np.zeros_like(near_tau)
            gap = np.full(near_tau.shape, np.inf)
        near_depth = two & (gap <= 2 * dtol.max(0) + 1e-6)
        amb = near_tau | near_depth
        lab_o = ora.label[v]
        assert np.array_equal(masks[v][~amb], lab_o[~amb]), (v, int((masks[v] != lab_o)[~amb].sum()))
        n_amb += int(amb.sum())
        n_pix += amb.size
    assert n_amb <= 0.005 * n_pix, (n_amb, n_pix)
    assert n_rho > 1000
    return n_amb


def test_binary_masks_of_the_ground_truth_foreground(fsb, tiny):
    """E = 2: the mask is [rho^1 > 0.1] over the foreground Gaussians."""
    cams = _novel_cams()
    bits = np.where(tiny.gt == 1, np.uint64(2), np.uint64(0))
    ora = oracle.render_masks(tiny.gaussians, cams, bits, 2, tau=TAU)
    gpu = _gpu_render(fsb, tiny.gaussians, cams, bits, 2)
    n_amb = _compare(gpu, ora)
    fg = sum(int((m == 1).sum()) for m in gpu[0])
    print("binary novel views: foreground pixels", fg, "ambiguous", n_amb)
    assert fg > 500 and fg < sum(m.size for m in gpu[0]) // 2


@pytest.mark.parametrize("coverage,out_dtype", [(0, "uint8"), (1, "int32")])
def test_scene_masks_depth_guided(fsb, tiny, coverage, out_dtype):
    """Four overlapping objects: each rendered alone, the nearest passing
    object wins; under exact and 3-sigma coverage, uint8 and int32 masks."""
    cams = _novel_cams()
    bits = _objects(tiny, np.random.default_rng(5))
    ora = oracle.render_masks(tiny.gaussians, cams, bits, 5, tau=TAU, coverage=coverage)
    gpu = _gpu_render(fsb, tiny.gaussians, cams, bits, 5, coverage=coverage, out_dtype=out_dtype)
    n_amb = _compare(gpu, ora)
    seen = set()
    for m in gpu[0]:
        seen |= set(np.unique(m).tolist())
    print("scene novel views: labels", sorted(seen), "ambiguous", n_amb)
    assert seen == {0, 1, 2, 3, 4}
    # pixels where two or more objects pass: the depth decided them
    multi = sum(int(((r > TAU).sum(0) >= 2).sum()) for r in ora.rho)
    assert multi > 200


def test_masks_from_the_solve(fsb, tiny):
    """The user path: solve on the training views, then render the solve's
    members into novel views; the oracle renders the same members."""
    import torch
    cams = _novel_cams()
    s = fsb.Solver(tiny.gaussians)
    try:
        out = s.solve(tiny.cams, tiny.masks, tiny.E, tiny.gamma)
        bits = out["bits"]
        r = s.render_masks(cams, bits, tiny.E, tau=TAU, want_planes=True)
        gpu = ([m.cpu().numpy().astype(np.int32) for m in r["masks"]],
               [x.cpu().numpy().astype(np.float64) for x in r["rho"]],
               [x.cpu().numpy().astype(np.float64) for x in r["depth"]])
        host_bits = bits.cpu().numpy().astype(np.uint64)
    finally:
        s.close()
    ora = oracle.render_masks(tiny.gaussians, cams, host_bits, tiny.E, tau=TAU)
    _compare(gpu, ora)
    assert sum(int(m.sum()) for m in gpu[0]) > 300
