"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Sizes span several 16x16 tiles with ragged right/bottom edges.  Contributions
must agree within 1e-5 relative (plus the oracle's near-threshold risk bound);
membership decisions must agree exactly wherever the table's error cannot
reach the decision (see tests/parity.py).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2409_08270_gb300 import synth
from parity import label_check, table_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fsb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_08270_gb300 import build, flashsplat
    build.build()
    flashsplat.load()
    return flashsplat


def _solve(fsb, w, table_dtype="float32", views_per_batch=0, masks=None, E=None, gamma=None,
           depth_chunks=0, recheck_margin=0.0, **solver_kw):
    s = fsb.Solver(w.gaussians, views_per_batch=views_per_batch, depth_chunks=depth_chunks,
                   recheck_margin=recheck_margin, **solver_kw)
    try:
        out = s.solve(w.cams, w.masks if masks is None else masks, w.E if E is None else E,
                      w.gamma if gamma is None else gamma, table_dtype=table_dtype)
        return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}
    finally:
        s.close()


def _check(gpu, acc, gamma, rtol=1e-5):
    ok, rel, summ = table_errors(gpu["table"], acc.table, acc.risk, rtol=rtol)
    if summ["violations"]:
        for b in np.argwhere(~ok)[:20]:
            i, e = int(b[0]), int(b[1])
            print(f"VIOLATION gaussian {i} label {e}: gpu {gpu['table'][i, e]:.9e} "
                  f"oracle {acc.table[i, e]:.9e} risk {acc.risk[i, e]:.3e} flags {acc.flags[i]}")
    assert summ["violations"] == 0, summ
    lab = label_check(gpu["bits"], acc.table, acc.risk, gamma, table_rtol=rtol)
    assert lab["mismatch_outside_window"] == 0, lab
    return summ, lab


def test_tiny_scene(fsb, tiny):
    gpu = _solve(fsb, tiny)
    acc = oracle.accumulate(tiny.gaussians, tiny.cams, tiny.masks, tiny.E)
    summ, lab = _check(gpu, acc, tiny.gamma)
    print("tiny", summ, lab)
    assert summ["checked_rel"] > 1000
    assert gpu["stats"].bad_labels == 0 and gpu["stats"].views == len(tiny.cams)


def test_tiny_scene_fp64_table_and_batching(fsb, tiny):
    gpu = _solve(fsb, tiny, table_dtype="float64", views_per_batch=3)
    acc = oracle.accumulate(tiny.gaussians, tiny.cams, tiny.masks, tiny.E)
    _check(gpu, acc, tiny.gamma)


@pytest.mark.parametrize("recheck_margin", [0.0, -1.0])
def test_view_batches_do_not_change_results(fsb, tiny, recheck_margin):
    """One view per batch gives the table of a single batch of all views: the
    per-view terms are the same, only the order of the FP64 atomic sums
    differs.  With the re-check on, the next batch's projection overlaps the
    current batch's binning and blending on a side stream, in alternating
    buffers; with it off the batches run one after another in one set."""
    one = _solve(fsb, tiny, table_dtype="float64", views_per_batch=len(tiny.cams),
                 recheck_margin=recheck_margin)
    many = _solve(fsb, tiny, table_dtype="float64", views_per_batch=1,
                  recheck_margin=recheck_margin)
    np.testing.assert_allclose(many["table"], one["table"], rtol=1e-12, atol=1e-15)
    np.testing.assert_array_equal(many["bits"], one["bits"])
    assert many["stats"].views == one["stats"].views == len(tiny.cams)


@pytest.mark.parametrize("E", [3, 7, 40])
def test_random_multilabel_masks(fsb, tiny, E):
    """i.i.d. random labels: every warp holds several labels, and with E = 7
    or 40 most tiles exceed the shared-memory label slots (direct path)."""
    rng = np.random.default_rng(E)
    masks = [rng.integers(0, E, size=m.shape).astype(np.int32) for m in tiny.masks[:4]]
    cams = tiny.cams[:4]
    w = synth.Workload("t", tiny.gaussians, cams, masks, E, 0.0, tiny.gt)
    gpu = _solve(fsb, w)
    acc = oracle.accumulate(tiny.gaussians, cams, masks, E)
    _check(gpu, acc, 0.0)


def test_bad_labels_skipped_and_counted(fsb, tiny):
    masks = [m.astype(np.int32).copy() for m in tiny.masks[:2]]
    masks[0][:3, :] = 9
    masks[1][:, :5] = -4
    w = synth.Workload("t", tiny.gaussians, tiny.cams[:2], masks, 2, 0.5, tiny.gt)
    gpu = _solve(fsb, w)
    acc = oracle.accumulate(tiny.gaussians, tiny.cams[:2], masks, 2)
    _check(gpu, acc, 0.5)
    assert gpu["stats"].bad_labels == acc.n_bad_label == 3 * 128 + 5 * 128


@pytest.mark.parametrize("gamma", [-1.0, -0.8, -0.4, 0.0, 0.4, 0.8, 1.0])
def test_assign_kernel_matches_oracle_rule(fsb, gamma):
    """The fused assignment on an FP64 table against the oracle's rule."""
    import torch
    rng = np.random.default_rng(3)
    A = rng.exponential(1.0, (20000, 5)) * (rng.random((20000, 5)) < 0.5)
    A[:30] = 0
    A[30:40] = np.array([1.0, 3.0, 0, 0, 0])   # exact ties for gamma = 0.5 ... and others
    s = fsb.Solver({"mean": np.zeros((1, 3), np.float32), "quat": np.array([[1, 0, 0, 0]], np.float32),
                    "scale": np.ones((1, 3), np.float32), "opacity": np.ones(1, np.float32)})
    try:
        for dt in (torch.float64, torch.float32):
            t = torch.from_numpy(A).to(dt).cuda()
            bits, label, margin = s.assign(t, gamma)
            torch.cuda.synchronize()
            Aref = t.double().cpu().numpy()
            S = oracle.assign(Aref, gamma)
            b = bits.cpu().numpy().astype(np.uint64)
            Sg = np.stack([((b >> np.uint64(e)) & np.uint64(1)).astype(bool) for e in range(5)])
            m = oracle.assign_margin(Aref, gamma).T
            safe = m > (1e-12 if dt == torch.float64 else 1e-6)
            assert np.array_equal(Sg[safe], S[safe])
            from oracle.assign import labels_from_membership
            lab = labels_from_membership(S)
            safe_lab = safe.all(0)
            assert np.array_equal(label.cpu().numpy()[safe_lab], lab[safe_lab])
            mo = m.min(0)
            mg = margin.cpu().numpy()
            fin = np.isfinite(mo)
            assert np.allclose(mg[fin], mo[fin], rtol=1e-5, atol=1e-6)
            assert np.isinf(mg[~fin]).all()
    finally:
        s.close()


def test_binary_scene_reduced(fsb):
    """Real-scene statistics (clustered, anisotropic log-scales N(-4,1)) at a
    size the oracle finishes in seconds; 1008x756 views keep the ragged rows."""
    w = synth.binary_scene(n=40000, views=3, width=1008, height=756)
    gpu = _solve(fsb, w)
    acc = oracle.accumulate(w.gaussians, w.cams, w.masks, w.E)
    summ, lab = _check(gpu, acc, w.gamma)
    print("binary", summ, lab)
    assert summ["checked_rel"] > 3000


def test_multi_scene_reduced(fsb):
    w = synth.multi_scene(n=60000, views=4, width=628, height=414)
    gpu = _solve(fsb, w)
    acc = oracle.accumulate(w.gaussians, w.cams, w.masks, w.E)
    summ, lab = _check(gpu, acc, w.gamma)
    print("multi", summ, lab)


def test_degenerate_inputs(fsb):
    """Nothing visible, a 1x1 view, a Gaussian behind the camera, one Gaussian."""
    g = {"mean": np.array([[0, 0, -5.0], [0, 0, 0.0]], np.float32),
         "quat": np.array([[1, 0, 0, 0], [0, 0, 0, 2.0]], np.float32),
         "scale": np.full((2, 3), 0.3, np.float32), "opacity": np.array([0.9, 0.7], np.float32)}
    cams = [synth.camera((0, 0, -3.0), 1, 1, 2.0), synth.camera((0, 0, 3.0), 17, 33, 20.0),
            synth.camera((0, 0, -3.0), 40, 24, 30.0)]
    masks = [np.ones((1, 1), np.uint8), np.zeros((33, 17), np.uint8), np.ones((24, 40), np.uint8)]
    w = synth.Workload("deg", g, cams, masks, 2, 0.5, np.zeros(2, np.int32))
    gpu = _solve(fsb, w)
    acc = oracle.accumulate(g, cams, masks, 2)
    _check(gpu, acc, 0.5)
    assert acc.table.sum() > 0


def test_scene_validation(fsb):
    bad = {"mean": np.zeros((2, 3), np.float32), "quat": np.zeros((2, 4), np.float32),
           "scale": np.ones((2, 3), np.float32), "opacity": np.ones(2, np.float32)}
    with pytest.raises(fsb.FlashSplatError) as ei:
        fsb.Solver(bad)
    assert ei.value.status == fsb.FS_INVALID_ARGUMENT


def test_depth_chunks_do_not_change_results(fsb):
    """Front-to-back chunked binning (tiles drop out once saturated) walks the
    same terms in the same order as one list per tile."""
    w = synth.binary_scene(n=30000, views=2, width=400, height=300)
    # FP32 path alone: a near-tie re-check could take a Gaussian in one run
    # and not in the other
    a = _solve(fsb, w, depth_chunks=1, recheck_margin=-1.0)
    b = _solve(fsb, w, depth_chunks=6, recheck_margin=-1.0)
    np.testing.assert_allclose(b["table"], a["table"], rtol=2e-6, atol=1e-9)
    assert b["stats"].list_entries < a["stats"].list_entries
    acc = oracle.accumulate(w.gaussians, w.cams, w.masks, w.E)
    _check(b, acc, w.gamma)


@pytest.mark.parametrize("case", ["opaque_stack", "two_layer"])
def test_golden_stacks_on_one_pixel(fsb, case):
    """Hand-derived compositing values (tests/golden/closed_forms.json) on a
    1x1 view whose pixel centre is the Gaussians' projected mean."""
    import json, os
    gd = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))[case]
    if case == "opaque_stack":
        means = [[0, 0, 2.0]] * gd["count"]
        opac = [gd["opacity"]] * gd["count"]
        order = list(range(gd["count"]))
    else:
        means = [[0, 0, 3.0], [0, 0, 2.0]]          # index 0 is behind
        opac = [gd["opacity_back"], gd["opacity_front"]]
        order = [1, 0]
    n = len(means)
    g = {"mean": np.array(means, np.float32), "quat": np.tile([1, 0, 0, 0], (n, 1)).astype(np.float32),
         "scale": np.full((n, 3), 0.05, np.float32), "opacity": np.array(opac, np.float32)}
    cam = {"R": np.eye(3), "t": np.zeros(3), "fx": 40.0, "fy": 40.0, "cx": 0.5, "cy": 0.5,
           "width": 1, "height": 1}
    w = synth.Workload("g", g, [cam], [np.ones((1, 1), np.uint8)], 2, 0.0, np.zeros(n, np.int32))
    gpu = _solve(fsb, w)
    got = [float(gpu["table"][i, 1]) for i in order]
    exp = list(gd["contributions"]) + [0.0] * (n - len(gd["contributions"]))
    np.testing.assert_allclose(got, exp, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("kind", ["tiny", "binary"])
def test_census_counts_the_oracles_work_unit(fsb, tiny, kind):
    """The work unit of the blend's roofline: (pixel, Gaussian) pairs with
    alpha >= 1/255 that a pixel's front-to-back walk reaches, its stop
    included (Sec. 3.1 Eq. 1 with the rasteriser's skip and stop rules).  The
    census variant counts them on the GPU; the oracle counts them in its own
    walk.  They may differ only where a decision sits on its threshold.  The
    census variant must give the same table as the timed one."""
    w = tiny if kind == "tiny" else synth.binary_scene(n=40000, views=2, width=1008, height=756)
    s = fsb.Solver(w.gaussians, census=True, recheck_margin=-1.0)
    try:
        c = s.solve(w.cams, w.masks, w.E, w.gamma)
        c = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in c.items()}
    finally:
        s.close()
    p = _solve(fsb, w, recheck_margin=-1.0)
    np.testing.assert_allclose(c["table"], p["table"], rtol=1e-6, atol=1e-12)
    acc = oracle.accumulate(w.gaussians, w.cams, w.masks, w.E)
    st = c["stats"]
    print(kind, "census", st.census_pairs, "oracle", acc.n_part, "evaluated", st.pairs,
          "staged", st.staged_entries)
    assert acc.n_part > 0
    assert abs(st.census_pairs - acc.n_part) <= max(16, 1e-5 * acc.n_part)
    assert st.pairs >= st.census_pairs
    assert p["stats"].census_pairs == 0 and p["stats"].pairs == 0


def test_label_boundaries_inside_sub_tiles(fsb, tiny):
    """Masks whose labels change inside 8x8 sub-tiles and between the two
    pixels a lane walks (vertical stripes of odd width, checkerboard blocks),
    with bad labels mixed in: every (Gaussian, label) sum still matches."""
    H, W = tiny.cams[0]["height"], tiny.cams[0]["width"]
    yy, xx = np.mgrid[0:H, 0:W]
    m1 = ((xx // 3) % 4).astype(np.int32)                 # stripes 3 px wide, 4 labels
    m2 = (((xx // 5) + (yy // 7)) % 3).astype(np.int32)    # blocks
    m2[::11, ::13] = 9                                     # out of range: skipped
    masks = [m1, m2] * 4
    w = synth.Workload("stripes", tiny.gaussians, tiny.cams, masks, 4, 0.3, tiny.gt)
    gpu = _solve(fsb, w)
    acc = oracle.accumulate(tiny.gaussians, tiny.cams, masks, 4)
    _check(gpu, acc, 0.3)
    assert gpu["stats"].bad_labels == acc.n_bad_label > 0


def test_bounded_wait_gives_up_with_timeout(fsb, tiny):
    """The binning's wait for a preceding block's offset is bounded: on a
    grid whose predecessor never publishes, it gives up after the given
    number of polls and reports FS_TIMEOUT; the device stays usable."""
    assert fsb.fs_check_wait_timeout(0, 2000) == fsb.FS_TIMEOUT
    assert "gave up" in fsb.fs_last_error()
    gpu = _solve(fsb, synth.tiny_scene(n=500, views=1))
    assert gpu["table"].sum() > 0


def _sigma3_scene(seed=41, n=3000, views=4, width=160, height=120):
    """Opaque Gaussians stretched along the image x or y axis (cameras look
    down z): their alpha >= 1/255 region reaches 3.3 sigma along the long
    axis, past the 3-sigma square, so the two coverages differ."""
    rng = np.random.default_rng(seed)
    ang = rng.uniform(-0.03, 0.03, n)
    quat = np.column_stack([np.cos(ang), np.zeros(n), np.zeros(n), np.sin(ang)]).astype(np.float32)
    long_, short = rng.uniform(0.04, 0.12, n), rng.uniform(0.005, 0.02, n)
    along_x = rng.random(n) < 0.5
    scale = np.column_stack([np.where(along_x, long_, short), np.where(along_x, short, long_),
                             rng.uniform(0.005, 0.02, n)]).astype(np.float32)
    mean = np.column_stack([rng.uniform(-1, 1, n), rng.uniform(-0.75, 0.75, n),
                            rng.uniform(-0.5, 0.5, n)]).astype(np.float32)
    g = {"mean": mean, "quat": quat, "scale": scale,
         "opacity": rng.uniform(0.5, 0.99, n).astype(np.float32)}
    cams = [synth.camera((rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1), -3.0), width, height,
                         150.0, target=(rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1), 0.0))
            for _ in range(views)]
    yy, xx = np.mgrid[0:height, 0:width]
    masks = [((xx + 0.5 * yy) > 0.6 * width).astype(np.uint8) for _ in cams]
    return synth.Workload("sigma3", g, cams, masks, 2, 0.0, np.zeros(n, np.int32))


@pytest.mark.parametrize("variant", ["main", "batched_recheck_all", "recheck_reproject"])
def test_3sigma_coverage_matches_the_oracle(fsb, variant):
    """FS_COVERAGE_3SIGMA against the oracle's 3-sigma mode (Sec. 4.2's
    standard rasteriser coverage): the table within the FP32 tolerance and
    the labels outside the decision window.  The variants run the clipped
    columns through every binning path: the main pass; one view per batch
    with every Gaussian re-checked from the kept lists; the re-check that
    projects again."""
    w = _sigma3_scene()
    acc3 = oracle.accumulate(w.gaussians, w.cams, w.masks, w.E, coverage=oracle.COVERAGE_3SIGMA)
    exact = oracle.accumulate(w.gaussians, w.cams, w.masks, w.E)
    moved = np.abs(acc3.table - exact.table).sum(1) / np.maximum(exact.table.sum(1), 1e-30)
    assert (moved > 1e-4).sum() >= 100          # the coverages differ well past the tolerance
    kw = {"coverage": fsb.FS_COVERAGE_3SIGMA}
    if variant == "batched_recheck_all":
        kw.update(views_per_batch=1, recheck_margin=10.0)
    elif variant == "recheck_reproject":
        kw.update(recheck_margin=10.0, recheck_reproject=True)
    gpu = _solve(fsb, w, table_dtype="float64", **kw)
    summ, lab = _check(gpu, acc3, w.gamma)
    print("3-sigma", variant, summ, lab)
    assert summ["checked_rel"] > 1000
    # and the GPU table is the 3-sigma one, not the exact one
    far = moved > 1e-4
    rel_exact = np.abs(gpu["table"][far] - exact.table[far]).sum(1) / exact.table[far].sum(1)
    assert np.all(rel_exact > 5e-5)
