"""Uses of the solve the paper describes around the hot path: solves split
over view subsets (Sec. 4.8, segmentation from a fraction of the masks) and
object removal (Sec. 4.4), through the C ABI against the oracle."""
import numpy as np
import pytest

import oracle
from oracle.assign import assign, assign_margin
from paper_2409_08270_gb300 import synth
from parity import MARGIN_BAR

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


def test_view_subsets_add_up_to_the_whole_solve(fsb):
    """fs_accumulate is additive (Eq. 6/7 sum over views): two calls over the
    two halves of the views give the one-call table (FP64 sums; only the
    order of the atomic additions differs), and a quarter of the views alone
    leaves more Gaussians unseen (Sec. 4.8)."""
    import torch
    w = synth.binary_scene(n=30000, views=8, width=400, height=300)
    s = fsb.Solver(w.gaussians, recheck_margin=-1.0)
    try:
        whole = s.solve(w.cams, w.masks, w.E, w.gamma, table_dtype="float64")["table"]
        t = torch.zeros((w.n, w.E), dtype=torch.float64, device=s.device)
        s.accumulate(w.cams[:3], w.masks[:3], w.E, t)
        s.accumulate(w.cams[3:], w.masks[3:], w.E, t)
        torch.cuda.synchronize()
        np.testing.assert_allclose(t.cpu().numpy(), whole.cpu().numpy(), rtol=1e-12, atol=1e-15)
        q = torch.zeros_like(t)
        s.accumulate(w.cams[:2], w.masks[:2], w.E, q)
        torch.cuda.synchronize()
    finally:
        s.close()
    seen_all = (whole.cpu().numpy().sum(1) > 0).sum()
    seen_q = (q.cpu().numpy().sum(1) > 0).sum()
    assert seen_q < seen_all
    acc = oracle.accumulate(w.gaussians, w.cams[:2], w.masks[:2], w.E)
    np.testing.assert_array_equal(q.cpu().numpy().sum(1) > 0, acc.table.sum(1) > 0)


def test_object_removal_keeps_the_rest(fsb):
    """Removal (Sec. 4.4, gamma = -0.4): the kept set is every Gaussian in
    none of the removed objects' subsets -- exactly the complement of the
    GPU's own membership bits, and the oracle's wherever its decisions are
    away from their ties."""
    import torch
    w = synth.multi_scene(n=40000, views=4, width=628, height=414, n_clusters=8)
    gamma = -0.4
    s = fsb.Solver(w.gaussians)
    try:
        out = s.solve(w.cams, w.masks, w.E, gamma)
        bits = out["bits"]
        remove = [2, 5, 7]
        keep = s.keep_after_removal(bits, remove).cpu().numpy()
        b = bits.cpu().numpy().astype(np.uint64)
        none_kept = s.keep_after_removal(bits, list(range(w.E)))
        all_kept = s.keep_after_removal(bits, [])
    finally:
        s.close()
    rm = np.uint64(sum(1 << e for e in remove))
    exp = np.flatnonzero((b & rm) == 0)
    np.testing.assert_array_equal(keep, exp)
    assert len(all_kept) == w.n
    assert len(none_kept) == int((b == 0).sum())
    # against the oracle's assignment at gamma = -0.4
    acc = oracle.accumulate(w.gaussians, w.cams, w.masks, w.E)
    S = assign(acc.table, gamma)
    m = assign_margin(acc.table, gamma).T
    decided = (m[remove] >= MARGIN_BAR).all(0)
    ora_keep = ~S[remove].any(0)
    gpu_keep = np.zeros(w.n, bool)
    gpu_keep[keep] = True
    assert decided.mean() > 0.9
    np.testing.assert_array_equal(gpu_keep[decided], ora_keep[decided])
    assert 0 < gpu_keep.sum() < w.n


def test_stage_times_cover_the_solve(fsb):
    """fs_options.time_stages: every stage of a solve is timed on its own
    stream (fs_stats.stage_ms); the blend's share is blend_ms, and without
    the option nothing is timed."""
    w = synth.tiny_scene()
    s = fsb.Solver(w.gaussians, time_stages=True, recheck_margin=1e30)
    try:
        st = s.solve(w.cams, w.masks, w.E, w.gamma)["stats"]
    finally:
        s.close()
    ms = dict(zip(fsb.STAGES, st.stage_ms))
    assert all(v >= 0.0 for v in ms.values()), ms
    for name in ("project", "depth_sort", "pixel_state", "binning", "tile_sort", "blend",
                 "recheck", "assign"):
        assert ms[name] > 0.0, (name, ms)
    assert st.blend_ms == ms["blend"]
    assert st.blend_launches > 0
    plain = fsb.Solver(w.gaussians)
    try:
        st0 = plain.solve(w.cams, w.masks, w.E, w.gamma)["stats"]
    finally:
        plain.close()
    assert all(v == 0.0 for v in st0.stage_ms)
