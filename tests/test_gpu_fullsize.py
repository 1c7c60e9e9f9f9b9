"""Full-size workloads through the C ABI, in the benchmark's launch
configuration (50 views per batch, 6 depth chunks, near-tie re-check on),
checked on sampled Gaussians against the oracle and on properties that hold
at any size.

The oracle tracks a sample of rows (each sampled Gaussian is walked over its
own footprint in every view), so it finishes in a minute or two even for
3*10^6 Gaussians and 200 views.  The sample holds seen Gaussians with
footprints of at most 96x96 pixels: those with the smallest decision margins
(where the FP32 table, or the re-check, decides), random ones and the
largest contributors.
"""
import numpy as np
import pytest

import oracle
from oracle.assign import assign, assign_margin
from paper_2409_08270_gb300 import synth
from parity import MARGIN_BAR, table_errors

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


def _solve(fsb, w, masks=None):
    s = fsb.Solver(w.gaussians)
    try:
        out = s.solve(w.cams, w.masks if masks is None else masks, w.E, w.gamma)
        return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}
    finally:
        s.close()


def _footprint_area(w, views=3):
    """Largest pixel bounding box (w x h) of each Gaussian over a few views."""
    area = np.zeros(w.n)
    V = len(w.cams)
    for v in sorted({0, V // 2, V - 1})[:views]:
        pv = oracle.project_view(w.gaussians, w.cams[v])
        area = np.maximum(area, pv[:, 8] * pv[:, 9])
    return area


def _sample(gpu, w, rng, n_tie=10, n_rand=14, n_big=4, max_area=96 * 96):
    """Seen Gaussians whose footprints stay below max_area pixels (the CPU
    oracle walks every pixel of a sampled footprint in every view)."""
    A = gpu["table"].astype(np.float64)
    S = A.sum(1)
    small = _footprint_area(w) <= max_area
    seen = np.flatnonzero((S > 0) & small)
    m = gpu["margin"][seen]
    ties = seen[np.argsort(m)[:n_tie]]
    rest = np.setdiff1d(seen, ties)
    rand = rng.choice(rest, n_rand, replace=False)
    pool = np.setdiff1d(rest, rand)
    big = pool[np.argsort(-S[pool])[:n_big]]
    return np.unique(np.concatenate([ties, rand, big]))


def _check_sample(gpu, w, sel):
    acc = oracle.accumulate(w.gaussians, w.cams, w.masks, w.E, sel=sel)
    ok, rel, summ = table_errors(gpu["table"][sel], acc.table, acc.risk)
    print(w.name, "sampled rows", len(sel), summ, flush=True)
    assert summ["violations"] == 0, summ
    # over 100+ views nearly every row meets some decision near its threshold
    # (risk > 0); the error itself must still be small for almost all entries
    ora = acc.table
    big = ora >= 1e-6 * ora.max()
    rel_all = np.abs(gpu["table"][sel].astype(np.float64) - ora)[big] / ora[big]
    print(w.name, "relative error of", int(big.sum()), "entries: median %.2e, 90%% %.2e, max %.2e"
          % (np.median(rel_all), np.quantile(rel_all, 0.9), rel_all.max()), flush=True)
    assert big.sum() >= len(sel) // 2
    assert np.quantile(rel_all, 0.9) <= 1e-4
    S = assign(acc.table, w.gamma)
    m = assign_margin(acc.table, w.gamma).T
    bits = gpu["bits"][sel].astype(np.uint64)
    Sg = np.stack([((bits >> np.uint64(e)) & np.uint64(1)).astype(bool) for e in range(w.E)])
    decided = m >= MARGIN_BAR
    print(w.name, "sampled decisions", int(decided.sum()), "below bar", int((~decided).sum()),
          "smallest oracle margin", float(m.min()), flush=True)
    assert np.array_equal(Sg[decided], S[decided])
    return acc


def _check_label_independence(fsb, w, gpu):
    """Row sums over labels depend on the scene and cameras only (Eq. 6/7):
    relabelling every pixel 0 must leave them unchanged."""
    zero = [np.zeros_like(m) for m in w.masks]
    g0 = _solve(fsb, w, masks=zero)
    s1 = gpu["table"].astype(np.float64).sum(1)
    s0 = g0["table"].astype(np.float64).sum(1)
    assert np.all(g0["table"][:, 1:] == 0)
    scale = s1.max()
    np.testing.assert_allclose(s1, s0, rtol=2e-5, atol=1e-9 * scale)
    # the whole table's sum is at most one per pixel (Lemma 1)
    assert s1.sum() <= w.pixels * (1 + 1e-5)


@pytest.mark.timeout(900, method="thread")
def test_binary_full_size_sampled(fsb):
    """1,000,000 Gaussians, 100 views of 1008x756, uint8 masks, gamma 0.5."""
    w = synth.binary_scene()
    gpu = _solve(fsb, w)
    st = gpu["stats"]
    assert st.views == 100 and st.pixels == w.pixels and st.bad_labels == 0
    print("binary full size: pairs", st.pairs, "list entries", st.list_entries,
          "re-checked", st.rechecked, "rebinned batches", st.recheck_rebinned, flush=True)
    sel = _sample(gpu, w, np.random.default_rng(11))
    _check_sample(gpu, w, sel)
    _check_label_independence(fsb, w, gpu)


@pytest.mark.timeout(1200, method="thread")
def test_multi_full_size_sampled(fsb):
    """3,000,000 Gaussians in 32 instances, 200 views of 1256x828, int32 id
    masks with 33 labels, FP32 [3M x 33] table, gamma 0.5."""
    w = synth.multi_scene()
    gpu = _solve(fsb, w)
    st = gpu["stats"]
    assert st.views == 200 and st.pixels == w.pixels and st.bad_labels == 0
    print("multi full size: pairs", st.pairs, "list entries", st.list_entries,
          "re-checked", st.rechecked, "rebinned batches", st.recheck_rebinned, flush=True)
    sel = _sample(gpu, w, np.random.default_rng(12), n_tie=8, n_rand=12, n_big=3)
    _check_sample(gpu, w, sel)
    # every instance label that has Gaussians gets some members
    lab = gpu["label"]
    assert len(np.unique(lab[lab > 0])) >= 16
