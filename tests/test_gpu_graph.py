"""A solve captured into a CUDA graph (fs_graph_*) against the uncaptured
fs_solve on the same context options.

The replay must give the same decisions (bits, labels) and the same FP64
table up to the order of the FP64 atomic additions -- the only difference
between any two solves -- checked at 1e-12 relative.  Replays after new
masks are written into the captured mask buffers must match uncaptured
solves of those masks, including masks with out-of-range labels, whose lists
are shorter than the capture's plan.
"""
import numpy as np
import pytest

from paper_2409_08270_gb300 import synth

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


@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_scene()


def _host(d):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in d.items() if v is not None}


def _same_solve(a, b, rtol=1e-12):
    np.testing.assert_array_equal(a["bits"], b["bits"])
    np.testing.assert_array_equal(a["label"], b["label"])
    ta, tb = a["table"].astype(np.float64), b["table"].astype(np.float64)
    scale = max(1e-300, float(np.abs(tb).max()))
    np.testing.assert_allclose(ta, tb, rtol=rtol, atol=rtol * 1e-6 * scale)
    np.testing.assert_allclose(a["margin"], b["margin"], rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("opts", [
    {},                                                 # one batch, re-check on
    {"views_per_batch": 3},                             # three batches
    {"views_per_batch": 2, "recheck_margin": -1.0},     # no re-check
    {"views_per_batch": 3, "coverage": 1},              # 3-sigma coverage
    {"record_precision": 3},                            # reduced-precision records (FS_F16)
    # every Gaussian re-checked after each replay: the re-check's full-depth
    # lists outgrow the main pass's, on a context of their own
    {"views_per_batch": 3, "recheck_margin": 10.0},
])
def test_captured_solve_replays_the_solve(fsb, tiny, opts):
    import torch
    s = fsb.Solver(tiny.gaussians, **opts)
    try:
        dm = s.upload_masks(tiny.masks)
        ref = _host(s.solve(tiny.cams, dm, tiny.E, tiny.gamma, table_dtype="float64"))
        g = s.capture(tiny.cams, dm, tiny.E, tiny.gamma, table_dtype="float64")
        try:
            for _ in range(2):
                g.launch()
                g.synchronize()
                _same_solve(_host(g.outputs), ref)
            # new masks written into the captured buffers: labels moved, and
            # some pixels with a label outside [0, E) (skipped: shorter lists)
            rng = np.random.default_rng(9)
            new = []
            for m in tiny.masks:
                x = m.copy()
                flip = rng.random(x.shape) < 0.2
                x[flip] = 1 - x[flip]
                x[rng.random(x.shape) < 0.1] = 7
                new.append(x)
            for d, x in zip(dm, new):
                d.copy_(torch.from_numpy(x).to(d.device))
            g.launch()
            st = g.synchronize()
            want = _host(s.solve(tiny.cams, dm, tiny.E, tiny.gamma, table_dtype="float64"))
            _same_solve(_host(g.outputs), want)
            assert st.bad_labels > 0
        finally:
            g.close()
    finally:
        s.close()


def test_captured_fp32_table_is_the_rounded_fp64_one(fsb, tiny):
    """An FP32 table output: the replay rounds its FP64 sums once, outside
    the graph, like fs_solve."""
    s = fsb.Solver(tiny.gaussians)
    try:
        dm = s.upload_masks(tiny.masks)
        ref = _host(s.solve(tiny.cams, dm, tiny.E, tiny.gamma))
        g = s.capture(tiny.cams, dm, tiny.E, tiny.gamma)
        try:
            g.launch()
            g.synchronize()
            out = _host(g.outputs)
            assert out["table"].dtype == np.float32
            _same_solve(out, ref, rtol=1e-7)
        finally:
            g.close()
    finally:
        s.close()
