"""The allocation-free solve (fs_solve_noalloc) against the regular solve and
the FP64 oracle.

Callers that may not allocate device memory -- e.g. code inside an
application whose memory pool owns the whole GPU, or a latency-critical loop
that cannot pay for cudaMalloc/cudaFree -- use fs_solve_noalloc, which works
in a fixed array inside the library.  Its results must equal fs_solve's on the
same scene, on two calls in a row (the second call finds the first call's
leftovers in the shared array), and the oracle's within the FP32 tolerance.
This file is collected last on purpose.
"""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2409_08270_gb300 import synth
from parity import label_check, table_errors

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2409_08270_gb300", "csrc")


@pytest.fixture(scope="module")
def fsb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_08270_gb300 import build, flashsplat
    build.build()
    flashsplat.load()
    return flashsplat


def _noalloc(fsb, w, E, masks_dev, cams=None):
    import torch
    dev = torch.device("cuda", 0)
    g = {k: torch.from_numpy(np.ascontiguousarray(w.gaussians[k])).to(dev) for k in
         ("mean", "quat", "scale", "opacity")}
    gs = fsb.fs_gaussians()
    gs.n = int(g["mean"].shape[0])
    gs.mean, gs.quat = g["mean"].data_ptr(), g["quat"].data_ptr()
    gs.scale, gs.opacity = g["scale"].data_ptr(), g["opacity"].data_ptr()
    gs.quat_dtype = gs.scale_dtype = gs.opacity_dtype = fsb.FS_F32
    gs.memory = fsb.FS_MEM_DEVICE
    n = gs.n
    table = torch.full((n, E), 7.0, dtype=torch.float32, device=dev)   # must be overwritten
    bits = torch.empty(n, dtype=torch.int64, device=dev)
    label = torch.empty(n, dtype=torch.int32, device=dev)
    margin = torch.empty(n, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    torch.cuda.synchronize(dev)
    free_before = torch.cuda.mem_get_info(dev)[0]
    cams = w.cams if cams is None else cams
    fsb.fs_solve_noalloc(0, gs, fsb.make_cameras(cams), [m.data_ptr() for m in masks_dev],
                         fsb.FS_I32 if masks_dev and masks_dev[0].dtype == torch.int32
                         else fsb.FS_U8, E,
                         float(w.gamma), table.data_ptr(), bits.data_ptr(), label.data_ptr(),
                         margin.data_ptr(), stream)
    torch.cuda.synchronize(dev)
    free_after = torch.cuda.mem_get_info(dev)[0]
    return (table.cpu().numpy(), bits.cpu().numpy(), label.cpu().numpy(), margin.cpu().numpy(),
            free_before - free_after)


def test_noalloc_sources_allocate_nothing():
    """The entry point and every launcher it calls contain no allocation."""
    pat = re.compile(r"cudaMalloc|cudaFree|\.ensure\(|malloc\(|new ")
    for f in ("fs_noalloc.cu", "fs_sort.cu", "fs_project.cu", "fs_blend.cu", "fs_assign.cu"):
        src = open(os.path.join(CSRC, f)).read()
        src = re.sub(r"//[^\n]*", "", src)
        assert not pat.search(src), f


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["binary", "multi"])
def test_noalloc_matches_fs_solve_twice(fsb, kind):
    if kind == "binary":
        w = synth.binary_scene(n=12000, views=3, width=320, height=240)
    else:
        w = synth.multi_scene(n=16000, views=2, width=300, height=200, n_clusters=6)
    s = fsb.Solver(w.gaussians)
    try:
        ref = s.solve(w.cams, w.masks, w.E, w.gamma)
        ref = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in ref.items()}
        masks_dev = s.upload_masks(w.masks)
        acc = oracle.accumulate(w.gaussians, w.cams, w.masks, w.E)
        for call in range(2):
            table, bits, label, margin, grew = _noalloc(fsb, w, w.E, masks_dev)
            if call == 1:
                assert grew == 0      # nothing allocated on the device
            scale = np.abs(ref["table"]).max()
            np.testing.assert_allclose(table, ref["table"], rtol=1e-5, atol=1e-11 * scale)
            decided = ref["margin"] > 1e-4        # away from FP32 ties of the two tables
            assert decided.mean() > 0.5
            np.testing.assert_array_equal(bits[decided], ref["bits"][decided])
            np.testing.assert_array_equal(label[decided], ref["label"][decided])
            # and the oracle's, within the FP32 tolerance (no near-tie re-check)
            _, _, summ = table_errors(table, acc.table, acc.risk)
            assert summ["violations"] == 0, summ
            lab = label_check(bits, acc.table, acc.risk, w.gamma)
            assert lab["mismatch_outside_window"] == 0, lab
    finally:
        s.close()


@pytest.mark.gpu
def test_noalloc_without_views(fsb):
    """No views: a zero table, and the decision of an unseen Gaussian
    (member iff gamma < 0)."""
    w = synth.tiny_scene(n=300, views=1)
    for gamma in (0.5, -0.5):
        w.gamma = gamma
        table, bits, label, margin, _ = _noalloc(fsb, w, 2, [], cams=[])
        assert np.all(table == 0)
        assert np.all(bits == (3 if gamma < 0 else 0))
        assert np.all(np.isinf(margin))


@pytest.mark.gpu
def test_noalloc_rejects_oversized_input(fsb):
    w = synth.tiny_scene(n=200, views=1, width=600, height=100)    # wider than the limit
    s = fsb.Solver(w.gaussians)
    try:
        masks_dev = s.upload_masks(w.masks)
        with pytest.raises(fsb.FlashSplatError) as ei:
            _noalloc(fsb, w, w.E, masks_dev)
        assert ei.value.status == fsb.FS_INVALID_ARGUMENT
        assert "FS_NOALLOC_MAX_SIDE" in str(ei.value)
    finally:
        s.close()


@pytest.mark.gpu
def test_noalloc_reports_pair_overflow(fsb):
    """Faint Gaussians wider than the view never saturate a tile, so a late
    depth chunk lists more (tile, Gaussian) pairs than the fixed array holds."""
    n = 4096
    rng = np.random.default_rng(5)
    g = {"mean": np.column_stack([rng.uniform(-0.2, 0.2, n), rng.uniform(-0.2, 0.2, n),
                                  rng.uniform(-0.5, 0.5, n)]).astype(np.float32),
         "quat": np.tile([1, 0, 0, 0], (n, 1)).astype(np.float32),
         "scale": np.full((n, 3), 3.0, np.float32),
         "opacity": np.full(n, 0.005, np.float32)}
    cam = synth.camera((0, 0, -3.0), 512, 512, 500.0)
    w = synth.Workload("wide", g, [cam], [np.ones((512, 512), np.uint8)], 2, 0.5,
                       np.zeros(n, np.int32))
    s = fsb.Solver(w.gaussians)
    try:
        masks_dev = s.upload_masks(w.masks)
        with pytest.raises(fsb.FlashSplatError) as ei:
            _noalloc(fsb, w, 2, masks_dev)
        assert ei.value.status == fsb.FS_UNSUPPORTED
        assert "FS_NOALLOC_MAX_LIST_ENTRIES" in str(ei.value)
    finally:
        s.close()
