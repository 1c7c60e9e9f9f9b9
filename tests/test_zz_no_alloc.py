"""The allocation-free solve (fs_solve_noalloc) against the regular solve.

Callers that may not allocate device memory -- e.g. code inside an
application whose memory pool owns the whole GPU, or a latency-critical loop
that cannot pay for cudaMalloc/cudaFree -- use fs_solve_noalloc, which works
in a fixed array inside the library.  Its results must equal fs_solve's on the
same scene, on two calls in a row (the second call finds the first call's
leftovers in the shared array).  This file is collected last on purpose.
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


def _noalloc(fsb, w, E, masks_dev):
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
    fsb.fs_solve_noalloc(0, gs, fsb.make_cameras(w.cams), [m.data_ptr() for m in masks_dev],
                         fsb.FS_I32 if masks_dev[0].dtype == torch.int32 else fsb.FS_U8, E,
                         float(w.gamma), table.data_ptr(), bits.data_ptr(), label.data_ptr(),
                         margin.data_ptr(), stream)
    torch.cuda.synchronize(dev)
    return table.cpu().numpy(), bits.cpu().numpy(), label.cpu().numpy(), margin.cpu().numpy()


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
        for _ in range(2):
            table, bits, label, margin = _noalloc(fsb, w, w.E, masks_dev)
            scale = np.abs(ref["table"]).max()
            np.testing.assert_allclose(table, ref["table"], rtol=1e-5, atol=1e-11 * scale)
            decided = ref["margin"] > 1e-4        # away from FP32 ties of the two tables
            assert decided.mean() > 0.5
            np.testing.assert_array_equal(bits[decided], ref["bits"][decided])
            np.testing.assert_array_equal(label[decided], ref["label"][decided])
    finally:
        s.close()


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
