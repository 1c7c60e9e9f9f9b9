"""The reduced-precision form (BF16 quaternions and scales, FP16 opacity,
per-view records with an FP16 whitening matrix and FP32 mean; blending in
FP32, table in FP64) against the oracle of that form.

The oracle of the form takes the same rounded attributes and evaluates alpha
from the record rounded the same way (oracle.accumulate(record_f16=True)), so
the FP32 path must meet the plain form's bars against it.  Against the plain
FP32 oracle the form is reported (precision cost), with a loose bound.
"""
import numpy as np
import pytest

import oracle
from oracle.assign import assign, assign_margin
from paper_2409_08270_gb300 import synth
from parity import MARGIN_BAR, label_check, table_errors

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


def _device_form(g):
    """Attributes in their storage types: bfloat16 quat/scale, float16 opacity."""
    import torch
    r = synth.rounded_gaussians(g)
    return {"mean": torch.from_numpy(r["mean"]),
            "quat": torch.from_numpy(r["quat"]).to(torch.bfloat16),
            "scale": torch.from_numpy(r["scale"]).to(torch.bfloat16),
            "opacity": torch.from_numpy(r["opacity"]).to(torch.float16)}, r


def _solve(fsb, g, w, table_dtype="float32", **kw):
    s = fsb.Solver(g, record_precision=fsb.FS_F16, **kw)
    try:
        out = s.solve(w.cams, w.masks, w.E, w.gamma, table_dtype=table_dtype)
        return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}
    finally:
        s.close()


@pytest.mark.parametrize("kind", ["tiny", "binary", "multi"])
def test_reduced_precision_form_matches_its_oracle(fsb, tiny, kind):
    if kind == "tiny":
        w = tiny
    elif kind == "binary":
        w = synth.binary_scene(n=40000, views=3, width=1008, height=756)
    else:
        w = synth.multi_scene(n=60000, views=3, width=628, height=414)
    gdev, grnd = _device_form(w.gaussians)
    gpu = _solve(fsb, gdev, w)
    acc = oracle.accumulate(grnd, w.cams, w.masks, w.E, record_f16=True)
    ok, rel, summ = table_errors(gpu["table"], acc.table, acc.risk)
    print(kind, "reduced-precision form vs its oracle", summ, flush=True)
    assert summ["violations"] == 0, summ
    lab = label_check(gpu["bits"], acc.table, acc.risk, w.gamma)
    assert lab["mismatch_outside_window"] == 0, lab
    # the precision cost: against the plain FP32 scene and records
    plain = oracle.accumulate(w.gaussians, w.cams, w.masks, w.E)
    S0 = assign(plain.table, w.gamma)
    bits = gpu["bits"].astype(np.uint64)
    Sg = np.stack([((bits >> np.uint64(e)) & np.uint64(1)).astype(bool) for e in range(w.E)])
    seen = plain.table.sum(1) > 0
    agree = (S0 == Sg)[:, seen].mean()
    big = plain.table >= 1e-4 * plain.table.max()
    err = np.abs(gpu["table"][big] - plain.table[big]) / plain.table[big]
    print(kind, "vs plain FP32 oracle: label agreement %.5f, rel. error mean %.2e max %.2e"
          % (agree, err.mean(), err.max()), flush=True)
    assert agree > 0.98


def test_reduced_precision_recheck_all_equals_its_oracle(fsb, tiny):
    """Re-checking every Gaussian evaluates the rounded record in float
    pairs: the FP64 table equals the form's oracle to FP64-level precision."""
    gdev, grnd = _device_form(tiny.gaussians)
    gpu = _solve(fsb, gdev, tiny, table_dtype="float64", recheck_margin=1e30)
    acc = oracle.accumulate(grnd, tiny.cams, tiny.masks, tiny.E, record_f16=True, event_rel=1e-9)
    ok, rel, summ = table_errors(gpu["table"], acc.table, acc.risk, rtol=1e-9)
    print("reduced-precision re-check", summ, flush=True)
    assert summ["violations"] == 0, summ
    S = assign(acc.table, tiny.gamma)
    m = assign_margin(acc.table, tiny.gamma).T
    bits = gpu["bits"].astype(np.uint64)
    Sg = np.stack([((bits >> np.uint64(e)) & np.uint64(1)).astype(bool) for e in range(tiny.E)])
    decided = m >= 1e-8
    assert np.array_equal(Sg[decided], S[decided])
