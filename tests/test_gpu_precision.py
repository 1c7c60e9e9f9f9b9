"""The reduced-precision form (BF16 quaternions and scales, FP16 opacity;
per-view records with an FP32 mean and an FP16 whitening matrix W computed in
plain FP32; blending in FP32, table in FP64) against the FP64 oracle.

The form is judged against the plain FP64 oracle on the ORIGINAL inputs: the
label agreement is asserted and the table's relative error reported.  Its
error budget comes from the roundings it makes: BF16 scales and quaternions
(2^-9 relative per value) and the FP16 entries of W (2^-11 relative), which
move the exponent q = |W d|^2 at a pixel by up to a few 1e-3 relative for
round footprints and more at the tips of elongated ones.

As a diagnostic the form is also compared with the oracle of its own model
(the same rounded attributes, alpha from W rounded to FP16: record_f16).  W
is built in FP64 there and in FP32 here; where the footprint is nearly round
the two are rotated differently and round to FP16 differently, so those
entries differ at the FP16 level, and the typical entry must agree to the
FP32 bar.
"""
import numpy as np
import pytest

import oracle
from oracle.assign import assign
from paper_2409_08270_gb300 import synth
from parity import table_errors

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


def _bits_matrix(bits, E):
    b = bits.astype(np.uint64)
    return np.stack([((b >> np.uint64(e)) & np.uint64(1)).astype(bool) for e in range(E)])


@pytest.mark.parametrize("kind", ["tiny", "binary", "multi"])
def test_reduced_precision_form_against_the_plain_oracle(fsb, tiny, kind):
    if kind == "tiny":
        w = tiny
    elif kind == "binary":
        w = synth.binary_scene(n=40000, views=3, width=1008, height=756)
    else:
        w = synth.multi_scene(n=60000, views=3, width=628, height=414)
    gdev, grnd = _device_form(w.gaussians)
    gpu = _solve(fsb, gdev, w)
    # the form's cost: against the plain FP64 oracle on the original inputs
    plain = oracle.accumulate(w.gaussians, w.cams, w.masks, w.E)
    S0 = assign(plain.table, w.gamma)
    Sg = _bits_matrix(gpu["bits"], w.E)
    seen = plain.table.sum(1) > 0
    agree = (S0 == Sg)[:, seen].mean()
    big = plain.table >= 1e-4 * plain.table.max()
    err = np.abs(gpu["table"][big] - plain.table[big]) / plain.table[big]
    print(kind, "vs plain FP64 oracle: label agreement %.5f, rel. error mean %.2e median %.2e "
          "max %.2e" % (agree, err.mean(), np.median(err), err.max()), flush=True)
    # budget: a BF16 scale moves 1/s^2 by up to 2^-8 = 3.9e-3 relative, so the
    # exponent q/2 of alpha = o e^(-q/2) moves by up to 3.9e-3 q/2, and q/2
    # averages 1 under the Gaussian's own weight; the FP16 entries of W add
    # up to ~1e-3 (2^-11 per entry, first order in |W d|): a typical entry
    # moves by a few 1e-3, the tails of elongated footprints and everything
    # behind a moved alpha (through T) by more
    assert agree > 0.99
    assert np.median(err) < 5e-3
    # diagnostic: against the oracle of the form's own model.  A nearly round
    # footprint has an ill-conditioned eigenvector, so FP32 and FP64 build W
    # at different angles, which round to FP16 differently: those entries
    # differ at the FP16 level; the typical entry agrees to the FP32 bar
    acc = oracle.accumulate(grnd, w.cams, w.masks, w.E, record_f16=True)
    ok, rel, summ = table_errors(gpu["table"], acc.table, acc.risk)
    frac = summ["violations"] / max(1, summ["checked_rel"] + summ["with_risk"])
    big2 = acc.table >= 1e-4 * acc.table.max()
    err2 = np.abs(gpu["table"][big2] - acc.table[big2]) / acc.table[big2]
    print(kind, "vs its record_f16 oracle", summ, "beyond 1e-5 + bound: %.4f, median %.2e, "
          "mean %.2e" % (frac, np.median(err2), err2.mean()), flush=True)
    assert np.median(err2) < 1e-5
    assert err2.mean() < 1e-4


def test_reduced_precision_recheck_agrees_with_its_fp32_pass(fsb, tiny):
    """Re-checking every Gaussian evaluates the same FP16 record in float
    pairs: its FP64 table agrees with the form's FP32 blend to the FP32 bar
    (up to the rare threshold decisions taken the other way), and every
    decision with a margin above 1e-4 is the same."""
    gdev, _ = _device_form(tiny.gaussians)
    main = _solve(fsb, gdev, tiny, table_dtype="float64", recheck_margin=-1.0)
    full = _solve(fsb, gdev, tiny, table_dtype="float64", recheck_margin=1e30)
    ref = full["table"]
    big = ref >= 1e-6 * ref.max()
    rel = np.abs(main["table"][big] - ref[big]) / ref[big]
    print("re-check vs FP32 pass: entries", int(big.sum()), "beyond 1e-5:",
          int((rel > 1e-5).sum()), "max %.2e" % rel.max(), flush=True)
    assert (rel > 1e-5).mean() < 2e-3
    from oracle.assign import assign_margin
    m = assign_margin(ref, tiny.gamma).T
    decided = m >= 1e-4
    assert np.array_equal(_bits_matrix(main["bits"], tiny.E)[decided],
                          _bits_matrix(full["bits"], tiny.E)[decided])
