"""Comparison helpers for GPU-vs-oracle parity tests (no test functions here)."""
from __future__ import annotations

import numpy as np

from oracle.assign import assign, assign_margin

RTOL = 1e-5          # contributions: relative error in FP32 (spec bar)
MARGIN_BAR = 1e-6    # labels: exact where the oracle's relative margin is at least this


def table_errors(gpu: np.ndarray, ora: np.ndarray, risk: np.ndarray, rtol: float = RTOL):
    """Element-wise check |gpu - ora| <= rtol |ora| + atol + risk.

    atol = 1e-11 * max|ora| covers entries far below the table's scale (the
    FP32 rounding of a sum whose terms are ~1e-6 of the largest entry);
    risk is the oracle's bound on how far an entry moves when a decision that
    sits on its threshold (alpha vs 1/255, T vs 1e-4, equal depths) flips.
    Returns (ok mask, relative errors of the entries without risk, summary dict).
    """
    gpu = np.asarray(gpu, dtype=np.float64)
    scale = float(np.abs(ora).max()) if ora.size else 0.0
    atol = 1e-11 * scale
    err = np.abs(gpu - ora)
    ok = err <= rtol * np.abs(ora) + atol + risk * (1 + 1e-3)
    big = (ora >= 1e-6 * scale) & (risk == 0)
    rel = err[big] / ora[big]
    summary = {
        "entries": int(ora.size), "checked_rel": int(big.sum()),
        "max_rel": float(rel.max()) if rel.size else 0.0,
        "mean_rel": float(rel.mean()) if rel.size else 0.0,
        "with_risk": int((risk > 0).sum()), "violations": int((~ok).sum()),
    }
    return ok, rel, summary


def label_check(gpu_bits: np.ndarray, ora_table: np.ndarray, risk: np.ndarray, gamma: float,
                table_rtol: float = RTOL):
    """Compare membership bits with the oracle's assignment.

    A decision is certain to survive the table's error when its relative
    margin exceeds 2*(table_rtol + risk/S); the gap between MARGIN_BAR and that
    window is what an FP64 re-check of near ties closes.  Returns a dict with
    the counts; 'mismatch_outside_window' must be 0.
    """
    E = ora_table.shape[1]
    S_ora = assign(ora_table, gamma)                           # [E, N]
    bits = np.asarray(gpu_bits).astype(np.uint64)
    S_gpu = np.stack([((bits >> np.uint64(e)) & np.uint64(1)).astype(bool) for e in range(E)])
    m = assign_margin(ora_table, gamma).T                      # [E, N]
    s = ora_table.sum(1)
    risk_rel = np.where(s > 0, risk.sum(1) / np.where(s > 0, s, 1), 0)[None, :]
    window = np.maximum(MARGIN_BAR, 2 * (table_rtol + risk_rel) * 1.05)
    mism = S_ora != S_gpu
    return {
        "decisions": int(S_ora.size),
        "mismatch": int(mism.sum()),
        "mismatch_outside_window": int((mism & (m >= window)).sum()),
        "in_window": int((m < window).sum()),
        "below_bar": int((m < MARGIN_BAR).sum()),
        "members_oracle": int(S_ora.sum()),
        "members_gpu": int(S_gpu.sum()),
    }
