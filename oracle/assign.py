"""Assignment step of the oracle (FP64, numpy) -- test infrastructure only.

Paper: FlashSplat (arXiv 2409.08270).
  Sec. 3.2 Eq. 6        P_i = argmax_n A_n^i (binary majority vote).
  Sec. 3.2 "Regularized ILP for Noise Reduction"
                        L1-normalise the pair, add the background bias gamma to
                        the background entry, take the argmax.
  Sec. 3.3 Eq. 7        object t against "others" = sum of every other label.
  Supp. Sec. 6, Listing 1 (multi-instance optimisation)
                        the column sum is taken once; for every object the pair
                        (others, object) is L1-normalised per Gaussian, gamma is
                        added to the "others" row and the argmax gives S[e, :].

Readings where the paper is silent: the L1 normalisation divides by
max(|others| + |object|, 1e-12) (the listing's normalisation with its default
epsilon); an exact tie after the bias goes to index 0 ("not a member"), which
is what an argmax that returns the first maximum does.
"""
from __future__ import annotations

import numpy as np

_EPS = 1e-12


def assign(A: np.ndarray, gamma: float) -> np.ndarray:
    """Segmentation matrix S (bool, [E, N]) from the table A ([N, E], FP64).

    For each object e, in order: others = column_sum - A_e; normalise the pair
    (others, A_e) by its L1 norm; add gamma to the normalised "others"; the
    Gaussian belongs to e iff the object entry is strictly the larger.
    """
    A = np.asarray(A, dtype=np.float64)
    N, E = A.shape
    col_sum = A.sum(axis=1)                      # taken once
    S = np.zeros((E, N), dtype=bool)
    for e in range(E):
        obj = A[:, e]
        others = col_sum - obj
        norm = np.maximum(np.abs(others) + np.abs(obj), _EPS)
        others_n = others / norm + gamma
        obj_n = obj / norm
        S[e] = obj_n > others_n                  # argmax, first index wins ties
    return S


def assign_margin(A: np.ndarray, gamma: float) -> np.ndarray:
    """Relative decision margin per (Gaussian, object), [N, E].

    |(1 - gamma) A_e - (1 + gamma)(sum A - A_e)| / sum A: how far object e's
    normalised, biased decision is from its tie.  +inf where sum A = 0 (the
    decision then depends on gamma's sign only).
    """
    A = np.asarray(A, dtype=np.float64)
    s = A.sum(axis=1, keepdims=True)
    num = np.abs((1.0 - gamma) * A - (1.0 + gamma) * (s - A))
    with np.errstate(divide="ignore", invalid="ignore"):
        m = np.where(s > 0, num / np.where(s > 0, s, 1.0), np.inf)
    return m


def labels_from_membership(S: np.ndarray) -> np.ndarray:
    """Single label per Gaussian: the unique member object, else -1."""
    cnt = S.sum(axis=0)
    lab = np.argmax(S, axis=0).astype(np.int32)
    lab[cnt != 1] = -1
    return lab
