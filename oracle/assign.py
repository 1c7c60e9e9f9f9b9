"""Assignment step of the oracle (FP64, numpy) -- test infrastructure only.

Paper: FlashSplat (arXiv 2409.08270).
  Sec. 3.2 Eq. 2-6      the binary problem is an integer linear program whose
                        objective is linear in the labels P_i; its minimiser
                        takes, per Gaussian, the label with the larger
                        accumulated contribution (Eq. 6).
  Sec. 3.2 "Regularized ILP for Noise Reduction"
                        the background entry gets a bias gamma after both
                        entries are L1-normalised per Gaussian.
  Sec. 3.3 Eq. 7        for object e the two entries are A_e and "others",
                        the sum of every other label's contribution.

Written here as one inequality per (object e, Gaussian i).  With S = the
row sum of A (all entries are non-negative, so the L1 norm of the pair
(others, A_e) is S) and the normalisation guarded by epsilon = 1e-12:

    member(e, i)  <=>  A_e / n > (S - A_e) / n + gamma,   n = max(S, 1e-12)
                  <=>  2 A_e - S > gamma * max(S, 1e-12).

For S > 0 this is the biased threshold law A_e > (1 + gamma) / 2 * S, i.e.
(1 - gamma) A_e > (1 + gamma)(S - A_e).  An exact tie is not a member (the
argmax returns the first maximum, "others").  For S = 0 (an unseen Gaussian)
it reads 0 > gamma * 1e-12: a member iff gamma < 0.
"""
from __future__ import annotations

import numpy as np

_EPS = 1e-12


def assign(A: np.ndarray, gamma: float) -> np.ndarray:
    """Segmentation matrix S (bool, [E, N]) from the table A ([N, E], FP64):
    member(e, i) <=> 2 A[i, e] - S_i > gamma * max(S_i, 1e-12)."""
    A = np.asarray(A, dtype=np.float64)
    s = A.sum(axis=1)                                       # S_i, taken once
    lhs = 2.0 * A - s[:, None]
    rhs = gamma * np.maximum(s, _EPS)[:, None]
    return (lhs > rhs).T


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
