"""Bounds from the two energy matrices (Def. upper_lower_bounds, Eq. approx_homog_with_error).

upper = A_bar (primal energies), lower = B_bar^{-1} (inverse of the dual energies),
mean = (upper + lower)/2, D = (upper - lower)/2 (guaranteed error). Oracle; test use only.
"""
from __future__ import annotations

import numpy as np


def element_bounds(upper: np.ndarray, lower: np.ndarray):
    """Intervals for the entries of A_H (Lemma bounds): the diagonal between the diagonals of
    the lower and upper bound (Eq. estimate_diagonal); an off-diagonal entry within
    mean_ab -+ (D_aa + D_bb) (Eq. estimate_nondiagonal)."""
    mean = 0.5 * (upper + lower)
    D = 0.5 * (upper - lower)
    d = upper.shape[0]
    lo = np.empty_like(upper)
    hi = np.empty_like(upper)
    for a in range(d):
        for b in range(d):
            if a == b:
                lo[a, b], hi[a, b] = lower[a, a], upper[a, a]
            else:
                r = D[a, a] + D[b, b]
                lo[a, b], hi[a, b] = mean[a, b] - r, mean[a, b] + r
    return lo, hi


def assemble_bounds(A_bar: np.ndarray, B_bar: np.ndarray) -> dict:
    lower = np.linalg.inv(B_bar)
    lo, hi = element_bounds(A_bar, lower)
    return {"upper": A_bar, "lower": lower, "B_upper": B_bar,
            "mean": 0.5 * (A_bar + lower), "D": 0.5 * (A_bar - lower), "elem_lo": lo, "elem_hi": hi}
