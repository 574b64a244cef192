"""Bounds from the two energy matrices (Def. upper_lower_bounds, Eq. approx_homog_with_error).

upper = A_bar (primal energies), lower = B_bar^{-1} (inverse of the dual energies),
mean = (upper + lower)/2, D = (upper - lower)/2 (guaranteed error). Oracle; test use only.
"""
from __future__ import annotations

import numpy as np


def assemble_bounds(A_bar: np.ndarray, B_bar: np.ndarray) -> dict:
    lower = np.linalg.inv(B_bar)
    return {"upper": A_bar, "lower": lower, "B_upper": B_bar,
            "mean": 0.5 * (A_bar + lower), "D": 0.5 * (A_bar - lower)}
