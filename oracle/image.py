"""Pixel-image values the oracle integrates, with the paper's optional smoothing
(oracle; TEST INFRASTRUCTURE ONLY, like the rest of this package).

Sec. 7.3 replaces the grid values of the image's characteristic function f by a local
average: 4/16 of the pixel itself, 2/16 of each of its four edge neighbours and 1/16 of
each of its four corner neighbours (periodic). The paper smooths the primal coefficient;
the dual side then takes the pointwise inverse of the smoothed values.

Written here as a matrix product: with S_P the P x P circulant matrix whose rows hold
1/2 on the diagonal and 1/4 on the two periodic neighbours, the stencil above is
S_{P1} F S_{P2}^T (the outer product of (1, 2, 1)/4 with itself is the 4/2/1 stencil
over 16). Because the weights sum to one, smoothing the conductivity image
a = a_0 + (a_1 - a_0) f equals forming it from the smoothed f, so the image of
conductivities is smoothed directly. Reading for 3D images (the paper gives 2D only):
the same circulant on every axis.
"""
from __future__ import annotations

import numpy as np


def smoothing_matrix(P: int) -> np.ndarray:
    """S_P: (S x)_i = x_i / 2 + (x_{i-1} + x_{i+1}) / 4, indices mod P."""
    S = np.zeros((P, P))
    for i in range(P):
        S[i, i] += 0.5
        S[i, (i - 1) % P] += 0.25
        S[i, (i + 1) % P] += 0.25
    return S


def smoothed_image(b: np.ndarray) -> np.ndarray:
    """The image multiplied by S_{P_a} along every axis a."""
    out = np.asarray(b, dtype=np.float64)
    for a in range(out.ndim):
        S = smoothing_matrix(out.shape[a])
        out = np.moveaxis(np.tensordot(S, out, axes=([1], [a])), 0, a)
    return out


def image_values(problem) -> np.ndarray:
    """The conductivity per pixel the method sees: the raw image, or its smoothing when
    the problem asks for it."""
    b = np.asarray(problem.bitmap, dtype=np.float64)
    return smoothed_image(b) if getattr(problem, "smooth", False) else b
