"""Fourier-side objects of the method, in float64 / complex128 (oracle; test use only).

Conventions (Sec. 2.2 and Sec. 4):
  * cell Y = prod (-Y_a/2, Y_a/2), |Y| = prod Y_a, frequency vector xi(k) = (k_a / Y_a)_a;
  * u_hat(k) = (1/|Y|) int_Y u(x) exp(-2 pi i xi(k).x) dx   (Eq. FT_def);
  * for odd n, Z_n = {-(n-1)/2, ..., (n-1)/2}, stored in centred order (index k + (n-1)/2).
"""
from __future__ import annotations

import numpy as np
from scipy import special

from microstructures import BALL, BOX, Problem

from .image import image_values


def freqs(n: int) -> np.ndarray:
    """Z_n for odd n, centred order (Eq. index_sets; the reduced and full sets agree)."""
    if n % 2 != 1:
        raise ValueError("odd grid sizes only")
    h = (n - 1) // 2
    return np.arange(-h, h + 1, dtype=np.int64)


def frequency_grid(shape) -> np.ndarray:
    """All k in Z_{shape} as an int array [..., d] (centred order per axis)."""
    axes = [freqs(int(n)) for n in shape]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack(mesh, axis=-1)


def topology_hat_at(inc, n: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Fourier coefficient (Eq. FT_def) of the centred inclusion indicator f at integer n [..., d].

    Box of sides h (Remark "inclusion"): (1/|Y|) prod_a h_a sinc(h_a n_a / Y_a).
    Ball of radius R in 3D: (1/|Y|) 4 pi R^3 j1(q)/q with q = 2 pi R |xi(n)|,
    since (sin q - q cos q)/q^3 = j1(q)/q; the value at q = 0 is the volume.
    Disk of radius R in 2D: (1/|Y|) 2 pi R^2 J1(q)/q, value pi R^2 at q = 0.
    The paper does not print the ball/disk formulas (it cites a thesis); these are
    the standard transforms of the indicator, pinned by brute-force quadrature.
    """
    Y = np.asarray(Y, dtype=np.float64)
    volY = float(np.prod(Y))
    n = np.asarray(n)
    d = n.shape[-1]
    if inc.shape == BOX:
        out = np.ones(n.shape[:-1])
        for a in range(d):
            h = inc.size[a]
            out = out * h * np.sinc(h * n[..., a] / Y[a])   # np.sinc(x) = sin(pi x)/(pi x)
        return out / volY
    R = float(inc.size[0])
    xi = n / Y
    q = 2.0 * np.pi * R * np.sqrt(np.sum(xi * xi, axis=-1))
    out = np.empty(q.shape)
    zero = q == 0.0
    qn = np.where(zero, 1.0, q)
    if d == 3:
        out = 4.0 * np.pi * R ** 3 * special.spherical_jn(1, qn) / qn
        out = np.where(zero, 4.0 / 3.0 * np.pi * R ** 3, out)
    elif d == 2:
        out = 2.0 * np.pi * R ** 2 * special.j1(qn) / qn
        out = np.where(zero, np.pi * R ** 2, out)
    else:
        raise ValueError("d must be 2 or 3")
    return out / volY


def phase_inverse(center, n: np.ndarray, Y) -> np.ndarray:
    """phi_{-n}(x_j) = exp(-2 pi i xi(n).x_j): the shift of an inclusion to centre x_j."""
    xi = n / np.asarray(Y, dtype=np.float64)
    return np.exp(-2j * np.pi * np.sum(xi * np.asarray(center), axis=-1))


def _phase_increments(problem: Problem, side: str):
    """(constant phase, per-inclusion increment tensors) for the primal or dual coefficient.

    Primal (Eq. A_with_inclusions): A = A0 + sum_j f_j (A_j - A0).
    Dual: for non-overlapping inclusions the pointwise inverse is again of that form,
    A^{-1} = A0^{-1} + sum_j f_j (A_j^{-1} - A0^{-1}); the dual problem uses its
    Fourier coefficients (the paper's bilinear form a^{-1}, Eq. bilinear_forms).
    """
    if side == "primal":
        return problem.A0, [inc.A - problem.A0 for inc in problem.inclusions]
    if side == "dual":
        B0 = np.linalg.inv(problem.A0)
        return B0, [np.linalg.inv(inc.A) - B0 for inc in problem.inclusions]
    raise ValueError(side)


def bitmap_hat_at(problem: Problem, n: np.ndarray, side: str = "primal") -> np.ndarray:
    """Fourier coefficient (Eq. FT_def) of a pixel image a(x) (or of 1/a for the dual) at
    integer n [..., d]: every pixel is a box of sides h_a = Y_a/P_a centred at
    c_a = -Y_a/2 + (i_a + 1/2) h_a (Remark "inclusion"), so
      a_hat(n) = sum_i v_i prod_a (1/P_a) sinc(n_a/P_a) exp(-2 pi i n_a c_a / Y_a),
    written as a sum over the pixels (no FFT). Returns a scalar per frequency."""
    n = np.asarray(n, dtype=np.int64)
    img = image_values(problem)
    v = img if side == "primal" else 1.0 / img
    Y = np.asarray(problem.Y, dtype=np.float64)
    factors = []
    for a in range(problem.d):
        P = v.shape[a]
        c = -0.5 * Y[a] + (np.arange(P) + 0.5) * (Y[a] / P)
        na = n[..., a].astype(np.float64)
        E = np.exp(-2j * np.pi * na[..., None] * c / Y[a])                      # [..., P]
        factors.append(E * (np.sinc(na / P) / P)[..., None])
    if problem.d == 2:
        return np.einsum("...i,...j,ij->...", factors[0], factors[1], v)
    return np.einsum("...i,...j,...k,ijk->...", factors[0], factors[1], factors[2], v)


def coefficient_hat_at(problem: Problem, n: np.ndarray, side: str = "primal") -> np.ndarray:
    """A_hat(n) (or the coefficient of A^{-1}) at integer frequencies n [..., d] -> [..., d, d].

    Lemma bounds_for_matrix-inclusion: A_hat(n) = A0 delta_{n0}
    + sum_j (A_j - A0) f_hat_j(n) phi_{-n}(x_j); a pixel image is a sum of pixel boxes
    (bitmap_hat_at) times the identity (the pointwise inverse for the dual).
    """
    n = np.asarray(n, dtype=np.int64)
    d = problem.d
    if problem.bitmap is not None:
        return bitmap_hat_at(problem, n, side)[..., None, None] * np.eye(d)
    C0, incr = _phase_increments(problem, side)
    out = np.zeros(n.shape[:-1] + (d, d), dtype=np.complex128)
    is0 = np.all(n == 0, axis=-1)
    out[is0] += C0
    for inc, dA in zip(problem.inclusions, incr):
        g = topology_hat_at(inc, n, problem.Y) * phase_inverse(inc.center, n, problem.Y)
        out += g[..., None, None] * dA
    return out


def coefficient_hat_grid(problem: Problem, shape, side: str = "primal") -> np.ndarray:
    """A_hat(n) for all n in Z_shape (centred), as [d, d, *shape]."""
    n = frequency_grid(shape)
    A = coefficient_hat_at(problem, n, side)
    return np.moveaxis(np.moveaxis(A, -1, 0), -1, 0)


def projection(shape, Y, side: str) -> np.ndarray:
    """Block symbols Gamma^E(k) = xi xi^T/|xi|^2 or Gamma^J = I - Gamma^E, zero at k = 0.

    Def. projection; on odd grids the fully discrete projections are these symbols
    on Z_N (Def. FD_projections). Returns [d, d, *shape].
    """
    k = frequency_grid(shape).astype(np.float64)
    d = k.shape[-1]
    xi = k / np.asarray(Y, dtype=np.float64)
    nrm2 = np.sum(xi * xi, axis=-1)
    safe = np.where(nrm2 == 0.0, 1.0, nrm2)
    GE = xi[..., :, None] * xi[..., None, :] / safe[..., None, None]
    GE[nrm2 == 0.0] = 0.0
    if side == "primal":
        G = GE
    elif side == "dual":
        G = np.eye(d) - GE
        G[nrm2 == 0.0] = 0.0
    else:
        raise ValueError(side)
    return np.moveaxis(np.moveaxis(G, -1, 0), -1, 0)
