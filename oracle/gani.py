"""GaNi: the Galerkin method with numerical integration (oracle; test use only).

Def. GaNi and Cor. FD_GaNi: the coefficient is sampled at the grid points
x_N^k = sum_a Y_a k_a / N_a e_a, k in Z_N (Eq. grid_points), and the bilinear form is the
grid quadrature a_N(u, v) = (1/|N|) sum_k A(x_N^k) u(x_N^k) . v(x_N^k) (Lemma FD_of_GaNi);
the dual form uses the pointwise inverse of the sampled matrices. The GaNi homogenized
matrices A_{H,N}, B_{H,N} are the minima over E_N and J_N of these forms. The bounds of the
paper's algorithm (Sec. 6.2, steps (i)-(iii), Eq. GaNi_bounds) evaluate the GaNi minimisers
in the exactly integrated (double-grid) forms of Lemma double-grid.

Sampling reading: a grid point on an inclusion's boundary belongs to the matrix (strict
inequalities, as in Eq. S and Eq. S1 of the numerical examples), with periodic images; a
problem marked `closed` puts it in the inclusion (non-strict, Eq. S2).

Everything is dense and in the Fourier basis (tiny grids): for trigonometric polynomials on
Z_N, a_N(u, v) = v_hat^H K_N u_hat with K_N[(l, a), (k, b)] = A_N_hat_ab(l - k mod N), the
length-N DFT (1/|N| normalisation, Eq. DFT) of the samples.

General (even) grids, Sec. "Fully discrete spaces --- general grids": the grid points are
x_N^k for k in Z_N = {-N/2, ..., N/2 - 1} along an even axis, and the conforming spaces
E_N = G^E_{N,0}[X_N], J_N = G^J_{N,0}[X_N] (Def. FD_proj_E, Def. FD_subspaces_E) carry no
Nyquist frequency: their fields are trigonometric polynomials on the reduced set Z_N^r, which
along an even axis is Z_{N-1}. The GaNi minimisers are searched there (Eq. FD_GaNi with the
0-projections), the grid quadrature still runs over all N grid points, and the double-grid
bounds of the minimisers are the exact Galerkin energies on Z_N^r. On odd grids nothing
changes (Z_N^r = Z_N). Prop. FD_even_problem gives B_{H,N}^{-1} <= A_{H,N} in general.
"""
from __future__ import annotations

import itertools

import numpy as np

from microstructures import BOX, Problem

from .bounds import assemble_bounds
from .dense import _galerkin_matrix, _projector
from .fourier import freqs, frequency_grid
from .image import image_values


def grid_indices(n: int) -> np.ndarray:
    """Z_n in centred order for any n: -(n-1)/2 .. (n-1)/2 (odd), -n/2 .. n/2 - 1 (even)."""
    lo = -(n // 2)
    return np.arange(lo, lo + n, dtype=np.int64)


def reduced_problem(problem: Problem) -> Problem:
    """The same cell on the reduced frequency set Z_N^r: N_a - 1 along even axes."""
    N = np.asarray(problem.N, dtype=np.int64)
    return problem.with_N(np.where(N % 2 == 0, N - 1, N))


def grid_points(problem: Problem) -> np.ndarray:
    """x_N^k for k in Z_N, centred order, shape [*N, d] (Eq. grid_points), odd or even N."""
    N = tuple(int(n) for n in problem.N)
    Y = np.asarray(problem.Y, dtype=np.float64)
    k = np.stack(np.meshgrid(*[grid_indices(n) for n in N], indexing="ij"), axis=-1)
    return k * (Y / np.asarray(N, dtype=np.float64))


def _inside(inc, x: np.ndarray, Y: np.ndarray, closed: bool = False) -> np.ndarray:
    """Membership of the points x [..., d] in the inclusion (periodic images): strict, or
    non-strict when `closed`."""
    dx = x - np.asarray(inc.center, dtype=np.float64)
    dx = dx - Y * np.round(dx / Y)
    lt = np.less_equal if closed else np.less
    if inc.shape == BOX:
        ins = np.ones(x.shape[:-1], dtype=bool)
        for a in range(x.shape[-1]):
            ins &= lt(np.abs(dx[..., a]), 0.5 * inc.size[a])
        return ins
    return lt(np.sqrt(np.sum(dx * dx, axis=-1)), inc.size[0])


def sample_coefficient(problem: Problem, side: str = "primal") -> np.ndarray:
    """A(x_N^k) (primal) or its pointwise inverse (dual), shape [*N, d, d], centred order."""
    d = problem.d
    Y = np.asarray(problem.Y, dtype=np.float64)
    x = grid_points(problem)
    if problem.bitmap is not None:
        # the pixel holding the grid point (pixel centres when N equals the image size)
        b = image_values(problem)
        idx = tuple(np.clip(np.floor((x[..., a] / Y[a] + 0.5) * b.shape[a]).astype(np.int64), 0, b.shape[a] - 1)
                    for a in range(d))
        A = b[idx][..., None, None] * np.eye(d)
        return np.linalg.inv(A) if side == "dual" else A
    A = np.broadcast_to(np.asarray(problem.A0, dtype=np.float64), x.shape[:-1] + (d, d)).copy()
    for inc in problem.inclusions:
        A[_inside(inc, x, Y, bool(getattr(problem, "closed", False)))] = np.asarray(inc.A, dtype=np.float64)
    if side == "dual":
        A = np.linalg.inv(A)
    return A


def gani_matrix(problem: Problem, side: str) -> np.ndarray:
    """K_N[(l, a), (k, b)] = (1/|N|) sum_x A_N(x)_ab exp(-2 pi i (l - k) . x / Y) written out
    as the grid sum over the N grid points (no FFT), l, k in the reduced set Z_N^r."""
    d = problem.d
    Y = np.asarray(problem.Y, dtype=np.float64)
    A = sample_coefficient(problem, side).reshape(-1, d, d)          # [npts, d, d]
    x = grid_points(problem).reshape(-1, d)                          # [npts, d]
    Nr = tuple(int(n) for n in reduced_problem(problem).N)
    k = frequency_grid(Nr).reshape(-1, d)                            # [nk, d]
    phase = np.exp(-2j * np.pi * (k / Y) @ x.T)                      # [nk, npts]: phi_{-k}(x)
    npts = x.shape[0]
    # K[(l, a), (k, b)] = (1/|N|) sum_x conj(phi_l(x)) A_ab(x) phi_k(x)
    K = np.einsum("lx,xab,kx->lakb", phase, A, np.conj(phase)) / npts
    nk = k.shape[0]
    return K.reshape(nk * d, nk * d)


def gani_fields(problem: Problem, side: str):
    """GaNi minimisers X (columns a = 1..d, Fourier coefficients on Z_N), E0 and K_N."""
    K = gani_matrix(problem, side)
    red = reduced_problem(problem)
    P = _projector(red, side)
    d = problem.d
    nkd = K.shape[0]
    k = frequency_grid(tuple(int(n) for n in red.N)).reshape(-1, d)
    k0 = int(np.flatnonzero(np.all(k == 0, axis=1))[0])
    E0 = np.zeros((nkd, d), dtype=np.complex128)
    for a in range(d):
        E0[k0 * d + a, a] = 1.0
    X = np.linalg.solve(P @ K @ P + (np.eye(nkd) - P), -(P @ (K @ E0)))
    return X, E0, K


def gani_bounds(problem: Problem) -> dict:
    """GaNi homogenized matrices and the bounds of the paper's algorithm.

    Returns dict(A_HN, B_HN (GaNi energies), upper, lower, mean, D (Ga energies of the GaNi
    minimisers, Eq. GaNi_bounds))."""
    out = {}
    W = {}
    for side in ("primal", "dual"):
        X, E0, KN = gani_fields(problem, side)
        U = E0 + X
        out["A_HN" if side == "primal" else "B_HN"] = (U.conj().T @ KN @ U).real
        W[side] = (U.conj().T @ _galerkin_matrix(reduced_problem(problem), side) @ U).real
    b = assemble_bounds(W["primal"], W["dual"])
    out.update({key: b[key] for key in ("upper", "lower", "mean", "D")})
    return out
