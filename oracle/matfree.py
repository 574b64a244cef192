"""O2: the paper's algorithm with the exact double-grid quadrature (oracle; test use only).

Unknowns are Fourier coefficients on Z_N (full, centred, complex128). One matvec
C u = Gamma P_N F_M A_M F_M^{-1} Pad(u), with M = 2N - 1, follows Lemma double-grid:
  1. zero-pad u_hat from Z_N to Z_M and apply the inverse DFT  u(x_j) = sum_n w_M^{jn} u_hat(n)
     (Eq. DFT, no normalisation) on the grid points x_j = sum_a Y_a j_a / M_a e_a, j in Z_M;
  2. multiply by A_M(x_j) = sum_{n in Z_M} w_M^{jn} A_hat(n)       (Eq. MBA_GA);
  3. forward DFT with the 1/|M| factor and keep the frequencies of Z_N (truncation);
  4. apply Gamma^E (primal) or Gamma^J (dual) per frequency  (Def. FD_projections).
The DFTs are plain matrix products, one axis at a time (a library matmul is the only
primitive). CG is textbook Hestenes-Stiefel from x0 = 0 (Sec. 6.1); the stopping test
is ||r_i|| <= tol ||E|| with the Parseval L^2 norm (Remark "Convergence criteria").
The bound energies use the double-grid form a(u, v) = (1/|M|) sum_j v(x_j).A_M(x_j) u(x_j).
"""
from __future__ import annotations

import numpy as np

from microstructures import Problem

from .bounds import assemble_bounds
from .fourier import coefficient_hat_at, coefficient_hat_grid, freqs, projection


def _apply_axis(mat: np.ndarray, arr: np.ndarray, axis: int) -> np.ndarray:
    out = np.tensordot(mat, arr, axes=([1], [axis]))
    return np.moveaxis(out, 0, axis)


def inner(u: np.ndarray, v: np.ndarray) -> float:
    """(u, v)_{L^2} of two real trigonometric polynomials from their Fourier coefficients."""
    return float(np.real(np.vdot(u, v)))


class MatFreeOperator:
    """Double-grid Galerkin operator of one side ("primal": A, Gamma^E; "dual": A^{-1}, Gamma^J)."""

    def __init__(self, problem: Problem, side: str):
        self.problem = problem
        self.side = side
        self.d = problem.d
        self.N = tuple(int(n) for n in problem.N)
        self.M = tuple(2 * n - 1 for n in self.N)
        self.Winv, self.Wfwd, Wsq = [], [], []
        for n, m in zip(self.N, self.M):
            j = freqs(m)
            k = freqs(n)
            self.Winv.append(np.exp(2j * np.pi * np.outer(j, k) / m))           # [M, N]
            self.Wfwd.append(np.exp(-2j * np.pi * np.outer(k, j) / m) / m)      # [N, M]
            Wsq.append(np.exp(2j * np.pi * np.outer(j, j) / m))                # [M, M]
        Ahat = coefficient_hat_grid(problem, self.M, side)                      # [d, d, *M]
        A = Ahat
        for ax in range(self.d):
            A = _apply_axis(Wsq[ax], A, 2 + ax)
        self.coef_imag_max = float(np.max(np.abs(A.imag)))
        self.A_grid = A.real.copy()                                             # [d, d, *M]
        self.G = projection(self.N, problem.Y, side)                           # [d, d, *N]

    # -- transforms --------------------------------------------------------------
    def to_grid(self, u_hat: np.ndarray) -> np.ndarray:
        """Pad Z_N -> Z_M and inverse DFT: values on the double grid, [d, *M]."""
        u = u_hat
        for ax in range(self.d):
            u = _apply_axis(self.Winv[ax], u, 1 + ax)
        return u

    def from_grid(self, w: np.ndarray) -> np.ndarray:
        """Forward DFT with 1/|M| and truncation to Z_N, [d, *N]."""
        v = w
        for ax in range(self.d):
            v = _apply_axis(self.Wfwd[ax], v, 1 + ax)
        return v

    def project(self, v: np.ndarray) -> np.ndarray:
        return np.einsum("ab...,b...->a...", self.G, v)

    def apply(self, u_hat: np.ndarray, project: bool = True) -> np.ndarray:
        w = np.einsum("ab...,b...->a...", self.A_grid, self.to_grid(u_hat))
        v = self.from_grid(w)
        return self.project(v) if project else v

    def constant_field(self, E) -> np.ndarray:
        """The constant field E as Fourier coefficients on Z_N (only k = 0 is nonzero)."""
        u = np.zeros((self.d,) + self.N, dtype=np.complex128)
        centre = tuple((n - 1) // 2 for n in self.N)
        u[(slice(None),) + centre] = np.asarray(E, dtype=np.float64)
        return u

    def energy_matrix(self, fields) -> np.ndarray:
        """W[a, b] = a(u_b, u_a) on the double grid for the list of fields u_a (Lemma double-grid)."""
        grids = [self.to_grid(u) for u in fields]
        Mtot = float(np.prod(self.M))
        n = len(fields)
        W = np.zeros((n, n))
        for b in range(n):
            Au = np.einsum("ab...,b...->a...", self.A_grid, grids[b])
            for a in range(n):
                W[a, b] = float(np.real(np.vdot(grids[a], Au))) / Mtot
        return W


def cg_solve(op: MatFreeOperator, E, tol: float = 1e-10, maxiter: int = 10000, x0=None, history=None):
    """CG on C x = b, b = -Gamma P F A F^{-1} E (Eq. linear_system_primal / _dual, double-grid C).

    Returns (x_hat, iterations, final recursive residual norm / ||E||). A list given as
    `history` receives the relative residual after each iteration (index 0: the start).
    """
    Ef = op.constant_field(E)
    normE = float(np.linalg.norm(np.asarray(E, dtype=np.float64)))
    b = -op.apply(Ef)
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = op.project(np.array(x0, dtype=np.complex128))
        r = b - op.apply(x)
    p = r.copy()
    rr = inner(r, r)
    it = 0
    if history is not None:
        history.append(float(np.sqrt(rr)) / normE)
    while np.sqrt(rr) > tol * normE and it < maxiter:
        q = op.apply(p)
        alpha = rr / inner(p, q)
        x = x + alpha * p
        r = r - alpha * q
        rr_new = inner(r, r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
        if history is not None:
            history.append(float(np.sqrt(rr)) / normE)
    return x, it, float(np.sqrt(rr)) / normE


def side_energy(problem: Problem, side: str, tol: float = 1e-10, maxiter: int = 10000):
    op = MatFreeOperator(problem, side)
    fields, iters = [], []
    for a in range(problem.d):
        E = np.zeros(problem.d)
        E[a] = 1.0
        x, it, _ = cg_solve(op, E, tol, maxiter)
        fields.append(op.constant_field(E) + x)
        iters.append(it)
    return op.energy_matrix(fields), iters


def matfree_bounds(problem: Problem, tol: float = 1e-10, maxiter: int = 10000) -> dict:
    """O2 bounds (CG to ``tol`` on both sides, exact double-grid energies)."""
    A_bar, it_p = side_energy(problem, "primal", tol, maxiter)
    B_bar, it_d = side_energy(problem, "dual", tol, maxiter)
    out = assemble_bounds(A_bar, B_bar)
    out["iters_primal"] = it_p
    out["iters_dual"] = it_d
    return out


def matvec_sampled(problem: Problem, side: str, u_hat: np.ndarray, ls: np.ndarray,
                   project: bool = True) -> np.ndarray:
    """Rows of the Galerkin operator at chosen output frequencies, one by one.

    v_hat(l) = Gamma(l) sum_{k in Z_N} A_hat(l - k) u_hat(k)      (Lemma Ga_full),
    with u_hat [d, *N] centred and ls an int array [m, d]; returns [m, d] complex.
    """
    d = problem.d
    N = tuple(int(n) for n in problem.N)
    ks = np.stack(np.meshgrid(*[freqs(n) for n in N], indexing="ij"), axis=-1).reshape(-1, d)
    U = np.moveaxis(u_hat.reshape((d, -1)), 0, -1)          # [nk, d]
    out = np.zeros((len(ls), d), dtype=np.complex128)
    for i, l in enumerate(np.asarray(ls, dtype=np.int64)):
        Ah = coefficient_hat_at(problem, l[None, :] - ks, side)   # [nk, d, d]
        v = np.einsum("kab,kb->a", Ah, U)
        if project:
            xi = l / problem.Y
            n2 = float(np.dot(xi, xi))
            if n2 == 0.0:
                v = np.zeros(d, dtype=np.complex128)
            else:
                GE = np.outer(xi, xi) / n2
                v = GE @ v if side == "primal" else v - GE @ v
        out[i] = v
    return out
