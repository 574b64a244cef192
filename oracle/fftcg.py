"""O3: the O2 algorithm with library FFTs (oracle; TEST INFRASTRUCTURE ONLY).

The same steps as O2 (oracle/matfree.py), written with multithreaded library FFTs
(scipy.fft, `workers` threads) instead of matrix DFTs, for grids where the O(M^(d+1))
matrix transforms are too slow (the 3D cell with 16 balls at N = 113, double grid 225^3):
  1. the double-grid coefficient A_M(x_j) = sum_{n in Z_M} w_M^{jn} A_hat(n) (Eq. MBA_GA)
     from the closed-form coefficients A_hat(n) (Lemma bounds_for_matrix-inclusion) by one
     inverse FFT times |M|;
  2. one matvec C u = Gamma P_N F_M A_M F_M^{-1} Pad(u) (Lemma double-grid): zero-pad the
     Fourier coefficients from Z_N to Z_M, inverse FFT times |M| (no normalisation, Eq. DFT),
     pointwise A_M, forward FFT over |M|, keep Z_N, project with Gamma^E or Gamma^J;
  3. CG and the double-grid energies exactly as in O2 (the same cg_solve).
Grid values are kept in FFT order (j = 0..M-1, grid point x = Y j / M, periodic); the
Fourier coefficients of the unknowns in the centred order of O2. A test shows O3 = O2
on grids where both run.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as sfft

from microstructures import Problem

from .bounds import assemble_bounds
from .fourier import coefficient_hat_at, freqs, projection
from .matfree import cg_solve


def default_workers() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def coefficient_slab(problem: Problem, side: str, M, i0: int) -> np.ndarray:
    """A_hat(n) for the frequencies with first index i0 (FFT order) of Z_M: the scalar for
    isotropic problems ([*M[1:]]), else [d, d, *M[1:]] (Lemma bounds_for_matrix-inclusion)."""
    kf = [np.fft.fftfreq(m, 1.0 / m).round().astype(np.int64) for m in M]
    rest = np.stack(np.meshgrid(*kf[1:], indexing="ij"), axis=-1)             # [*M[1:], d-1]
    n = np.concatenate([np.full(rest.shape[:-1] + (1,), kf[0][i0]), rest], axis=-1)
    c = coefficient_hat_at(problem, n, side)                                   # [*M[1:], d, d]
    if problem.is_isotropic():
        return c[..., 0, 0]
    return np.moveaxis(c, (-2, -1), (0, 1))


class FFTOperator:
    """Double-grid Galerkin operator of one side, FFT-based (same interface as O2's). A caller
    that already holds the double-grid coefficient passes it as A_grid (FFT order)."""

    def __init__(self, problem: Problem, side: str, workers: int = None, A_grid: np.ndarray = None):
        self.problem = problem
        self.side = side
        self.d = d = problem.d
        self.workers = workers or default_workers()
        self.N = tuple(int(n) for n in problem.N)
        self.M = tuple(2 * n - 1 for n in self.N)
        self.axes = tuple(range(1, d + 1))
        # FFT-order position of every k in Z_N inside a length-M axis
        self.pos = [np.mod(freqs(n), m) for n, m in zip(self.N, self.M)]
        self.iso = problem.is_isotropic()
        if A_grid is None:
            Ahat = np.zeros(self.M if self.iso else (d, d) + self.M, dtype=np.complex128)
            for i0 in range(self.M[0]):
                if self.iso:
                    Ahat[i0] = coefficient_slab(problem, side, self.M, i0)
                else:
                    Ahat[:, :, i0] = coefficient_slab(problem, side, self.M, i0)
            gaxes = tuple(range(d)) if self.iso else tuple(range(2, d + 2))
            A = sfft.ifftn(Ahat, axes=gaxes, workers=self.workers) * float(np.prod(self.M))
            self.coef_imag_max = float(np.max(np.abs(A.imag)))
            A_grid = A.real.copy()
        self.A_grid = A_grid                    # [*M] (isotropic: A = a I) or [d, d, *M]
        self.G = projection(self.N, problem.Y, side)                           # [d, d, *N]

    def _pad(self, u_hat):
        U = np.zeros((u_hat.shape[0],) + self.M, dtype=np.complex128)
        U[(slice(None),) + np.ix_(*self.pos)] = u_hat
        return U

    def to_grid(self, u_hat: np.ndarray) -> np.ndarray:
        """Pad Z_N -> Z_M and inverse DFT without normalisation: [d, *M] (FFT order)."""
        return sfft.ifftn(self._pad(u_hat), axes=self.axes, workers=self.workers) * float(np.prod(self.M))

    def from_grid(self, w: np.ndarray) -> np.ndarray:
        """Forward DFT with 1/|M| and truncation to Z_N (centred), [d, *N]."""
        V = sfft.fftn(w, axes=self.axes, workers=self.workers) / float(np.prod(self.M))
        return V[(slice(None),) + np.ix_(*self.pos)]

    def coef_times(self, g: np.ndarray) -> np.ndarray:
        if self.iso:
            return self.A_grid[None] * g
        return np.einsum("ab...,b...->a...", self.A_grid, g)

    def project(self, v: np.ndarray) -> np.ndarray:
        return np.einsum("ab...,b...->a...", self.G, v)

    def apply(self, u_hat: np.ndarray, project: bool = True) -> np.ndarray:
        v = self.from_grid(self.coef_times(self.to_grid(u_hat)))
        return self.project(v) if project else v

    def constant_field(self, E) -> np.ndarray:
        u = np.zeros((self.d,) + self.N, dtype=np.complex128)
        centre = tuple((n - 1) // 2 for n in self.N)
        u[(slice(None),) + centre] = np.asarray(E, dtype=np.float64)
        return u

    def energy_matrix(self, fields) -> np.ndarray:
        """W[a, b] = a(u_b, u_a) = (1/|M|) sum_j conj(u_a(x_j)) . A_M(x_j) u_b(x_j)."""
        grids = [self.to_grid(u) for u in fields]
        Mtot = float(np.prod(self.M))
        n = len(fields)
        W = np.zeros((n, n))
        for b in range(n):
            Au = self.coef_times(grids[b])
            for a in range(n):
                W[a, b] = float(np.real(np.vdot(grids[a], Au))) / Mtot
        return W


def fft_side_energy(problem: Problem, side: str, tol: float = 1e-10, maxiter: int = 10000, workers: int = None,
                    log=None):
    op = FFTOperator(problem, side, workers)
    fields, iters, resid, hist = [], [], [], []
    for a in range(problem.d):
        E = np.zeros(problem.d)
        E[a] = 1.0
        h = []
        x, it, res = cg_solve(op, E, tol, maxiter, history=h)
        fields.append(op.constant_field(E) + x)
        iters.append(it)
        resid.append(res)
        hist.append(h)
        if log:
            log(f"{side} rhs {a}: {it} iterations, residual {res:.3e}")
    return op.energy_matrix(fields), iters, resid, hist


def fft_bounds(problem: Problem, tol: float = 1e-10, maxiter: int = 10000, workers: int = None, log=None) -> dict:
    """O3 bounds (CG to ``tol`` on both sides, exact double-grid energies)."""
    A_bar, it_p, r_p, h_p = fft_side_energy(problem, "primal", tol, maxiter, workers, log)
    B_bar, it_d, r_d, h_d = fft_side_energy(problem, "dual", tol, maxiter, workers, log)
    out = assemble_bounds(A_bar, B_bar)
    out.update(iters_primal=it_p, iters_dual=it_d, resid_primal=r_p, resid_dual=r_d, history_primal=h_p,
               history_dual=h_d)
    return out
