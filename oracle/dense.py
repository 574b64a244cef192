"""O1: the Galerkin bounds written out as their definition (oracle; test use only).

For odd N the upper bound is (Def. upper_lower_bounds with the Galerkin fields)
    A_up[a, b] = a(e_b + e^(b), e_a + e^(a)),
    e^(a) = argmin_{e in E_N} a(e_a + e, e_a + e),
where E_N holds the trigonometric polynomials on Z_N whose Fourier coefficients lie
in span xi(k) (zero mean), and a(u, v) = (A u, v)_{L^2} is integrated exactly. In the
Fourier basis a(u, v) = v_hat^H K u_hat with the dense block matrix
    K[(l, a), (k, b)] = A_hat_ab(l - k),   l, k in Z_N        (Lemma Ga_full),
and the constraint is u_hat = P u_hat with P = blockdiag Gamma^E(k). The minimiser
solves  P K P x = -P K E0  on range(P); adding (I - P) makes the matrix regular
without changing the solution on range(P). The dual side is the same with the
coefficient of A^{-1} and Gamma^J (Eq. D_homog_form), giving B_up; lower = B_up^{-1}.
Everything stays in the Fourier basis: no DFT is needed.
"""
from __future__ import annotations

import numpy as np

from microstructures import Problem

from .bounds import assemble_bounds
from .fourier import coefficient_hat_at, frequency_grid, projection


def _galerkin_matrix(problem: Problem, side: str) -> np.ndarray:
    N = tuple(int(n) for n in problem.N)
    d = problem.d
    k = frequency_grid(N).reshape(-1, d)                 # all k in Z_N
    diff = k[:, None, :] - k[None, :, :]                  # l - k, inside Z_{2N-1}
    Ahat = coefficient_hat_at(problem, diff, side)        # [nk, nk, d, d]
    nk = k.shape[0]
    K = np.transpose(Ahat, (0, 2, 1, 3)).reshape(nk * d, nk * d)
    return K


def _projector(problem: Problem, side: str) -> np.ndarray:
    N = tuple(int(n) for n in problem.N)
    d = problem.d
    G = projection(N, problem.Y, side)                    # [d, d, *N]
    G = np.moveaxis(np.moveaxis(G, 0, -1), 0, -1).reshape(-1, d, d)   # [nk, a, b]
    nk = G.shape[0]
    P = np.zeros((nk, d, nk, d))
    idx = np.arange(nk)
    P[idx, :, idx, :] = G
    return P.reshape(nk * d, nk * d)


def dense_fields(problem: Problem, side: str):
    """Exact Galerkin minimisers x^(a) (columns, Fourier coefficients on Z_N) and K."""
    K = _galerkin_matrix(problem, side)
    P = _projector(problem, side)
    d = problem.d
    nkd = K.shape[0]
    k = frequency_grid(tuple(int(n) for n in problem.N)).reshape(-1, d)
    k0 = int(np.flatnonzero(np.all(k == 0, axis=1))[0])
    E0 = np.zeros((nkd, d), dtype=np.complex128)
    for a in range(d):
        E0[k0 * d + a, a] = 1.0
    lhs = P @ K @ P + (np.eye(nkd) - P)
    rhs = -(P @ (K @ E0))
    X = np.linalg.solve(lhs, rhs)
    return X, E0, K


def dense_energy_matrix(problem: Problem, side: str) -> np.ndarray:
    """[a, b] = a(E_b + x^(b), E_a + x^(a)) (primal) or the a^{-1} analogue (dual)."""
    X, E0, K = dense_fields(problem, side)
    U = E0 + X
    W = U.conj().T @ (K @ U)
    return W.real.copy()


def dense_bounds(problem: Problem):
    """O1 bounds: dict(upper, lower, mean, D, B_upper)."""
    return assemble_bounds(dense_energy_matrix(problem, "primal"),
                           dense_energy_matrix(problem, "dual"))
