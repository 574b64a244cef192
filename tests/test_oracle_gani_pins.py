"""Pins of the GaNi oracle (oracle/gani.py) against what the paper and the mathematics fix.

* Prop. FD_odd_problem: on odd grids the primal and dual GaNi homogenized matrices are
  mutually inverse, A_{H,N} = B_{H,N}^{-1}.
* Eq. GaNi_bounds: the exactly integrated energies of the GaNi minimisers bound the Galerkin
  bounds from outside (the Galerkin minimisers minimise those energies over the same spaces).
* A homogeneous cell gives A0 everywhere; N = 1 gives the sample at the origin and the
  Voigt/Reuss bounds.
* Discrete laminate: a coefficient that depends on x1 only gives the harmonic mean of the
  samples along x1 and their arithmetic mean along x2.
* The Fourier-basis GaNi matrix reproduces the grid quadrature of the definition for random
  trigonometric polynomials evaluated at the grid points by direct sums.
"""
import numpy as np
import pytest

import microstructures as ms
from oracle import dense, gani
from oracle.fourier import frequency_grid

CELLS = {
    "square2d_N9": lambda: ms.square_inclusion_2d(N=9),
    "aniso2d_N7": lambda: ms.random_anisotropic_2d(3, N=7),
    "rect2d_N11": lambda: ms.random_rectangles_2d(4, N=11),
    "paper_rho100_N15": lambda: ms.paper_square_2d(15, 100.0),
    "aniso3d_N5": lambda: ms.random_anisotropic_3d(4, N=5),
}


def loewner_ge(A, B, tol=1e-12):
    S = 0.5 * ((A - B) + (A - B).T)
    return np.linalg.eigvalsh(S).min() >= -tol * max(1.0, np.abs(A).max())


@pytest.mark.parametrize("name", list(CELLS))
def test_odd_grid_duality(name):
    out = gani.gani_bounds(CELLS[name]())
    A, B = out["A_HN"], out["B_HN"]
    assert np.abs(A - np.linalg.inv(B)).max() <= 1e-10 * np.abs(A).max()


@pytest.mark.parametrize("name", list(CELLS))
def test_gani_field_bounds_enclose_galerkin_bounds(name):
    p = CELLS[name]()
    g = gani.gani_bounds(p)
    ga = dense.dense_bounds(p)
    assert loewner_ge(g["upper"], ga["upper"])
    assert loewner_ge(ga["lower"], g["lower"])
    assert loewner_ge(g["upper"], g["lower"])


def test_homogeneous_and_single_point():
    A0 = np.array([[2.0, 0.3, 0.1], [0.3, 1.5, 0.2], [0.1, 0.2, 1.0]])
    out = gani.gani_bounds(ms.homogeneous(3, 5, A0))
    for key in ("A_HN", "upper", "lower"):
        assert np.abs(out[key] - A0).max() < 1e-13
    assert np.abs(np.linalg.inv(out["B_HN"]) - A0).max() < 1e-13
    p = ms.random_anisotropic_2d(8, N=1)
    out = gani.gani_bounds(p)
    a0 = gani.sample_coefficient(p)[0, 0]
    assert np.abs(out["A_HN"] - a0).max() < 1e-13
    ref = dense.dense_bounds(p)        # N = 1: Voigt / Reuss from the exact integrals
    assert np.abs(out["upper"] - ref["upper"]).max() < 1e-13
    assert np.abs(out["lower"] - ref["lower"]).max() < 1e-13


@pytest.mark.parametrize("N", [5, 9, 15])
def test_discrete_laminate_means(N):
    p = ms.laminate_2d(N, width=0.37, a_incl=7.0)
    a = gani.sample_coefficient(p)[:, 0, 0, 0]             # depends on x1 only
    assert np.allclose(gani.sample_coefficient(p)[..., 0, 0], a[:, None])
    out = gani.gani_bounds(p)
    assert abs(out["A_HN"][0, 0] - 1.0 / np.mean(1.0 / a)) < 1e-12
    assert abs(out["A_HN"][1, 1] - np.mean(a)) < 1e-12
    assert abs(out["A_HN"][0, 1]) < 1e-12


def test_fourier_matrix_is_the_grid_quadrature():
    p = ms.random_anisotropic_2d(5, N=7)
    d = 2
    N = tuple(int(n) for n in p.N)
    Y = np.asarray(p.Y, dtype=np.float64)
    rng = np.random.default_rng(0)
    k = frequency_grid(N).reshape(-1, d)
    x = gani.grid_points(p).reshape(-1, d)
    A = gani.sample_coefficient(p).reshape(-1, d, d)
    K = gani.gani_matrix(p, "primal")
    for _ in range(3):
        uh = rng.normal(size=(k.shape[0], d)) + 1j * rng.normal(size=(k.shape[0], d))
        vh = rng.normal(size=(k.shape[0], d)) + 1j * rng.normal(size=(k.shape[0], d))
        # u(x) = sum_k u_hat(k) exp(2 pi i k.x / Y), one grid point at a time
        u = np.array([sum(uh[j] * np.exp(2j * np.pi * np.dot(k[j] / Y, xx)) for j in range(k.shape[0])) for xx in x])
        v = np.array([sum(vh[j] * np.exp(2j * np.pi * np.dot(k[j] / Y, xx)) for j in range(k.shape[0])) for xx in x])
        quad = sum(np.conj(v[i]) @ A[i] @ u[i] for i in range(x.shape[0])) / x.shape[0]
        four = np.conj(vh.reshape(-1)) @ K @ uh.reshape(-1)
        assert abs(quad - four) < 1e-11 * abs(quad)


# ---- general (even) grids -------------------------------------------------------------
EVEN = {
    "square2d_N8": lambda: ms.square_inclusion_2d(N=9).with_N(8),
    "aniso2d_N6": lambda: ms.random_anisotropic_2d(3, N=7).with_N(6),
    "rect2d_N6x5": lambda: ms.random_rectangles_2d(4, N=11).with_N((6, 5)),
    "paper_rho100_N8": lambda: ms.paper_square_2d(15, 100.0).with_N(8),
    "aniso3d_N4": lambda: ms.random_anisotropic_3d(4, N=5).with_N(4),
    "spheres3d_N4x5x6": lambda: ms.random_spheres_3d(2, N=7, n_balls=6, phi=0.25, contrast=30.0).with_N((4, 5, 6)),
}


def real_space_gani(problem, side, nyquist="zero"):
    """A_{H,N} (primal) or B_{H,N} (dual) from the grid formulation of Eq. FD_GaNi written in
    real space: e in X_N with e = G_{N,0} e and G_{N,0}[A (E + e)] = 0, where G_{N,0} =
    F^-1 G_hat F (numpy FFTs) with G_hat zero at k = 0 and at the Nyquist frequencies
    (Def. FD_proj_E). nyquist="identity" takes G_{N,I} instead (identity at the Nyquist
    frequencies): the enlarged spaces E_N^app, J_N^app of Eq. FD_GaNi_tilde. The dense system
    is assembled by applying the operator to unit vectors; the energy is the grid mean of
    A (E + e) . (E + e)."""
    d = problem.d
    N = tuple(int(n) for n in problem.N)
    Y = np.asarray(problem.Y, dtype=np.float64)
    A = np.fft.ifftshift(gani.sample_coefficient(problem, side), axes=tuple(range(d)))   # [*N, d, d], x_j = Y j / N
    k = np.stack(np.meshgrid(*[np.fft.fftfreq(n) * n for n in N], indexing="ij"), axis=-1)
    xi = k / Y
    n2 = np.sum(xi * xi, axis=-1)
    nyq = np.zeros(N, dtype=bool)
    for a in range(d):
        if N[a] % 2 == 0:
            nyq |= np.isclose(k[..., a], -N[a] / 2)
    keep = (n2 > 0) & ~nyq
    GE = np.where(keep[..., None, None], xi[..., :, None] * xi[..., None, :] / np.where(keep, n2, 1.0)[..., None, None], 0.0)
    G = GE if side == "primal" else np.where(keep[..., None, None], np.eye(d) - GE, 0.0)
    if nyquist == "identity":
        G = np.where(nyq[..., None, None], np.eye(d), G)
    axes = tuple(range(d))

    def proj(v):                                  # v [*N, d] real
        vh = np.fft.fftn(v, axes=axes)
        return np.real(np.fft.ifftn(np.einsum("...ab,...b->...a", G, vh), axes=axes))

    npts = int(np.prod(N))
    n = npts * d

    def op(e):
        e = e.reshape(N + (d,))
        return (proj(np.einsum("...ab,...b->...a", A, proj(e))) + e - proj(e)).reshape(-1)

    L = np.stack([op(np.eye(n)[:, j]) for j in range(n)], axis=1)
    H = np.zeros((d, d))
    U = []
    for b in range(d):
        E = np.zeros(N + (d,))
        E[..., b] = 1.0
        rhs = -proj(np.einsum("...ab,...b->...a", A, E)).reshape(-1)
        U.append(E + np.linalg.solve(L, rhs).reshape(N + (d,)))
    for a in range(d):
        for b in range(d):
            H[a, b] = np.mean(np.einsum("...a,...ab,...b->...", U[a], A, U[b]))
    return H


@pytest.mark.parametrize("name", list(EVEN))
def test_even_grid_gani_equals_real_space_formulation(name):
    p = EVEN[name]()
    out = gani.gani_bounds(p)
    for side, key in (("primal", "A_HN"), ("dual", "B_HN")):
        ref = real_space_gani(p, side)
        assert np.abs(out[key] - ref).max() <= 1e-10 * np.abs(ref).max(), (side, out[key], ref)


@pytest.mark.parametrize("name", ["square2d_N9", "aniso2d_N7", "aniso3d_N5"])
def test_real_space_formulation_on_odd_grids(name):
    """The same real-space construction on odd grids (no Nyquist) gives the odd-grid oracle."""
    p = CELLS[name]()
    out = gani.gani_bounds(p)
    assert np.abs(out["A_HN"] - real_space_gani(p, "primal")).max() <= 1e-10 * np.abs(out["A_HN"]).max()


@pytest.mark.parametrize("name", list(EVEN))
def test_even_grid_duality_inequality_and_enclosure(name):
    """Prop. FD_even_problem: B_{H,N}^{-1} <= A_{H,N}; the GaNi minimisers live in the
    Galerkin spaces of the reduced set Z_N^r = Z_{N-1}, so their double-grid bounds enclose
    the Galerkin bounds on N - 1 (Eq. GaNi_bounds)."""
    p = EVEN[name]()
    out = gani.gani_bounds(p)
    assert loewner_ge(out["A_HN"], np.linalg.inv(out["B_HN"]), 1e-10)
    ga = dense.dense_bounds(gani.reduced_problem(p))
    assert loewner_ge(out["upper"], ga["upper"], 1e-11)
    assert loewner_ge(ga["lower"], out["lower"], 1e-11)
    assert loewner_ge(out["upper"], out["lower"], 1e-11)


def test_even_grid_duality_gap_is_real():
    """On even grids the inequality of Prop. FD_even_problem is strict for a contrasted cell
    (the odd-grid equality does not carry over)."""
    out = gani.gani_bounds(EVEN["paper_rho100_N8"]())
    gap = out["A_HN"] - np.linalg.inv(out["B_HN"])
    assert np.linalg.eigvalsh(0.5 * (gap + gap.T)).max() > 1e-3 * np.abs(out["A_HN"]).max()


def test_even_grid_points_and_homogeneous_cell():
    p = ms.square_inclusion_2d(N=9).with_N((4, 6))
    x = gani.grid_points(p)
    assert np.allclose(x[:, 0, 0], np.array([-2, -1, 0, 1]) / 4.0)
    assert np.allclose(x[0, :, 1], np.array([-3, -2, -1, 0, 1, 2]) / 6.0)
    A0 = np.array([[2.0, 0.3], [0.3, 1.0]])
    hom = ms.make_problem(2, 6, 1.0, A0, [])
    out = gani.gani_bounds(hom)
    for key in ("A_HN", "upper", "lower"):
        assert np.abs(out[key] - A0).max() < 1e-13


def test_closed_and_open_inclusions_on_even_grids():
    """The paper's S1 (|x| < 3/4) and S2 (|x| <= 3/4) cells: on grids whose points avoid the
    interface (N = 4: x in {-1, -1/2, 0, 1/2}) they are the same GaNi problem; for N = 8 the
    points x = +-3/4 lie on it, S2 puts them in the inclusion, so its GaNi homogenized matrix
    is larger (Loewner order: more stiff samples) and both keep B^-1 <= A. The Galerkin bounds
    do not depend on the choice."""
    for rho in (10.0, 1000.0):
        s1, s2 = ms.paper_square_even_2d(4, rho), ms.paper_square_even_2d(4, rho, closed=True)
        a, b = gani.gani_bounds(s1), gani.gani_bounds(s2)
        assert np.abs(a["A_HN"] - b["A_HN"]).max() < 1e-13
        s1, s2 = ms.paper_square_even_2d(8, rho), ms.paper_square_even_2d(8, rho, closed=True)
        assert gani.sample_coefficient(s2)[..., 0, 0].sum() > gani.sample_coefficient(s1)[..., 0, 0].sum()
        a, b = gani.gani_bounds(s1), gani.gani_bounds(s2)
        assert b["A_HN"][0, 0] > a["A_HN"][0, 0] * (1 + 1e-3)
        for o in (a, b):
            assert loewner_ge(o["A_HN"], np.linalg.inv(o["B_HN"]), 1e-10)
        g1, g2 = dense.dense_bounds(s1.with_N(7)), dense.dense_bounds(s2.with_N(7))
        assert np.abs(g1["upper"] - g2["upper"]).max() < 1e-13


@pytest.mark.parametrize("name", ["square2d_N8", "aniso2d_N6", "rect2d_N6x5", "paper_rho100_N8", "aniso3d_N4"])
def test_even_grid_duality_with_the_enlarged_spaces(name):
    """Prop. FD_even_problem (i): on general grids the GaNi matrices are dual to the problems on
    the enlarged spaces E_N^app, J_N^app (projections G_{N,I}, identity at the Nyquist
    frequencies, Eq. FD_GaNi_tilde): A_{H,N} = B~_{H,N}^{-1} and B_{H,N}^{-1} = A~_{H,N}. The
    enlarged problems are computed by the independent real-space construction; A_{H,N} and
    B_{H,N} come from the oracle."""
    p = EVEN[name]()
    out = gani.gani_bounds(p)
    Bt = real_space_gani(p, "dual", nyquist="identity")
    At = real_space_gani(p, "primal", nyquist="identity")
    A, B = out["A_HN"], out["B_HN"]
    assert np.abs(A - np.linalg.inv(Bt)).max() <= 1e-10 * np.abs(A).max()
    assert np.abs(np.linalg.inv(B) - At).max() <= 1e-10 * np.abs(At).max()


@pytest.mark.parametrize("name", ["square2d_N9", "aniso2d_N7", "rect2d_N11", "aniso3d_N5"])
def test_odd_grid_dual_fields_from_the_primal_ones(name):
    """Eq. FD_superposition_odd_A: on odd grids the dual GaNi fields follow from the primal ones
    pointwise, e_b + j^(b) = A_N sum_a E_a (e_a + e^(a)) with E = B_{H,N} e_b. In the Fourier
    basis the grid product with A_N is the GaNi matrix K_N (exact on Z_N), so the dual fields
    of the oracle equal K_N U E column by column."""
    p = CELLS[name]()
    Xp, E0, Kp = gani.gani_fields(p, "primal")
    Xd, _, _ = gani.gani_fields(p, "dual")
    Up, Ud = E0 + Xp, E0 + Xd
    B = (Ud.conj().T @ gani.gani_matrix(p, "dual") @ Ud).real
    J = Kp @ Up @ B                      # column b: A_N sum_a (B e_b)_a (e_a + e^(a))
    assert np.abs(J - Ud).max() <= 1e-10 * np.abs(Ud).max()
