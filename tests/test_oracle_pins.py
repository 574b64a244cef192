"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test names the passage it follows. They are chosen so that a plausible slip
in the oracle (a dropped term, a sign, a transposed operand, a wrong normalisation,
a wrong dual coefficient or projector) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import microstructures as ms
import oracle
from oracle import fourier, matfree

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def loewner_ge(A, B, tol=1e-12):
    """A >= B in the Loewner order (up to tol * scale)."""
    S = 0.5 * ((A - B) + (A - B).T)
    scale = max(1.0, np.abs(A).max(), np.abs(B).max())
    return np.linalg.eigvalsh(S).min() >= -tol * scale


def voigt_reuss(p):
    """<A> and <A^{-1}>^{-1} from volume fractions (Remark Aeff_spd), geometry only."""
    volY = float(np.prod(p.Y))
    fr = [inc.volume() / volY for inc in p.inclusions]
    mA = p.A0 * (1 - sum(fr)) + sum(f * inc.A for f, inc in zip(fr, p.inclusions))
    mB = np.linalg.inv(p.A0) * (1 - sum(fr)) + sum(
        f * np.linalg.inv(inc.A) for f, inc in zip(fr, p.inclusions))
    return mA, np.linalg.inv(mB)


def A_pointwise(p, pts):
    """A(x) at points [..., d] straight from the geometry (periodic), no Fourier series."""
    out = np.broadcast_to(p.A0, pts.shape[:-1] + (p.d, p.d)).copy()
    for inc in p.inclusions:
        t = pts - inc.center
        t = t - p.Y * np.round(t / p.Y)          # minimum image
        if inc.shape == ms.BOX:
            inside = np.all(np.abs(t) < 0.5 * inc.size, axis=-1)
        else:
            inside = np.sqrt(np.sum(t * t, axis=-1)) < inc.size[0]
        out[inside] = inc.A
    return out


# ---------------------------------------------------------------------------------
# closed-form inclusion coefficients vs brute-force quadrature (Remark "inclusion")
# ---------------------------------------------------------------------------------
def _midpoint_grid(Y, n):
    axes = [(-0.5 + (np.arange(n) + 0.5) / n) * y for y in Y]
    return np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1)


@pytest.mark.parametrize("shape", ["box2", "disk2", "ball3"])
def test_topology_coefficients_match_quadrature(shape):
    if shape == "box2":
        Y = np.array([1.0, 1.3])
        inc = ms.box([0.13, -0.21], [0.37, 0.52], 2.0, 2)
        n_pts = 3000
        ns = np.array([[0, 0], [1, 0], [0, 1], [2, -3], [-5, 4], [7, 1]])
    elif shape == "disk2":
        Y = np.array([1.0, 1.0])
        inc = ms.ball([0.11, -0.07], 0.23, 2.0, 2)
        n_pts = 3000
        ns = np.array([[0, 0], [1, 0], [1, 1], [3, -2], [-4, 5]])
    else:
        Y = np.array([1.0, 1.0, 1.0])
        inc = ms.ball([0.1, -0.15, 0.05], 0.2, 2.0, 3)
        n_pts = 180
        ns = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 1], [2, -1, 3], [-3, 2, 1]])
    x = _midpoint_grid(Y, n_pts)
    t = x - inc.center
    t = t - Y * np.round(t / Y)
    if inc.shape == ms.BOX:
        ind = np.all(np.abs(t) < 0.5 * inc.size, axis=-1)
    else:
        ind = np.sqrt(np.sum(t * t, axis=-1)) < inc.size[0]
    xs = x[ind]
    dV = 1.0 / n_pts ** len(Y)          # cell volume fraction per point (cells of |Y| / n^d)
    for n in ns:
        brute = np.sum(np.exp(-2j * np.pi * xs @ (n / Y))) * dV
        closed = fourier.topology_hat_at(inc, n[None, :], Y)[0] * \
            fourier.phase_inverse(inc.center, n[None, :], Y)[0]
        vol = inc.volume() / np.prod(Y)
        assert abs(brute - closed) < 4e-3 * max(vol, 1e-2), (shape, n, brute, closed)
    # the mean value is exactly the volume fraction
    z = np.zeros((1, len(Y)), dtype=np.int64)
    assert fourier.topology_hat_at(inc, z, Y)[0] == pytest.approx(inc.volume() / np.prod(Y), rel=1e-15)


def test_coefficient_is_hermitian_and_real_on_grid():
    """A real coefficient has A_hat(-n) = conj A_hat(n) (Eq. FT_def); A_M(x) comes out real."""
    p = ms.random_anisotropic_3d(3, N=5)
    n = fourier.frequency_grid((9, 9, 9))
    A = fourier.coefficient_hat_at(p, n, "primal")
    Am = fourier.coefficient_hat_at(p, -n, "primal")
    assert np.abs(A - Am.conj()).max() < 1e-14
    assert np.abs(A - np.swapaxes(A, -1, -2)).max() < 1e-14
    op = matfree.MatFreeOperator(p, "primal")
    assert op.coef_imag_max < 1e-12


def test_double_grid_coefficient_interpolates_truncated_series():
    """A_M(x_j) (Eq. MBA_GA) equals the truncated Fourier series of A evaluated at x_j."""
    p = ms.random_anisotropic_2d(5, N=5)
    op = matfree.MatFreeOperator(p, "primal")
    M = op.M
    rng = np.random.default_rng(0)
    for _ in range(5):
        j = np.array([rng.integers(-(m - 1) // 2, (m - 1) // 2 + 1) for m in M])
        x = j * p.Y / np.array(M)
        n = fourier.frequency_grid(M).reshape(-1, 2)
        Ah = fourier.coefficient_hat_at(p, n, "primal")
        val = np.einsum("kab,k->ab", Ah, np.exp(2j * np.pi * (n / p.Y) @ x)).real
        idx = tuple(int(jj + (m - 1) // 2) for jj, m in zip(j, M))
        assert np.abs(op.A_grid[(slice(None), slice(None)) + idx] - val).max() < 1e-12


# ---------------------------------------------------------------------------------
# projections (Def. projection, Lemma matrix_orthogonality)
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("shape,Y", [((5, 7), (1.0, 1.7)), ((3, 5, 7), (1.0, 0.6, 1.4))])
def test_projections_partition_of_unity(shape, Y):
    GE = fourier.projection(shape, Y, "primal")
    GJ = fourier.projection(shape, Y, "dual")
    d = len(shape)
    GEk = np.moveaxis(np.moveaxis(GE, 0, -1), 0, -1).reshape(-1, d, d)
    GJk = np.moveaxis(np.moveaxis(GJ, 0, -1), 0, -1).reshape(-1, d, d)
    k = fourier.frequency_grid(shape).reshape(-1, d)
    for i in range(k.shape[0]):
        GU = np.eye(d) if np.all(k[i] == 0) else np.zeros((d, d))
        assert np.abs(GU + GEk[i] + GJk[i] - np.eye(d)).max() < 1e-15
        assert np.abs(GEk[i] @ GEk[i] - GEk[i]).max() < 1e-14
        assert np.abs(GEk[i] @ GJk[i]).max() < 1e-14
        if not np.all(k[i] == 0):
            xi = k[i] / np.asarray(Y)
            assert np.abs(GEk[i] @ xi - xi).max() < 1e-14       # curl-free: span xi
            assert np.abs(GJk[i] @ xi).max() < 1e-14            # divergence-free: xi^perp


# ---------------------------------------------------------------------------------
# bounds: exact special cases
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("d", [2, 3])
def test_homogeneous_cell_gives_A0(d):
    """No inclusion: b = 0, the minimisers vanish, both bounds equal A0 (Def. homog_problem)."""
    rng = np.random.default_rng(d)
    Q, _ = np.linalg.qr(rng.normal(size=(d, d)))
    A0 = Q @ np.diag(10.0 ** rng.uniform(-1, 1, d)) @ Q.T
    p = ms.homogeneous(d, 3 if d == 3 else 5, A0)
    b = oracle.dense_bounds(p)
    assert np.abs(b["upper"] - A0).max() < 1e-13
    assert np.abs(b["lower"] - A0).max() < 1e-13


@pytest.mark.parametrize("maker", [lambda: ms.random_anisotropic_2d(11, N=1),
                                   lambda: ms.random_anisotropic_3d(12, N=1),
                                   lambda: ms.square_inclusion_2d(N=1)])
def test_N1_gives_voigt_and_reuss(maker):
    """E_1 = J_1 = {0}: upper = <A> (Voigt), lower = <A^{-1}>^{-1} (Reuss), Remark Aeff_spd."""
    p = maker()
    vA, rA = voigt_reuss(p)
    b = oracle.dense_bounds(p)
    assert np.abs(b["upper"] - vA).max() < 1e-13 * np.abs(vA).max()
    assert np.abs(b["lower"] - rA).max() < 1e-13 * np.abs(rA).max()


def test_golden_voigt_reuss_square():
    g = json.load(open(os.path.join(GOLDEN, "voigt_reuss_square_2d.json")))
    p = ms.square_inclusion_2d(N=1, side=g["side"], a_matrix=g["a_matrix"], a_incl=g["a_incl"])
    b = oracle.dense_bounds(p)
    assert b["upper"][0, 0] == pytest.approx(g["voigt"], rel=1e-14)
    assert b["lower"][0, 0] == pytest.approx(g["reuss"], rel=1e-14)


@pytest.mark.parametrize("N", [3, 5, 9])
def test_laminate_closed_forms(N):
    """Layers normal to x1: A_up[1,1] = arithmetic mean and lower[0,0] = harmonic mean, exactly.

    With the stripe spanning the cell, sinc(h_2 n_2 / Y_2) = delta_{n_2 0}: A_hat(k)
    vanishes off the k_2 = 0 axis, where Gamma^E(k) e_2 = 0, so the primal minimiser
    for E = e_2 is zero; likewise the dual minimiser for J = e_1 (Gamma^J(k) e_1 = 0 there).
    """
    g = json.load(open(os.path.join(GOLDEN, "laminate_2d.json")))
    p = ms.laminate_2d(N, width=g["width"], a_matrix=g["a_matrix"], a_incl=g["a_incl"])
    b = oracle.dense_bounds(p)
    assert b["upper"][1, 1] == pytest.approx(g["arithmetic"], rel=1e-13)
    assert b["lower"][0, 0] == pytest.approx(g["harmonic"], rel=1e-13)
    assert abs(b["upper"][0, 1]) < 1e-13 and abs(b["lower"][0, 1]) < 1e-13
    # the other two entries are strict guaranteed bounds on the exact laminate values
    assert b["upper"][0, 0] > g["harmonic"] and b["lower"][1, 1] < g["arithmetic"]


def test_rotation_identity_2d():
    """2D: J_N = R E_N (R = rotation by 90 degrees), so B_up[A] = R A_up[R^T A^{-1} R] R^T.

    The dual path (Gamma^J, coefficient of A^{-1}) is pinned by the primal path.
    """
    Rm = np.array([[0.0, -1.0], [1.0, 0.0]])
    for seed in range(3):
        p = ms.random_anisotropic_2d(seed, N=7)
        q = ms.make_problem(2, p.N, p.Y, Rm.T @ np.linalg.inv(p.A0) @ Rm, [])
        q.inclusions = [ms.Inclusion(inc.shape, inc.center, inc.size,
                                     Rm.T @ np.linalg.inv(inc.A) @ Rm) for inc in p.inclusions]
        B_up = oracle.dense_energy_matrix(p, "dual")
        A_up_rot = oracle.dense_energy_matrix(q, "primal")
        assert np.abs(B_up - Rm @ A_up_rot @ Rm.T).max() < 1e-12 * np.abs(B_up).max()


# ---------------------------------------------------------------------------------
# structure: ordering, monotonicity, symmetry, invariances
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("maker", [lambda: ms.random_anisotropic_2d(1, N=7),
                                   lambda: ms.random_anisotropic_3d(2, N=5),
                                   lambda: ms.square_inclusion_2d(N=9, a_incl=1000.0),
                                   lambda: ms.random_rectangles_2d(4, N=9)])
def test_ordering_reuss_lower_upper_voigt(maker):
    """<A^-1>^-1 <= lower <= upper <= <A> (Lemma bounds, Remark Aeff_spd)."""
    p = maker()
    vA, rA = voigt_reuss(p)
    b = oracle.dense_bounds(p)
    assert loewner_ge(b["lower"], rA)
    assert loewner_ge(b["upper"], b["lower"])
    assert loewner_ge(vA, b["upper"])
    assert np.abs(b["upper"] - b["upper"].T).max() < 1e-12 * np.abs(b["upper"]).max()


def test_monotone_in_odd_N():
    """Nested spaces E_N in E_M for odd N <= M (Eq. two_grids) with exact integration:
    the upper bound does not increase and the lower bound does not decrease."""
    prev = None
    for N in (1, 3, 5, 7, 9, 11, 13):
        b = oracle.dense_bounds(ms.paper_square_2d(N, 10.0))
        if prev is not None:
            assert loewner_ge(prev["upper"], b["upper"], 1e-13)
            assert loewner_ge(b["lower"], prev["lower"], 1e-13)
        prev = b
    assert np.trace(prev["D"]) < 0.3 * np.trace(oracle.dense_bounds(ms.paper_square_2d(3, 10.0))["D"])


def test_centred_square_is_isotropic():
    b = oracle.dense_bounds(ms.square_inclusion_2d(N=11))
    for key in ("upper", "lower"):
        M = b[key]
        assert abs(M[0, 1]) < 1e-13 and abs(M[0, 0] - M[1, 1]) < 1e-12


def test_translation_and_scaling_invariance():
    """Shifting every inclusion is a phase factor (Lemma bounds_for_matrix-inclusion):
    bounds are unchanged; scaling the cell and all lengths together changes nothing."""
    p = ms.random_anisotropic_2d(7, N=7)
    b0 = oracle.dense_bounds(p)
    shift = np.array([0.31, -0.17])
    q = ms.make_problem(2, p.N, p.Y, p.A0, [ms.Inclusion(i.shape, i.center + shift, i.size, i.A)
                                            for i in p.inclusions])
    b1 = oracle.dense_bounds(q)
    s = 2.7
    r = ms.make_problem(2, p.N, p.Y * s, p.A0, [ms.Inclusion(i.shape, i.center * s, i.size * s, i.A)
                                                for i in p.inclusions])
    b2 = oracle.dense_bounds(r)
    for key in ("upper", "lower"):
        assert np.abs(b0[key] - b1[key]).max() < 1e-12
        assert np.abs(b0[key] - b2[key]).max() < 1e-12


def test_checkerboard_keller_dykhne():
    """Two-phase checkerboard: A_H = sqrt(a1 a2) I (textbook); the bounds must bracket it."""
    a1, a2 = 1.0, 5.0
    b = oracle.dense_bounds(ms.checkerboard_2d(15, a1, a2))
    ex = math.sqrt(a1 * a2)
    for a in range(2):
        assert b["lower"][a, a] <= ex <= b["upper"][a, a]
    assert b["upper"][0, 0] - b["lower"][0, 0] < 0.25


# ---------------------------------------------------------------------------------
# the two oracle paths against each other and against brute force
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("maker", [lambda: ms.random_anisotropic_2d(21, N=7),
                                   lambda: ms.random_anisotropic_3d(22, N=5),
                                   lambda: ms.square_inclusion_2d(N=9),
                                   lambda: ms.random_rectangles_2d(3, N=11)])
def test_dense_equals_double_grid_cg(maker):
    """Lemma double-grid: the double-grid quadrature inside CG (O2) reproduces the exact
    Fourier-convolution Galerkin problem (O1)."""
    p = maker()
    b1 = oracle.dense_bounds(p)
    b2 = oracle.matfree_bounds(p, tol=1e-12)
    for key in ("upper", "lower"):
        assert np.abs(b1[key] - b2[key]).max() < 1e-11 * np.abs(b1[key]).max()


def test_matvec_double_grid_equals_convolution_rows():
    """Operator level: the O2 matvec equals rows of the Lemma Ga_full matrix."""
    p = ms.random_anisotropic_3d(5, N=5)
    rng = np.random.default_rng(1)
    for side in ("primal", "dual"):
        op = matfree.MatFreeOperator(p, side)
        u = rng.normal(size=(3, 5, 5, 5)) + 1j * rng.normal(size=(3, 5, 5, 5))
        v = op.apply(u, project=True)
        ls = np.array([[0, 0, 0], [1, 0, -2], [-2, 2, 1], [2, -1, 0]])
        rows = matfree.matvec_sampled(p, side, u, ls)
        for i, l in enumerate(ls):
            idx = tuple(l + 2)
            assert np.abs(v[(slice(None),) + idx] - rows[i]).max() < 1e-12


def test_bounds_from_brute_force_quadrature_tiny_N():
    """N = 3: assemble the Galerkin matrix by brute-force quadrature of
    (1/|Y|) int A(x) phi_k phi_{-l} dx on a fine grid (A evaluated pointwise from the
    geometry, no Fourier coefficients) and minimise directly; compare with O1."""
    p = ms.random_anisotropic_2d(31, N=3)
    n_pts = 1200
    x = _midpoint_grid(p.Y, n_pts).reshape(-1, 2)
    Ax = A_pointwise(p, x)                      # [P, 2, 2]
    k = fourier.frequency_grid((3, 3)).reshape(-1, 2)
    out = {}
    for side in ("primal", "dual"):
        C = Ax if side == "primal" else np.linalg.inv(Ax)
        ph = np.exp(2j * np.pi * x @ (k / p.Y).T)           # [P, nk] phi_k(x)
        # K[(l,a),(k,b)] = mean_x C_ab(x) phi_k(x) conj(phi_l(x))
        K = np.einsum("pab,pk,pl->lakb", C, ph, ph.conj()) / x.shape[0]
        nk = k.shape[0]
        K = K.reshape(nk * 2, nk * 2)
        G = fourier.projection((3, 3), p.Y, side)
        Gk = np.moveaxis(np.moveaxis(G, 0, -1), 0, -1).reshape(-1, 2, 2)
        P = np.zeros((nk, 2, nk, 2))
        P[np.arange(nk), :, np.arange(nk), :] = Gk
        P = P.reshape(nk * 2, nk * 2)
        E0 = np.zeros((nk * 2, 2), dtype=complex)
        k0 = int(np.flatnonzero(np.all(k == 0, axis=1))[0])
        E0[2 * k0, 0] = E0[2 * k0 + 1, 1] = 1.0
        X = np.linalg.solve(P @ K @ P + np.eye(nk * 2) - P, -(P @ K @ E0))
        U = E0 + X
        out[side] = (U.conj().T @ K @ U).real
    b_ref = oracle.dense_bounds(p)
    assert np.abs(out["primal"] - b_ref["upper"]).max() < 5e-3 * np.abs(b_ref["upper"]).max()
    assert np.abs(out["dual"] - b_ref["B_upper"]).max() < 5e-3 * np.abs(b_ref["B_upper"]).max()


def test_energy_error_identity():
    """Lemma estimates / Galerkin orthogonality: for any delta in E_N,
    a(E + e_N + delta, E + e_N + delta) - a(E + e_N, E + e_N) = a(delta, delta) > 0."""
    p = ms.random_anisotropic_2d(41, N=5)
    op = matfree.MatFreeOperator(p, "primal")
    x, _, _ = matfree.cg_solve(op, [1.0, 0.0], tol=1e-14)
    u = op.constant_field([1.0, 0.0]) + x
    rng = np.random.default_rng(3)
    delta = op.project(rng.normal(size=u.shape) + 1j * rng.normal(size=u.shape))
    # make delta a real field: symmetrise its Fourier coefficients
    delta = 0.5 * (delta + np.conj(delta[:, ::-1, ::-1]))
    delta *= 1e-2
    W = op.energy_matrix([u, u + delta, delta])
    assert W[1, 1] - W[0, 0] == pytest.approx(W[2, 2], rel=1e-9)
    assert W[2, 2] > 0


def test_cg_stops_on_residual_criterion():
    """Remark "Convergence criteria": ||r_i|| <= tol ||E||, x_0 = 0, Krylov iterates stay in E_N."""
    p = ms.square_inclusion_2d(N=9)
    op = matfree.MatFreeOperator(p, "primal")
    x, it, res = matfree.cg_solve(op, [0.0, 1.0], tol=1e-6)
    assert res <= 1e-6 and it > 0
    assert np.abs(op.project(x) - x).max() < 1e-14
    x2, it2, _ = matfree.cg_solve(op, [0.0, 1.0], tol=1e-3)
    assert it2 < it


def _anisotropic_laminate(N, width=0.35):
    """Layers normal to x1 of two SPD anisotropic phases (a stripe spanning the cell height)."""
    A0 = np.array([[2.0, 0.7], [0.7, 1.5]])
    A1 = np.array([[9.0, -2.5], [-2.5, 4.0]])
    return ms.make_problem(2, N, 1.0, A0, [ms.box(0.0, (width, 1.0), A1, 2)]), A0, A1, width


def _laminate_exact(A0, A1, w):
    """Homogenized tensor of a laminate normal to e1 (continuity of e_2 and j_1 across the
    layers): A_11 = <1/A11>^-1, A_12 = <A12/A11>/<1/A11>,
    A_22 = <A22 - A12^2/A11> + <A12/A11>^2/<1/A11>, volume averages with fractions 1-w, w."""
    f = np.array([1.0 - w, w])
    P = [A0, A1]
    m = lambda g: sum(fi * g(Pi) for fi, Pi in zip(f, P))   # noqa: E731
    inv11 = m(lambda A: 1.0 / A[0, 0])
    r = m(lambda A: A[0, 1] / A[0, 0])
    a11 = 1.0 / inv11
    a12 = r / inv11
    a22 = m(lambda A: A[1, 1] - A[0, 1] ** 2 / A[0, 0]) + r * r / inv11
    return np.array([[a11, a12], [a12, a22]])


@pytest.mark.parametrize("N", [3, 5, 9, 15])
def test_element_bounds_contain_exact_anisotropic_laminate(N):
    """Lemma bounds, Eqs. estimate_diagonal and estimate_nondiagonal: the entry intervals
    built from the guaranteed bounds contain every entry of the exact homogenized tensor of an
    anisotropic laminate (closed form independent of the oracle), also at coarse grids where
    the bounds are far apart; the off-diagonal entry is nonzero, so the non-diagonal estimate
    is exercised."""
    p, A0, A1, w = _anisotropic_laminate(N)
    exact = _laminate_exact(A0, A1, w)
    assert abs(exact[0, 1]) > 0.1
    out = oracle.dense_bounds(p)
    lo, hi = out["elem_lo"], out["elem_hi"]
    assert np.all(lo <= exact + 1e-12) and np.all(exact <= hi + 1e-12), (lo, exact, hi)
    # the interval of an off-diagonal entry is the mean -+ (D_11 + D_22), here checked by hand
    D = 0.5 * (out["upper"] - out["lower"])
    assert abs(hi[0, 1] - lo[0, 1] - 2 * (D[0, 0] + D[1, 1])) < 1e-13


@pytest.mark.parametrize("which", ["original", "smoothed"])
def test_mean_and_error_matrix_reproduce_the_papers_printed_values(which):
    """Eq. approx_homog_with_error on the paper's own numbers (Sec. 7.3: Eqs. flyash_orig_bounds
    and flyash_orig_mean, Eqs. flyash_smooth_bounds and flyash_smooth_mean). The oracle forms the
    mean and the guaranteed error matrix D from the printed upper bound and inverse dual bound.
    They equal the printed mean and D to the printing precision: inputs and outputs are rounded
    to 7 decimals, so they are at most 1e-7 apart. A D without the factor 1/2, or a mean of the
    dual energies instead of their inverse, fails."""
    from oracle import bounds
    g = json.load(open(os.path.join(GOLDEN, "paper_flyash_printed_matrices.json")))
    m = g["sets"][which]
    up, lo = np.array(m["upper"]), np.array(m["lower"])
    out = bounds.assemble_bounds(up, np.linalg.inv(lo))
    tol = 10.0 ** -g["decimals"] + 1e-12
    assert np.abs(out["mean"] - np.array(m["mean"])).max() <= tol
    assert np.abs(out["D"] - np.array(m["D"])).max() <= tol
    # which printed matrix is the upper bound: upper - lower is positive definite
    assert np.linalg.eigvalsh(up - lo).min() > 0
