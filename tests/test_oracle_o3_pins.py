"""Pins of O3, the library-FFT form of the oracle's double-grid CG (oracle/fftcg.py).

O3 takes the same steps as O2 with scipy FFTs in place of matrix DFTs. It is pinned to O2
(itself pinned to the dense Galerkin oracle O1 and the paper's closed forms): the same
operator on random fields to 1e-12, the same double-grid coefficient, the same bounds at
a tight CG tolerance to 1e-12, in 2D and 3D (up to N = 21), isotropic and anisotropic,
both sides. Beyond the sizes O2 reaches quickly, the laminate's closed forms (harmonic
mean across the layers, arithmetic along them, exact for every N) pin it at a 3D grid of
41^3 (double grid 81^3).
"""
import numpy as np
import pytest

import microstructures as ms
from oracle import fftcg, matfree
from oracle.fourier import freqs

CASES = {
    "aniso2d_N11": lambda: ms.random_anisotropic_2d(5, N=11),
    "rects2d_N21": lambda: ms.random_rectangles_2d(7, N=21),
    "aniso3d_N7": lambda: ms.random_anisotropic_3d(2, N=7),
    "spheres3d_N13": lambda: ms.random_spheres_3d(4, N=13, n_balls=5, phi=0.25, contrast=1000.0),
}


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("side", ["primal", "dual"])
def test_o3_operator_equals_o2(name, side):
    p = CASES[name]()
    o2 = matfree.MatFreeOperator(p, side)
    o3 = fftcg.FFTOperator(p, side, workers=2)
    # the same coefficient: O2 keeps centred grid order, O3 FFT order
    A2 = o2.A_grid if not o3.iso else o2.A_grid[0, 0]
    shift = tuple(range(A2.ndim - p.d, A2.ndim))
    assert rel(np.fft.ifftshift(A2, axes=shift), o3.A_grid) < 1e-13
    rng = np.random.default_rng(3)
    u = rng.normal(size=(p.d,) + tuple(p.N)) + 1j * rng.normal(size=(p.d,) + tuple(p.N))
    for project in (True, False):
        assert rel(o3.apply(u, project), o2.apply(u, project)) < 1e-12


def test_o3_real_field_stays_real():
    p = CASES["spheres3d_N13"]()
    o3 = fftcg.FFTOperator(p, "primal", workers=2)
    g = o3.to_grid(o3.apply(o3.constant_field([0.3, -1.0, 0.5])))
    assert np.abs(g.imag).max() < 1e-13 * np.abs(g.real).max()


@pytest.mark.parametrize("name", ["aniso2d_N11", "rects2d_N21", "aniso3d_N7", "spheres3d_N13"])
def test_o3_bounds_equal_o2(name):
    p = CASES[name]()
    tol = 1e-9 if name == "spheres3d_N13" else 1e-11     # contrast 1000: fewer O2 iterations
    a = fftcg.fft_bounds(p, tol=tol, workers=2)
    b = matfree.matfree_bounds(p, tol=tol)
    for key in ("upper", "lower"):
        assert rel(a[key], b[key]) < 1e-12, (key, rel(a[key], b[key]))


def test_o3_3d_operator_and_energy_at_n21_equal_o2():
    """At N = 21 (double grid 41^3): the operator on a random field and the double-grid energy
    matrix of three fields (the steps CG and the bounds use) equal O2's."""
    p = ms.random_spheres_3d(9, N=21, n_balls=6, phi=0.3, contrast=100.0)
    rng = np.random.default_rng(4)
    for side in ("primal", "dual"):
        o2 = matfree.MatFreeOperator(p, side)
        o3 = fftcg.FFTOperator(p, side, workers=4)
        u = rng.normal(size=(3,) + tuple(p.N)) + 1j * rng.normal(size=(3,) + tuple(p.N))
        assert rel(o3.apply(u), o2.apply(u)) < 1e-12
        fields = [o2.constant_field(np.eye(3)[a]) + 0.1 * o2.apply(o2.constant_field(np.eye(3)[a]))
                  for a in range(3)]
        assert rel(o3.energy_matrix(fields), o2.energy_matrix(fields)) < 1e-12


def test_o3_laminate_closed_forms_3d_n41():
    """A slab inclusion filling the cell in x2 and x3 (layers normal to x1): upper_22 =
    upper_33 = arithmetic mean and lower_11 = harmonic mean, exactly for every N."""
    h, a1 = 0.4, 10.0
    p = ms.make_problem(3, 41, 1.0, 1.0, [ms.box((0.0, 0.0, 0.0), (h, 1.0, 1.0), a1, 3)])
    out = fftcg.fft_bounds(p, tol=1e-12, workers=4)
    arith = (1 - h) + h * a1
    harm = 1.0 / ((1 - h) + h / a1)
    assert abs(out["upper"][1, 1] - arith) < 1e-12 * arith
    assert abs(out["upper"][2, 2] - arith) < 1e-12 * arith
    assert abs(out["lower"][0, 0] - harm) < 1e-12 * harm
    assert out["lower"][0, 0] <= out["upper"][0, 0]
