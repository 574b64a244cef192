"""Pins of the oracle's pixel-image coefficient (oracle/fourier.py bitmap_hat_at).

* An image of a pixel-aligned box is the same function as that box inclusion: the bounds
  of the two descriptions agree (2D and 3D).
* A constant image is a homogeneous cell; an image that varies along x1 only is a laminate
  (harmonic mean across, arithmetic along, exactly for every N).
* The pixel sum equals numpy's FFT of the image times the pixel sinc and the centring phase.
* GaNi on the image grid (N = image size) samples the pixel values and keeps the odd-grid
  duality.
"""
import numpy as np
import pytest

import microstructures as ms
from oracle import dense, gani
from oracle.fourier import bitmap_hat_at, frequency_grid


@pytest.mark.parametrize("N", [5, 9, 11])
def test_box_image_equals_box_inclusion(N):
    P, lo, hi = 9, 2, 7
    img = ms.bitmap_problem(ms.box_bitmap(P, lo, hi, 10.0), N=N)
    side = (hi - lo) / P
    inc = ms.make_problem(2, N, 1.0, 1.0, [ms.box((0.0, 0.0), (side, side), 10.0, 2)])
    a, b = dense.dense_bounds(img), dense.dense_bounds(inc)
    for key in ("upper", "lower"):
        assert np.abs(a[key] - b[key]).max() < 1e-12


def test_box_image_equals_box_inclusion_3d():
    img = ms.bitmap_problem(ms.box_bitmap(5, 1, 4, 7.0, d=3), N=5)
    inc = ms.make_problem(3, 5, 1.0, 1.0, [ms.box((0.0, 0.0, 0.0), (0.6, 0.6, 0.6), 7.0, 3)])
    a, b = dense.dense_bounds(img), dense.dense_bounds(inc)
    for key in ("upper", "lower"):
        assert np.abs(a[key] - b[key]).max() < 1e-12


def test_constant_and_laminate_images():
    out = dense.dense_bounds(ms.bitmap_problem(np.full((7, 7), 2.5), N=5))
    assert np.abs(out["upper"] - 2.5 * np.eye(2)).max() < 1e-13
    assert np.abs(out["lower"] - 2.5 * np.eye(2)).max() < 1e-13
    rng = np.random.default_rng(3)
    col = np.exp(rng.uniform(-1, 2, size=9))
    img = np.repeat(col[:, None], 9, axis=1)          # varies along x1 only
    for N in (3, 7, 9):
        out = dense.dense_bounds(ms.bitmap_problem(img, N=N))
        assert abs(out["upper"][1, 1] - col.mean()) < 1e-12
        assert abs(out["lower"][0, 0] - 1.0 / np.mean(1.0 / col)) < 1e-12
        assert abs(out["upper"][0, 1]) < 1e-12 and abs(out["lower"][0, 1]) < 1e-12


def test_pixel_sum_equals_fft():
    rng = np.random.default_rng(4)
    P = 7
    img = rng.uniform(0.5, 3.0, size=(P, P))
    p = ms.bitmap_problem(img, N=P)
    n = frequency_grid((P, P))
    direct = bitmap_hat_at(p, n)
    F = np.fft.fft2(img) / P ** 2                      # sum_i v_i exp(-2 pi i n i / P) / P^2
    idx = np.mod(n, P)
    phase = np.exp(1j * np.pi * (n[..., 0] + n[..., 1]) * (1.0 - 1.0 / P))
    ref = F[idx[..., 0], idx[..., 1]] * phase * np.sinc(n[..., 0] / P) * np.sinc(n[..., 1] / P)
    assert np.abs(direct - ref).max() < 1e-13


def test_gani_on_the_image_grid():
    rng = np.random.default_rng(5)
    img = np.where(rng.uniform(size=(9, 9)) < 0.4, 0.029, 0.49)
    p = ms.bitmap_problem(img)
    s = gani.sample_coefficient(p)[..., 0, 0]
    # centred order: index j <-> k = j - 4 <-> pixel j
    assert np.array_equal(s, img)
    out = gani.gani_bounds(p)
    assert np.abs(out["A_HN"] - np.linalg.inv(out["B_HN"])).max() <= 1e-10 * np.abs(out["A_HN"]).max()
    ga = dense.dense_bounds(p)
    assert np.linalg.eigvalsh(out["upper"] - ga["upper"]).min() >= -1e-12
    assert np.linalg.eigvalsh(ga["lower"] - out["lower"]).min() >= -1e-12


# ----------------------------------------------------------------------------------
# the paper's smoothing of the image (Sec. 7.3), oracle/image.py
# ----------------------------------------------------------------------------------
def stencil_by_loops(img):
    """The Sec. 7.3 local average written out pixel by pixel (periodic): 4/16 the pixel,
    2/16 each edge neighbour, 1/16 each corner neighbour."""
    P1, P2 = img.shape
    out = np.zeros_like(img)
    for i in range(P1):
        for j in range(P2):
            f = lambda a, b: img[(i + a) % P1, (j + b) % P2]
            out[i, j] = (4 * f(0, 0) + 2 * (f(1, 0) + f(-1, 0) + f(0, 1) + f(0, -1))
                         + (f(1, 1) + f(-1, -1) + f(-1, 1) + f(1, -1))) / 16.0
    return out


def test_smoothing_of_one_pixel_gives_the_paper_weights():
    from oracle.image import smoothed_image
    f = np.zeros((7, 6))
    f[3, 2] = 1.0
    g = smoothed_image(f)
    want = np.zeros_like(f)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            want[3 + a, 2 + b] = {0: 4.0, 1: 2.0, 2: 1.0}[abs(a) + abs(b)] / 16.0
    assert np.array_equal(g, want)                    # exact: dyadic weights


def test_smoothing_multiplies_the_dft_by_its_symbol():
    from oracle.image import smoothed_image
    rng = np.random.default_rng(11)
    P1, P2 = 9, 10
    img = rng.uniform(0.1, 2.0, size=(P1, P2))
    k1 = np.arange(P1)[:, None]
    k2 = np.arange(P2)[None, :]
    symbol = (2 + 2 * np.cos(2 * np.pi * k1 / P1)) * (2 + 2 * np.cos(2 * np.pi * k2 / P2)) / 16.0
    assert np.abs(np.fft.fft2(smoothed_image(img)) - np.fft.fft2(img) * symbol).max() < 1e-13 * P1 * P2


def test_smoothing_equals_the_stencil_and_commutes_with_phase_values():
    from oracle.image import smoothed_image
    rng = np.random.default_rng(12)
    chi = (rng.uniform(size=(8, 5)) < 0.45).astype(float)         # characteristic function
    assert np.abs(smoothed_image(chi) - stencil_by_loops(chi)).max() < 1e-15
    a0, a1 = 0.029, 0.49
    # forming the conductivity from the smoothed characteristic function (the paper's order)
    # equals smoothing the conductivity image (the weights sum to one)
    assert np.abs(smoothed_image(a0 + (a1 - a0) * chi) - (a0 + (a1 - a0) * smoothed_image(chi))).max() < 1e-15
    assert abs(smoothed_image(chi).mean() - chi.mean()) < 1e-15
    assert np.array_equal(smoothed_image(np.full((4, 3), 0.3)), np.full((4, 3), 0.3))


def test_smoothing_3d_is_separable_reading():
    from oracle.image import smoothed_image
    f = np.zeros((5, 5, 5))
    f[2, 2, 2] = 1.0
    g = smoothed_image(f)
    w = np.array([0.25, 0.5, 0.25])
    assert np.array_equal(g[1:4, 1:4, 1:4], np.einsum("i,j,k->ijk", w, w, w))
    assert g.sum() == 1.0


def test_smooth_flag_reaches_the_coefficient_and_the_samples():
    """smooth=True gives the same Fourier coefficients, GaNi samples and bounds as the raw
    image replaced by its pixel-by-pixel stencil."""
    rng = np.random.default_rng(13)
    img = np.where(rng.uniform(size=(9, 9)) < 0.4, 0.029, 0.49)
    flag = ms.bitmap_problem(img, smooth=True)
    manual = ms.bitmap_problem(stencil_by_loops(img))
    n = frequency_grid((17, 17))
    for side in ("primal", "dual"):
        assert np.abs(bitmap_hat_at(flag, n, side) - bitmap_hat_at(manual, n, side)).max() < 1e-15
    assert np.abs(gani.sample_coefficient(flag) - gani.sample_coefficient(manual)).max() < 1e-15
    a, b = dense.dense_bounds(flag.with_N(5)), dense.dense_bounds(manual.with_N(5))
    raw = dense.dense_bounds(ms.bitmap_problem(img, N=5))
    for key in ("upper", "lower"):
        assert np.abs(a[key] - b[key]).max() < 1e-13
        assert np.abs(a[key] - raw[key]).max() > 1e-4           # the flag changes the problem
