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
