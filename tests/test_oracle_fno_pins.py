"""Pins of the warm-start network reference (oracle/fno.py) against independent forms.

The reference writes the spectral layer as products with DFT basis matrices. Here the same
network is restated with numpy's FFTs: a forward 2D DFT of each channel, the kept modes
(kx in [0, K), ky in [-K, K)), complex channel mixing, and the inverse real 2D DFT of the
half spectrum (numpy's irfft2, which weights kx > 0 twice and takes the real part of kx = 0).
A wrong sign, mode window, weight or normalisation in the bases fails the comparison.
The gradient is checked by central differences.
"""
import math

import numpy as np
import pytest
from scipy.special import erf

torch = pytest.importorskip("torch")
from oracle import fno  # noqa: E402

CFG = dict(N=11, cin=1, width=4, modes=3, layers=2, proj=6, cout=3)


def numpy_forward(cfg, params, x):
    N, W, K, L = cfg["N"], cfg["width"], cfg["modes"], cfg["layers"]
    o = fno.offsets(**cfg)

    def P(name, shape):
        s, n = o[name]
        return params[s:s + n].reshape(shape)

    gelu = lambda z: 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))   # noqa: E731
    ky = np.r_[np.arange(K), np.arange(-K, 0)]                      # storage order of the mixing weights
    v = x @ P("lift_w", (cfg["cin"], W)) + P("lift_b", (W,))        # [B, y, x, W]
    for l in range(L):
        R = P(f"R{l}", (2, 2 * K, K, W, W))
        Rc = R[0] + 1j * R[1]
        X = np.fft.fft2(v, axes=(1, 2))                              # [B, ky, kx, W]
        Xk = X[:, ky % N][:, :, :K]                                  # [B, 2K, K, W]
        Y = np.einsum("bqkw,qkwv->bqkv", Xk, Rc)
        half = np.zeros((v.shape[0], N, N // 2 + 1, W), dtype=complex)
        half[:, ky % N, :K] = Y
        s = np.fft.irfft2(half, s=(N, N), axes=(1, 2))
        z = s + v @ P(f"W{l}", (W, W)) + P(f"b{l}", (W,))
        v = gelu(z) if l + 1 < L else z
    h = gelu(v @ P("p1_w", (W, cfg["proj"])) + P("p1_b", (cfg["proj"],)))
    return h @ P("p2_w", (cfg["proj"], cfg["cout"])) + P("p2_b", (cfg["cout"],))


def test_reference_network_equals_fft_form():
    rng = np.random.default_rng(5)
    n = fno.offsets(**CFG)["total"]
    params = rng.normal(size=n) * 0.3
    x = rng.normal(size=(2, CFG["N"], CFG["N"], CFG["cin"]))
    ref = fno.forward(CFG, torch.from_numpy(params), torch.from_numpy(x)).numpy()
    alt = numpy_forward(CFG, params, x)
    assert np.abs(ref - alt).max() < 1e-12 * max(1.0, np.abs(alt).max())


def test_reference_gradient_central_differences():
    rng = np.random.default_rng(6)
    n = fno.offsets(**CFG)["total"]
    params = torch.from_numpy(rng.normal(size=n) * 0.3)
    x = torch.from_numpy(rng.normal(size=(2, CFG["N"], CFG["N"], CFG["cin"])))
    t = torch.from_numpy(rng.normal(size=(2, CFG["N"], CFG["N"], CFG["cout"])))
    loss, grad, _ = fno.loss_and_grad(CFG, params, x, t)

    def L(p):
        return float(torch.mean((fno.forward(CFG, p, x) - t) ** 2))

    assert abs(L(params) - loss) < 1e-14 * max(1.0, loss)
    for k in range(4):
        d = torch.from_numpy(rng.normal(size=n))
        h = 1e-6
        fd = (L(params + h * d) - L(params - h * d)) / (2 * h)
        assert abs(fd - float(grad @ d)) < 1e-6 * max(1.0, abs(fd)), k


CFG3 = dict(N=7, cin=1, width=3, modes=2, layers=2, proj=5, cout=4, d=3)


def numpy_forward_3d(cfg, params, x):
    """The 3D network with numpy's FFTs: fftn over (z, y, x), the kept modes kz, ky in
    [-K, K), kx in [0, K), complex mixing, irfftn of the half spectrum."""
    N, W, K, L = cfg["N"], cfg["width"], cfg["modes"], cfg["layers"]
    o = fno.offsets(**cfg)

    def P(name, shape):
        s, n = o[name]
        return params[s:s + n].reshape(shape)

    gelu = lambda z: 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))   # noqa: E731
    kq = np.r_[np.arange(K), np.arange(-K, 0)] % N
    B = x.shape[0]
    sel = np.ix_(np.arange(B), kq, kq, np.arange(K))
    v = x @ P("lift_w", (cfg["cin"], W)) + P("lift_b", (W,))        # [B, z, y, x, W]
    for l in range(L):
        R = P(f"R{l}", (2, 2 * K, 2 * K, K, W, W))
        Rc = R[0] + 1j * R[1]
        X = np.fft.fftn(v, axes=(1, 2, 3))
        Y = np.einsum("bpqkw,pqkwv->bpqkv", X[sel], Rc)
        half = np.zeros((B, N, N, N // 2 + 1, W), dtype=complex)
        half[sel] = Y
        s = np.fft.irfftn(half, s=(N, N, N), axes=(1, 2, 3))
        z = s + v @ P(f"W{l}", (W, W)) + P(f"b{l}", (W,))
        v = gelu(z) if l + 1 < L else z
    h = gelu(v @ P("p1_w", (W, cfg["proj"])) + P("p1_b", (cfg["proj"],)))
    return h @ P("p2_w", (cfg["proj"], cfg["cout"])) + P("p2_b", (cfg["cout"],))


def test_reference_network_3d_equals_fft_form():
    rng = np.random.default_rng(7)
    n = fno.offsets(**CFG3)["total"]
    params = rng.normal(size=n) * 0.3
    N = CFG3["N"]
    x = rng.normal(size=(2, N, N, N, CFG3["cin"]))
    ref = fno.forward(CFG3, torch.from_numpy(params), torch.from_numpy(x)).numpy()
    alt = numpy_forward_3d(CFG3, params, x)
    assert np.abs(ref - alt).max() < 1e-12 * max(1.0, np.abs(alt).max())


def test_reference_network_3d_shift_equivariance():
    """Every layer commutes with periodic shifts of the grid (DFT-diagonal spectral path,
    pointwise rest): a rolled input gives the rolled output."""
    rng = np.random.default_rng(8)
    n = fno.offsets(**CFG3)["total"]
    params = torch.from_numpy(rng.normal(size=n) * 0.3)
    N = CFG3["N"]
    x = torch.from_numpy(rng.normal(size=(1, N, N, N, CFG3["cin"])))
    out = fno.forward(CFG3, params, x)
    sh = (2, 5, 3)
    rolled = fno.forward(CFG3, params, torch.roll(x, sh, dims=(1, 2, 3)))
    assert (rolled - torch.roll(out, sh, dims=(1, 2, 3))).abs().max() < 1e-12


def test_reference_gradient_3d_central_differences():
    rng = np.random.default_rng(9)
    n = fno.offsets(**CFG3)["total"]
    N = CFG3["N"]
    params = torch.from_numpy(rng.normal(size=n) * 0.3)
    x = torch.from_numpy(rng.normal(size=(2, N, N, N, CFG3["cin"])))
    t = torch.from_numpy(rng.normal(size=(2, N, N, N, CFG3["cout"])))
    loss, grad, _ = fno.loss_and_grad(CFG3, params, x, t)

    def L(p):
        return float(torch.mean((fno.forward(CFG3, p, x) - t) ** 2))

    for k in range(3):
        dvec = torch.from_numpy(rng.normal(size=n))
        h = 1e-6
        fd = (L(params + h * dvec) - L(params - h * dvec)) / (2 * h)
        assert abs(fd - float(grad @ dvec)) < 1e-6 * max(1.0, abs(fd)), k
