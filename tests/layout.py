"""Test-side conversions between the oracle's arrays and the library's device layouts.

Oracle: full centred Fourier coefficients [C, N1, N2(, N3)] (axis 1 = x_1) and
double-grid values [d, d, M1, M2(, M3)] at centred grid indices.
Library: half spectrum [C, N3, N2, Nh] (x_1 fastest, k1 >= 0, other axes in FFT
order) and coefficients [q, M3, M2, M1] at grid indices in FFT order.
"""
import numpy as np


def _to_dev_axes(a, d):
    # oracle [C, n1, n2, n3] -> [C, n3, n2, n1]
    return np.transpose(a, (0,) + tuple(range(d, 0, -1)))


def full_to_half(u, d):
    """Oracle full centred [C, *N] -> device half spectrum [C, (N3,) N2, Nh] (complex)."""
    v = np.fft.ifftshift(u, axes=tuple(range(1, d + 1)))      # FFT order on every axis
    v = _to_dev_axes(v, d)
    N1 = u.shape[1]
    Nh = (N1 + 1) // 2
    return np.ascontiguousarray(v[..., :Nh])


def half_to_full(h, d, N1):
    """Device half spectrum -> oracle full centred array, using Hermitian symmetry."""
    Nh = (N1 + 1) // 2
    shp = h.shape[:-1] + (N1,)
    full = np.zeros(shp, dtype=np.complex128)
    full[..., :Nh] = h
    # negative k1: u(-k) = conj u(k): index N1 - k1 holds -k1, other axes negated
    neg = np.conj(h[..., 1:Nh])
    for ax in range(1, d):          # device axes 1..d-1 are k3/k2 (FFT order): negate
        neg = np.roll(np.flip(neg, axis=ax), 1, axis=ax)
    full[..., N1 - np.arange(1, Nh)] = neg
    f = np.transpose(full, (0,) + tuple(range(d, 0, -1)))     # back to [C, n1, n2, n3]
    return np.fft.fftshift(f, axes=tuple(range(1, d + 1)))


def coef_to_dev(A_grid, d, iso):
    """Oracle A_grid [d, d, *M] (centred) -> device [q, (M3,) M2, M1] in FFT order."""
    G = np.fft.ifftshift(A_grid, axes=tuple(range(2, d + 2)))
    G = np.transpose(G, (0, 1) + tuple(range(d + 1, 1, -1)))
    if iso:
        return G[0, 0][None].copy()
    pairs = [(0, 0), (1, 1), (0, 1)] if d == 2 else [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    return np.stack([G[a, b] for a, b in pairs])


def random_real_field(rng, C, N):
    """Fourier coefficients (full, centred) of a random real trigonometric polynomial."""
    x = rng.normal(size=(C,) + tuple(N))
    u = np.fft.fftn(x, axes=tuple(range(1, len(N) + 1))) / np.prod(N)
    return np.fft.fftshift(u, axes=tuple(range(1, len(N) + 1)))
