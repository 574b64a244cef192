"""Reference of the learned warm-start network in plain PyTorch CPU float64 (test use only).

The same Fourier-layer network as the library's tensor-core implementation, written
directly: truncated DFTs along x (kx in [0, K)) and along y (and z in 3D) (k in [-K, K)),
per-mode complex channel mixing, inverse transforms back to the N grid (half-spectrum
inverse along x with weights 1 and 2 and the 1/N^d factor), 1x1 path, bias, exact (erf)
GELU; lift and two-layer projection. Parameters use the library's flat layout (spectral
weights [re/im][kz][ky][kx][W][W]). Gradients come from autograd; they check the library's
hand-written backward kernels.
"""
from __future__ import annotations

import math

import torch


def offsets(N, cin, width, modes, layers, proj, cout, d=2):
    K1 = 2 * modes
    off = 0
    o = {}

    def take(name, n):
        nonlocal off
        o[name] = (off, n)
        off += n

    take("lift_w", cin * width)
    take("lift_b", width)
    for l in range(layers):
        take(f"R{l}", 2 * K1 ** (d - 1) * modes * width * width)
        take(f"W{l}", width * width)
        take(f"b{l}", width)
    take("p1_w", width * proj)
    take("p1_b", proj)
    take("p2_w", proj * cout)
    take("p2_b", cout)
    o["total"] = off
    return o


def bases(N, modes, d=2):
    K, K1 = modes, 2 * modes
    x = torch.arange(N, dtype=torch.float64)
    kx = torch.arange(K, dtype=torch.float64)
    ky = torch.tensor([i if i < K else i - K1 for i in range(K1)], dtype=torch.float64)
    ax = 2 * math.pi * torch.outer(kx, x) / N                 # [K, N]
    ay = 2 * math.pi * torch.outer(ky, x) / N                 # [K1, N]
    w = torch.where(kx == 0, torch.ones_like(kx), 2.0 * torch.ones_like(kx)) / float(N) ** d
    return {"Fr": torch.cos(ax), "Fi": -torch.sin(ax), "Gc": torch.cos(ay), "Gs": torch.sin(ay),
            "Hc": torch.cos(ay).T, "Hs": torch.sin(ay).T, "Er": (w[:, None] * torch.cos(ax)).T,
            "Ei": (-w[:, None] * torch.sin(ax)).T}


def gelu(x):
    return 0.5 * x * (1.0 + torch.erf(x / math.sqrt(2.0)))


def _dft_along(b_, Xr, Xi, spec):
    """Forward complex DFT along one axis on the kept modes: X e^{-2 pi i k y / N} (spec:
    einsum string with the basis index first)."""
    return (torch.einsum(spec, b_["Gc"], Xr) + torch.einsum(spec, b_["Gs"], Xi),
            torch.einsum(spec, b_["Gc"], Xi) - torch.einsum(spec, b_["Gs"], Xr))


def _idft_along(b_, Yr, Yi, spec):
    """Inverse complex DFT along one axis from the kept modes: sum_k Y e^{+2 pi i k y / N}."""
    return (torch.einsum(spec, b_["Hc"], Yr) - torch.einsum(spec, b_["Hs"], Yi),
            torch.einsum(spec, b_["Hc"], Yi) + torch.einsum(spec, b_["Hs"], Yr))


def spectral(cfg, b_, R, v):
    """The spectral path of one layer, v [B, (z,) y, x, W] -> s of the same shape."""
    d, K, W = cfg.get("d", 2), cfg["modes"], cfg["width"]
    K1 = 2 * K
    B = v.shape[0]
    Rr, Ri = R[0], R[1]
    if d == 2:
        X1r = torch.einsum("kx,byxw->bykw", b_["Fr"], v)
        X1i = torch.einsum("kx,byxw->bykw", b_["Fi"], v)
        Xr, Xi = _dft_along(b_, X1r, X1i, "qy,bykw->bqkw")
    else:
        X1r = torch.einsum("kx,bzyxw->bzykw", b_["Fr"], v)
        X1i = torch.einsum("kx,bzyxw->bzykw", b_["Fi"], v)
        X2r, X2i = _dft_along(b_, X1r, X1i, "qy,bzykw->bzqkw")
        Xr, Xi = _dft_along(b_, X2r, X2i, "pz,bzqkw->bpqkw")
    shape = Xr.shape
    Xr = Xr.reshape(B, -1, W)
    Xi = Xi.reshape(B, -1, W)
    Yr = torch.einsum("bmw,mwv->bmv", Xr, Rr) - torch.einsum("bmw,mwv->bmv", Xi, Ri)
    Yi = torch.einsum("bmw,mwv->bmv", Xr, Ri) + torch.einsum("bmw,mwv->bmv", Xi, Rr)
    Yr = Yr.reshape(shape)
    Yi = Yi.reshape(shape)
    if d == 2:
        Z1r, Z1i = _idft_along(b_, Yr, Yi, "yq,bqkw->bykw")
        return torch.einsum("xk,bykw->byxw", b_["Er"], Z1r) + torch.einsum("xk,bykw->byxw", b_["Ei"], Z1i)
    Z2r, Z2i = _idft_along(b_, Yr, Yi, "zp,bpqkw->bzqkw")
    Z1r, Z1i = _idft_along(b_, Z2r, Z2i, "yq,bzqkw->bzykw")
    return torch.einsum("xk,bzykw->bzyxw", b_["Er"], Z1r) + torch.einsum("xk,bzykw->bzyxw", b_["Ei"], Z1i)


def forward(cfg, params, x):
    """cfg: dict(N, cin, width, modes, layers, proj, cout[, d]); params: 1-D float64;
    x: [B, N, N, cin] (2D) or [B, N, N, N, cin] (3D)."""
    N, W, K, L, d = cfg["N"], cfg["width"], cfg["modes"], cfg["layers"], cfg.get("d", 2)
    K1 = 2 * K
    o = offsets(**cfg)
    b_ = bases(N, K, d)

    def P(name, shape):
        s, n = o[name]
        return params[s:s + n].reshape(shape)

    v = x @ P("lift_w", (cfg["cin"], W)) + P("lift_b", (W,))
    for l in range(L):
        R = P(f"R{l}", (2, K1 ** (d - 1) * K, W, W))
        z = spectral(cfg, b_, R, v) + v @ P(f"W{l}", (W, W)) + P(f"b{l}", (W,))
        v = gelu(z) if l + 1 < L else z
    h = gelu(v @ P("p1_w", (W, cfg["proj"])) + P("p1_b", (cfg["proj"],)))
    return h @ P("p2_w", (cfg["proj"], cfg["cout"])) + P("p2_b", (cfg["cout"],))


def loss_and_grad(cfg, params, x, target):
    p = params.clone().detach().requires_grad_(True)
    out = forward(cfg, p, x)
    loss = torch.mean((out - target) ** 2)
    loss.backward()
    return float(loss.detach()), p.grad.detach(), out.detach()
