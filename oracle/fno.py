"""Reference of the learned warm-start network in plain PyTorch CPU float64 (test use only).

The same Fourier-layer network as the library's tensor-core implementation, written
directly: truncated DFTs along x (kx in [0, K)) and y (ky in [-K, K)), per-mode complex
channel mixing, inverse transforms back to the N grid (half-spectrum inverse along x
with weights 1 and 2 and the 1/N^2 factor), 1x1 path, bias, exact (erf) GELU; lift and
two-layer projection. Parameters use the library's flat layout. Gradients come from
autograd; they check the library's hand-written backward kernels.
"""
from __future__ import annotations

import math

import torch


def offsets(N, cin, width, modes, layers, proj, cout):
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
        take(f"R{l}", 2 * K1 * modes * width * width)
        take(f"W{l}", width * width)
        take(f"b{l}", width)
    take("p1_w", width * proj)
    take("p1_b", proj)
    take("p2_w", proj * cout)
    take("p2_b", cout)
    o["total"] = off
    return o


def bases(N, modes):
    K, K1 = modes, 2 * modes
    x = torch.arange(N, dtype=torch.float64)
    kx = torch.arange(K, dtype=torch.float64)
    ky = torch.tensor([i if i < K else i - K1 for i in range(K1)], dtype=torch.float64)
    ax = 2 * math.pi * torch.outer(kx, x) / N                 # [K, N]
    ay = 2 * math.pi * torch.outer(ky, x) / N                 # [K1, N]
    w = torch.where(kx == 0, torch.ones_like(kx), 2.0 * torch.ones_like(kx)) / (N * N)
    return {"Fr": torch.cos(ax), "Fi": -torch.sin(ax), "Gc": torch.cos(ay), "Gs": torch.sin(ay),
            "Hc": torch.cos(ay).T, "Hs": torch.sin(ay).T, "Er": (w[:, None] * torch.cos(ax)).T,
            "Ei": (-w[:, None] * torch.sin(ax)).T}


def gelu(x):
    return 0.5 * x * (1.0 + torch.erf(x / math.sqrt(2.0)))


def forward(cfg, params, x):
    """cfg: dict(N, cin, width, modes, layers, proj, cout); params: 1-D float64; x: [B, N, N, cin]."""
    N, W, K, L = cfg["N"], cfg["width"], cfg["modes"], cfg["layers"]
    K1 = 2 * K
    o = offsets(**cfg)
    b_ = bases(N, K)

    def P(name, shape):
        s, n = o[name]
        return params[s:s + n].reshape(shape)

    v = x @ P("lift_w", (cfg["cin"], W)) + P("lift_b", (W,))
    for l in range(L):
        R = P(f"R{l}", (2, K1 * K, W, W))
        Rr, Ri = R[0], R[1]
        X1r = torch.einsum("kx,byxw->bykw", b_["Fr"], v)
        X1i = torch.einsum("kx,byxw->bykw", b_["Fi"], v)
        X2r = torch.einsum("qy,bykw->bqkw", b_["Gc"], X1r) + torch.einsum("qy,bykw->bqkw", b_["Gs"], X1i)
        X2i = torch.einsum("qy,bykw->bqkw", b_["Gc"], X1i) - torch.einsum("qy,bykw->bqkw", b_["Gs"], X1r)
        B = x.shape[0]
        X2r = X2r.reshape(B, K1 * K, W)
        X2i = X2i.reshape(B, K1 * K, W)
        Yr = torch.einsum("bmw,mwv->bmv", X2r, Rr) - torch.einsum("bmw,mwv->bmv", X2i, Ri)
        Yi = torch.einsum("bmw,mwv->bmv", X2r, Ri) + torch.einsum("bmw,mwv->bmv", X2i, Rr)
        Yr = Yr.reshape(B, K1, K, W)
        Yi = Yi.reshape(B, K1, K, W)
        Z1r = torch.einsum("yq,bqkw->bykw", b_["Hc"], Yr) - torch.einsum("yq,bqkw->bykw", b_["Hs"], Yi)
        Z1i = torch.einsum("yq,bqkw->bykw", b_["Hc"], Yi) + torch.einsum("yq,bqkw->bykw", b_["Hs"], Yr)
        s = torch.einsum("xk,bykw->byxw", b_["Er"], Z1r) + torch.einsum("xk,bykw->byxw", b_["Ei"], Z1i)
        z = s + v @ P(f"W{l}", (W, W)) + P(f"b{l}", (W,))
        v = gelu(z) if l + 1 < L else z
    h = gelu(v @ P("p1_w", (W, cfg["proj"])) + P("p1_b", (cfg["proj"],)))
    return h @ P("p2_w", (cfg["proj"], cfg["cout"])) + P("p2_b", (cfg["cout"],))


def loss_and_grad(cfg, params, x, target):
    p = params.clone().detach().requires_grad_(True)
    out = forward(cfg, p, x)
    loss = torch.mean((out - target) ** 2)
    loss.backward()
    return float(loss.detach()), p.grad.detach(), out.detach()
