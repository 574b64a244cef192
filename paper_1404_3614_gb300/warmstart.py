"""Learned CG warm start: data from the method, training and evaluation (driver).

The heavy lifting is in the library: the batched solver produces the training fields
(the converged primal and dual correctors of each cell), hom_net_features samples the
cells on their N grid, hom_net_train_step runs forward, backward and Adam on the tensor
cores, hom_net_forward predicts, hom_grid_to_half turns the prediction into half spectra
and the batched solver starts CG from them after projecting with Gamma. Torch only holds
device buffers and picks minibatch indices.

Channels of a field block (8): index side*4 + rhs*2 + component, for side 0 (primal
corrector e^(rhs)) and 1 (dual corrector j^(rhs)), matching the solver's field pools.
"""
from __future__ import annotations

import time

import numpy as np

import microstructures as ms

from . import binding as bd


def torch_cat(parts):
    import torch
    return torch.cat(parts, dim=-1)


class WarmStart:
    def __init__(self, solver, N, width=32, modes=12, layers=4, proj=128, batch=32, seed=0, energy=False):
        import torch
        self.torch = torch
        self.solver = solver
        self.ctx = solver.ctx
        self.N = N
        self.batch = batch
        self.cfg = bd.net_config(N, 1, width, modes, layers, proj, 8)
        self.n_params, self.ws_bytes = bd.hom_net_sizes(self.ctx, self.cfg, batch)
        dev = f"cuda:{solver.device}"
        self.dev = dev
        self.params = torch.empty(self.n_params, dtype=torch.float32, device=dev)
        bd.hom_net_init(self.ctx, self.cfg, seed, self.params.data_ptr())
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.step = 0
        self.energy = energy   # train on sqrt(energy weight) * field, divide it out at inference

    # -- data -------------------------------------------------------------------------
    def features(self, problems):
        """log10 of the phase value on the grid, divided by 3 (phase values span 1e-2..1e3)."""
        torch = self.torch
        out = torch.empty((len(problems), self.N, self.N, 1), dtype=torch.float32, device=self.dev)
        ws = torch.empty(1 << 22, dtype=torch.uint8, device=self.dev)
        chunk = 2048   # inclusion tables of 2048 cells fit the 4 MiB staging area
        for s in range(0, len(problems), chunk):
            part = problems[s:s + chunk]
            bd.hom_net_features(self.ctx, part, out[s:s + len(part)].data_ptr(), ws.data_ptr(), ws.numel())
        out.mul_(1.0 / 3.0)
        return out

    @staticmethod
    def energy_weights(x):
        """sqrt of the pointwise energy weight of each output channel, [n, N, N, 8]: a(x) for
        the primal correctors, 1/a(x) for the dual ones (features are log10(a)/3). The
        energy norm of a field error is the a-weighted L2 norm (a(u, u) = (A u, u), no
        derivative), so a plain MSE on sqrt(w) * field is the energy-norm error of the start."""
        la = x[..., :1] * (3.0 * 2.302585092994046)   # ln a
        primal = (0.5 * la).exp().expand(*x.shape[:-1], 4)
        dual = (-0.5 * la).exp().expand(*x.shape[:-1], 4)
        return torch_cat((primal, dual))

    @staticmethod
    def normalise_targets(y):
        """Scale each (side, rhs) pair of channels of each cell to unit RMS: the network
        learns the shape of each corrector; the solver finds its scale (Rayleigh-Ritz on
        the start direction), so the magnitude need not be predicted."""
        n = y.shape[0]
        blocks = y.view(n, -1, 4, 2)
        rms = blocks.pow(2).mean(dim=(1, 3), keepdim=True).sqrt().clamp_min(1e-12)
        return (blocks / rms).view_as(y)

    def solve(self, problems, precision, tol, x0=None, want_fields=False, max_iter=10000):
        torch = self.torch
        Nh = (self.N + 1) // 2
        cdt = torch.complex64 if precision == bd.HOM_MIXED else torch.complex128
        fields = torch.empty((len(problems), 2, 2, 2, self.N, Nh), dtype=cdt, device=self.dev) if want_fields else None
        out = self.solver.batched(problems, precision=precision, tol=tol, x0=x0, fields=fields, max_iter=max_iter)
        return out, fields

    def fields_to_grid(self, fields):
        torch = self.torch
        n = fields.shape[0]
        grid = torch.empty((n, self.N, self.N, 8), dtype=torch.float32, device=self.dev)
        prec = bd.HOM_FP32 if fields.dtype == torch.complex64 else bd.HOM_FP64
        bd.hom_half_to_grid(self.ctx, self.N, n, 8, fields.data_ptr(), grid.data_ptr(), prec)
        return grid

    def grid_to_fields(self, grid, precision):
        torch = self.torch
        n = grid.shape[0]
        Nh = (self.N + 1) // 2
        cdt = torch.complex64 if precision == bd.HOM_MIXED else torch.complex128
        half = torch.empty((n, 2, 2, 2, self.N, Nh), dtype=cdt, device=self.dev)
        bd.hom_grid_to_half(self.ctx, self.N, n, 8, grid.data_ptr(), half.data_ptr(),
                            bd.HOM_FP32 if precision == bd.HOM_MIXED else bd.HOM_FP64)
        return half

    # -- training / inference -----------------------------------------------------------
    def train(self, x, y, epochs, lr=2e-3, seed=0):
        torch = self.torch
        n = x.shape[0]
        B = self.batch
        g = torch.Generator(device=self.dev).manual_seed(seed)
        loss = torch.zeros(1, device=self.dev)
        history = []
        xb = torch.empty((B,) + tuple(x.shape[1:]), dtype=x.dtype, device=self.dev)
        yb = torch.empty((B,) + tuple(y.shape[1:]), dtype=y.dtype, device=self.dev)
        steps_per_epoch = n // B
        total = epochs * steps_per_epoch
        for ep in range(epochs):
            perm = torch.randperm(n, generator=g, device=self.dev)
            acc = torch.zeros(1, device=self.dev)
            for s in range(steps_per_epoch):
                idx = perm[s * B:(s + 1) * B]
                torch.index_select(x, 0, idx, out=xb)
                torch.index_select(y, 0, idx, out=yb)
                self.step += 1
                frac = self.step / max(total, 1)
                lr_t = lr * (0.5 * (1 + np.cos(np.pi * min(frac, 1.0))) * 0.9 + 0.1)
                bd.hom_net_train_step(self.ctx, self.cfg, self.params.data_ptr(), self.m.data_ptr(),
                                      self.v.data_ptr(), self.grad.data_ptr(), self.step, float(lr_t), B,
                                      xb.data_ptr(), yb.data_ptr(), loss.data_ptr(), self.ws.data_ptr(),
                                      self.ws.numel())
                acc += loss
            history.append(float(acc.item()) / max(steps_per_epoch, 1))
        return history

    def predict(self, x):
        torch = self.torch
        n = x.shape[0]
        B = self.batch
        out = torch.empty((n, self.N, self.N, 8), dtype=torch.float32, device=self.dev)
        xb = torch.zeros((B,) + tuple(x.shape[1:]), dtype=x.dtype, device=self.dev)
        ob = torch.empty((B, self.N, self.N, 8), dtype=torch.float32, device=self.dev)
        for s in range(0, n, B):
            m = min(B, n - s)
            xb[:m].copy_(x[s:s + m])
            bd.hom_net_forward(self.ctx, self.cfg, self.params.data_ptr(), B, xb.data_ptr(), ob.data_ptr(),
                               self.ws.data_ptr(), self.ws.numel())
            out[s:s + m].copy_(ob[:m])
        return out


def train_and_evaluate(N=63, n_train=20000, n_test=1024, epochs=20, batch=32, width=32, modes=12, layers=4,
                       proj=128, seed_train=1000, seed_test=100000, tol=1e-4, precision="mixed", lr=2e-3,
                       gen_tol=1e-6, solver=None, tight_tol=1e-8, energy=False):
    """The learned warm-start workload: random-rectangle cells on an N grid (the batched
    workload's distribution at one N). Returns a dict of measurements."""
    import torch
    import paper_1404_3614_gb300 as hb
    own = solver is None
    if own:
        solver = hb.Bounds(0)
    prec = bd.HOM_MIXED if precision == "mixed" else bd.HOM_FP64
    ws = WarmStart(solver, N, width, modes, layers, proj, batch, seed=seed_train, energy=energy)
    t0 = time.perf_counter()
    train_probs = [ms.random_rectangles_2d(seed_train + i, N=N) for i in range(n_train)]
    test_probs = [ms.random_rectangles_2d(seed_test + i, N=N) for i in range(n_test)]
    t_probs = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, fields = ws.solve(train_probs, prec, gen_tol, want_fields=True)
    x = ws.features(train_probs)
    y = ws.fields_to_grid(fields)
    if energy:
        y = y * WarmStart.energy_weights(x)
    y = WarmStart.normalise_targets(y)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    del fields
    t0 = time.perf_counter()
    hist = ws.train(x, y, epochs, lr=lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    # held-out cells: plain CG from zero vs from the projected prediction
    xt = ws.features(test_probs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    zero, _ = ws.solve(test_probs, prec, tol)
    torch.cuda.synchronize()
    t_zero = time.perf_counter() - t0
    t0 = time.perf_counter()
    pred = ws.predict(xt)
    if energy:
        pred = pred / WarmStart.energy_weights(xt)
    x0 = ws.grid_to_fields(pred, prec)
    warm, _ = ws.solve(test_probs, prec, tol, x0=x0)
    torch.cuda.synchronize()
    t_warm = time.perf_counter() - t0
    # the same comparison at a tight tolerance, in FP64 (the FP32 inner CG of the batched
    # mixed path stops near FP32 accuracy)
    x0_64 = ws.grid_to_fields(pred, bd.HOM_FP64)
    zero_t, _ = ws.solve(test_probs, bd.HOM_FP64, tight_tol)
    warm_t, _ = ws.solve(test_probs, bd.HOM_FP64, tight_tol, x0=x0_64)
    # the network's field alone (no CG iteration) is a conforming field: a valid, looser bound
    net_only, _ = ws.solve(test_probs, prec, tol, x0=x0, max_iter=0)
    it_zero = zero["iters"].reshape(n_test, -1).sum(axis=1)
    it_warm = warm["iters"].reshape(n_test, -1).sum(axis=1)
    rel = []
    ok = True
    gap_net = []
    for i in range(n_test):
        for key in ("upper", "lower"):
            a, b = warm[key][i], zero[key][i]
            rel.append(np.abs(a - b).max() / np.linalg.norm(b))
        S = warm["upper"][i] - warm["lower"][i]
        ok = ok and np.linalg.eigvalsh(0.5 * (S + S.T)).min() >= -1e-9 * np.abs(warm["upper"][i]).max()
        gap_net.append(np.trace(net_only["upper"][i] - net_only["lower"][i]) /
                       max(np.trace(zero["upper"][i] - zero["lower"][i]), 1e-300))
    if own:
        solver.close()
    return {
        "N": N, "n_train": n_train, "n_test": n_test, "epochs": epochs, "batch": batch, "energy_loss": energy,
        "network": {"width": width, "modes": modes, "layers": layers, "proj": proj, "params": ws.n_params},
        "loss_first_epoch": hist[0] if hist else None, "loss_last_epoch": hist[-1] if hist else None,
        "iters_zero_mean": float(it_zero.mean()), "iters_warm_mean": float(it_warm.mean()),
        "iters_saved_frac": float(1.0 - it_warm.mean() / max(it_zero.mean(), 1e-300)),
        "tight_tol": tight_tol,
        "iters_zero_mean_tight": float(zero_t["iters"].reshape(n_test, -1).sum(axis=1).mean()),
        "iters_warm_mean_tight": float(warm_t["iters"].reshape(n_test, -1).sum(axis=1).mean()),
        "time_zero_s": t_zero, "time_warm_s": t_warm, "time_data_s": t_data, "time_train_s": t_train,
        "time_geometry_s": t_probs,
        "max_rel_bound_diff": float(max(rel)), "ordering_ok": bool(ok),
        "net_only_gap_ratio_median": float(np.median(gap_net)),
    }
