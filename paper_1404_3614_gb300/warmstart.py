"""Learned CG warm start: data from the method, training and evaluation.

The heavy lifting is in the library: the solver produces the training fields (the
converged primal and dual correctors of each cell; the batched solver in 2D, hom_bounds_io
per cell in 3D), hom_net_features samples the cells on their N grid, hom_net_train_step
runs forward, backward and Adam on the tensor cores, hom_net_forward predicts,
hom_grid_to_half turns the prediction into half spectra and the solver starts CG from them
after projecting with Gamma and scaling by Rayleigh-Ritz. Torch only holds device buffers
and picks minibatch indices.

Channels of a field block (2 d^2): index (side * d + rhs) * d + component, for side 0
(primal corrector e^(rhs)) and 1 (dual corrector j^(rhs)), matching the solver's field
layout [side][rhs][comp][(z)][y][kx].
"""
from __future__ import annotations

import time

import numpy as np

import microstructures as ms

from . import binding as bd


class WarmStart:
    def __init__(self, solver, N, width=32, modes=12, layers=4, proj=128, batch=32, seed=0, d=2):
        import torch
        self.torch = torch
        self.solver = solver
        self.ctx = solver.ctx
        self.N = N
        self.d = d
        self.ch = 2 * d * d
        self.grid = (N,) * d
        self.batch = batch
        self.arch = dict(width=width, modes=modes, layers=layers, proj=proj)
        self.cfg = bd.net_config(N, 1, width, modes, layers, proj, self.ch, d)
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

    # -- data -------------------------------------------------------------------------
    def features(self, problems):
        """log10 of the phase value on the grid, divided by 3 (phase values span 1e-2..1e3),
        computed by the library."""
        torch = self.torch
        out = torch.empty((len(problems),) + self.grid + (1,), dtype=torch.float32, device=self.dev)
        ws = torch.empty(1 << 22, dtype=torch.uint8, device=self.dev)
        chunk = 2048   # inclusion tables of 2048 cells fit the 4 MiB staging area
        for s in range(0, len(problems), chunk):
            part = problems[s:s + chunk]
            bd.hom_net_features(self.ctx, part, out[s:s + len(part)].data_ptr(), ws.data_ptr(), ws.numel())
        return out

    def normalise_targets(self, y):
        """Scale each (side, rhs) group of channels of each cell to unit RMS, in place, in the
        library: the network learns the shape of each corrector; the solver finds its scale
        (Rayleigh-Ritz on the start direction), so the magnitude need not be predicted."""
        bd.hom_net_normalise_targets(self.ctx, self.d, self.N, y.shape[0], y.data_ptr())
        return y

    def field_shape(self, n):
        d = self.d
        return (n, 2, d, d) + self.grid[:-1] + ((self.N + 1) // 2,)

    def solve(self, problems, precision, tol, x0=None, want_fields=False, max_iter=10000):
        """2D: one batched launch (complex64 fields in mixed precision)."""
        torch = self.torch
        cdt = torch.complex64 if precision == bd.HOM_MIXED else torch.complex128
        fields = torch.empty(self.field_shape(len(problems)), dtype=cdt, device=self.dev) if want_fields else None
        out = self.solver.batched(problems, precision=precision, tol=tol, x0=x0, fields=fields, max_iter=max_iter)
        return out, fields

    def fields_to_grid(self, fields, out=None):
        torch = self.torch
        n = fields.shape[0]
        grid = out if out is not None else torch.empty((n,) + self.grid + (self.ch,), dtype=torch.float32,
                                                       device=self.dev)
        prec = bd.HOM_FP32 if fields.dtype == torch.complex64 else bd.HOM_FP64
        nws = bd.hom_half_to_grid_workspace_size(self.ctx, self.d, self.N, n, self.ch)
        ws = torch.empty(max(nws, 256), dtype=torch.uint8, device=self.dev)
        bd.hom_half_to_grid(self.ctx, self.d, self.N, n, self.ch, fields.data_ptr(), grid.data_ptr(), prec,
                            ws.data_ptr(), ws.numel())
        return grid

    def grid_to_fields(self, grid, precision):
        """Half spectra of predicted grid fields: complex64 for the 2D batched mixed path,
        complex128 otherwise (hom_bounds_io takes FP64 starts)."""
        torch = self.torch
        n = grid.shape[0]
        c64 = precision == bd.HOM_MIXED and self.d == 2
        half = torch.empty(self.field_shape(n), dtype=torch.complex64 if c64 else torch.complex128, device=self.dev)
        bd.hom_grid_to_half(self.ctx, self.d, self.N, n, self.ch, grid.data_ptr(), half.data_ptr(),
                            bd.HOM_FP32 if c64 else bd.HOM_FP64)
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
            acc = 0.0
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
                acc += float(loss.item())            # the step has synchronised its stream
            history.append(acc / max(steps_per_epoch, 1))
        return history

    def predict(self, x):
        torch = self.torch
        n = x.shape[0]
        B = self.batch
        out = torch.empty((n,) + self.grid + (self.ch,), dtype=torch.float32, device=self.dev)
        xb = torch.zeros((B,) + tuple(x.shape[1:]), dtype=x.dtype, device=self.dev)
        ob = torch.empty((B,) + self.grid + (self.ch,), dtype=torch.float32, device=self.dev)
        for s in range(0, n, B):
            m = min(B, n - s)
            xb[:m].copy_(x[s:s + m])
            bd.hom_net_forward(self.ctx, self.cfg, self.params.data_ptr(), B, xb.data_ptr(), ob.data_ptr(),
                               self.ws.data_ptr(), self.ws.numel())
            out[s:s + m].copy_(ob[:m])
        return out

    def predict_on_grid(self, x, N):
        """The trained network on another grid N (same parameters: the spectral weights
        act on the kept modes, whose coefficients the 1/N^d-normalised transforms make
        grid-independent), one cell at a time. x: [n, (N,) N, N, 1]."""
        torch = self.torch
        a = self.arch
        cfg = bd.net_config(N, 1, a["width"], a["modes"], a["layers"], a["proj"], self.ch, self.d)
        _, nws = bd.hom_net_sizes(self.ctx, cfg, 1)
        if getattr(self, "_ws_grid", None) is None or self._ws_grid.numel() < nws:
            self._ws_grid = torch.empty(nws, dtype=torch.uint8, device=self.dev)
        n = x.shape[0]
        out = torch.empty((n,) + (N,) * self.d + (self.ch,), dtype=torch.float32, device=self.dev)
        for i in range(n):
            xi = x[i:i + 1].contiguous()
            bd.hom_net_forward(self.ctx, cfg, self.params.data_ptr(), 1, xi.data_ptr(), out[i:i + 1].data_ptr(),
                               self._ws_grid.data_ptr(), self._ws_grid.numel())
        return out

    def with_grid(self, N):
        """A view of this network for features / fields on grid N (shares the parameters)."""
        other = object.__new__(WarmStart)
        other.__dict__.update(self.__dict__)
        other.N = N
        other.grid = (N,) * self.d
        other._ws_grid = None
        return other


def train_and_evaluate(N=63, n_train=20000, n_test=1024, epochs=20, batch=32, width=32, modes=12, layers=4,
                       proj=128, seed_train=1000, seed_test=100000, tol=1e-4, precision="mixed", lr=2e-3,
                       gen_tol=1e-6, solver=None, tight_tol=1e-8):
    """The learned warm-start workload: random-rectangle cells on an N grid (the batched
    workload's distribution at one N). Returns a dict of measurements."""
    import torch
    import paper_1404_3614_gb300 as hb
    own = solver is None
    if own:
        solver = hb.Bounds(0)
    prec = bd.HOM_MIXED if precision == "mixed" else bd.HOM_FP64
    ws = WarmStart(solver, N, width, modes, layers, proj, batch, seed=seed_train)
    t0 = time.perf_counter()
    train_probs = [ms.random_rectangles_2d(seed_train + i, N=N) for i in range(n_train)]
    test_probs = [ms.random_rectangles_2d(seed_test + i, N=N) for i in range(n_test)]
    t_probs = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, fields = ws.solve(train_probs, prec, gen_tol, want_fields=True)
    x = ws.features(train_probs)
    y = ws.normalise_targets(ws.fields_to_grid(fields))
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
        "N": N, "n_train": n_train, "n_test": n_test, "epochs": epochs, "batch": batch,
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


def _iters(out):
    return int(np.asarray(out["report"]["iters"]).sum())


def train_and_evaluate_3d(N_train=41, N_eval=113, n_train=1000, n_test=32, eval_seeds=(0,), epochs=30, batch=8,
                          width=24, modes=8, layers=4, proj=64, seed_train=200000, seed_test=300000, tol=1e-4,
                          precision="mixed", lr=2e-3, gen_tol=1e-6, solver=None, chunk=16, tight_tol=None):
    """The 3D learned warm start: random-sphere cells (16 equal balls, volume fraction 0.3,
    contrast 1000), training fields generated by hom_bounds_io at N_train, evaluation on
    held-out cells at N_train and on the cells `eval_seeds` at N_eval (seed 0 at N = 113 is
    the 3D sphere workload), with and without the start. The warm timings include the
    features, the network forward on the evaluation grid and the transform to half
    spectra. With tight_tol, the iterations from zero and from the start are also counted
    at that tolerance (same precision). Returns a dict of measurements."""
    import torch
    import paper_1404_3614_gb300 as hb
    own = solver is None
    if own:
        solver = hb.Bounds(0)
    prec = bd.HOM_MIXED if precision == "mixed" else bd.HOM_FP64
    ws = WarmStart(solver, N_train, width, modes, layers, proj, batch, seed=seed_train, d=3)
    t0 = time.perf_counter()
    train_probs = [ms.random_spheres_3d(seed_train + i, N=N_train) for i in range(n_train)]
    test_probs = [ms.random_spheres_3d(seed_test + i, N=N_train) for i in range(n_test)]
    eval_probs = [ms.random_spheres_3d(s, N=N_eval) for s in eval_seeds]
    t_probs = time.perf_counter() - t0
    # training data: converged FP64 fields of each cell, chunks of `chunk` cells to the grid
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    y = torch.empty((n_train,) + ws.grid + (ws.ch,), dtype=torch.float32, device=ws.dev)
    fb = torch.empty(ws.field_shape(chunk), dtype=torch.complex128, device=ws.dev)
    gen_iters = []
    for s in range(0, n_train, chunk):
        m = min(chunk, n_train - s)
        for i in range(m):
            out = solver(train_probs[s + i], precision=prec, tol=gen_tol, fields=fb[i])
            gen_iters.append(_iters(out))
        ws.fields_to_grid(fb[:m], out=y[s:s + m])
    del fb
    x = ws.features(train_probs)
    y = ws.normalise_targets(y)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    hist = ws.train(x, y, epochs, lr=lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del x, y

    def coarse_start(p, fields_c):
        """Half spectrum of the N_train field fields_c [1, 2, 3, 3, N, N, Nh] on p's grid."""
        x0 = torch.zeros(ws.with_grid(int(p.N[0])).field_shape(1), dtype=torch.complex128, device=ws.dev)
        bd.hom_resample_fields(solver.ctx, 3, (N_train,) * 3, tuple(int(n) for n in p.N), 2 * 9, bd.HOM_FP64,
                               fields_c.data_ptr(), x0.data_ptr())
        return x0

    def compare(cells, wsg, tight=None, coarse=False):
        rows = []
        for p in cells:
            solver(p, precision=prec, tol=tol)                      # warm-up (graphs, tables)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            zero = solver(p, precision=prec, tol=tol)
            t_zero = time.perf_counter() - t0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            xf = wsg.features([p])
            pred = wsg.predict_on_grid(xf, wsg.N)
            x0 = wsg.grid_to_fields(pred, bd.HOM_FP64)
            torch.cuda.synchronize()
            t_net = time.perf_counter() - t0
            warm = solver(p, precision=prec, tol=tol, x0=x0)
            t_warm = time.perf_counter() - t0
            net_only = solver(p, precision=prec, tol=tol, x0=x0, max_iter=0)
            S = warm["upper"] - warm["lower"]

            def psd(M):
                return bool(np.linalg.eigvalsh(0.5 * (M + M.T)).min() >= -1e-9 * np.abs(zero["upper"]).max())
            row = {
                "iters_zero": _iters(zero), "iters_warm": _iters(warm), "ms_zero": 1e3 * t_zero,
                "ms_warm_total": 1e3 * t_warm, "ms_network": 1e3 * t_net,
                "rel_bound_diff": float(max(np.abs(warm[k] - zero[k]).max() / np.linalg.norm(zero[k])
                                            for k in ("upper", "lower"))),
                "ordering_ok": psd(S),
                # every bound of either run encloses the same A_H: the cross orderings hold too
                "cross_ordering_ok": psd(warm["upper"] - zero["lower"]) and psd(zero["upper"] - warm["lower"]) and
                psd(net_only["upper"] - zero["lower"]) and psd(zero["upper"] - net_only["lower"]),
                "net_only_gap_ratio": float(np.trace(net_only["upper"] - net_only["lower"]) /
                                            max(np.trace(zero["upper"] - zero["lower"]), 1e-300)),
            }
            if tight is not None:
                zt = solver(p, precision=prec, tol=tight)
                wt = solver(p, precision=prec, tol=tight, x0=x0)
                row.update({"iters_zero_tight": _iters(zt), "iters_warm_tight": _iters(wt)})
            if coarse:
                # (a) the network at its training grid on the cell sampled there, prolonged
                # exactly to the fine grid (nested spaces); (b) the method's own coarse
                # solution prolonged the same way (a non-learned reference start)
                pc = p.with_N(N_train)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                predc = ws.predict_on_grid(ws.features([pc]), N_train)
                xc = coarse_start(p, ws.grid_to_fields(predc, bd.HOM_FP64))
                cw = solver(p, precision=prec, tol=tol, x0=xc)
                t_cw = time.perf_counter() - t0
                cw_only = solver(p, precision=prec, tol=tol, x0=xc, max_iter=0)
                fc = torch.empty(ws.field_shape(1), dtype=torch.complex128, device=ws.dev)
                solver(pc, precision=prec, tol=tol)                 # warm-up of the coarse grid
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                solver(pc, precision=prec, tol=tol, fields=fc)
                xs = coarse_start(p, fc)
                cs = solver(p, precision=prec, tol=tol, x0=xs)
                t_cs = time.perf_counter() - t0
                row.update({
                    "iters_coarse_net": _iters(cw), "ms_coarse_net_total": 1e3 * t_cw,
                    "coarse_net_only_gap_ratio": float(np.trace(cw_only["upper"] - cw_only["lower"]) /
                                                       max(np.trace(zero["upper"] - zero["lower"]), 1e-300)),
                    "iters_coarse_solve": _iters(cs), "ms_coarse_solve_total": 1e3 * t_cs,
                    "coarse_ordering_ok": psd(cw["upper"] - zero["lower"]) and psd(zero["upper"] - cw["lower"]) and
                    psd(cs["upper"] - zero["lower"]) and psd(zero["upper"] - cs["lower"]),
                })
                if tight is not None:
                    row.update({"iters_coarse_net_tight": _iters(solver(p, precision=prec, tol=tight, x0=xc)),
                                "iters_coarse_solve_tight": _iters(solver(p, precision=prec, tol=tight, x0=xs))})
                del predc, xc, xs, fc
            rows.append(row)
            del pred, x0
        return rows

    rows_test = compare(test_probs, ws, tight_tol)
    rows_eval = compare(eval_probs, ws.with_grid(N_eval), tight_tol, coarse=N_eval != N_train)
    if own:
        solver.close()

    def mean(rows, k):
        return float(np.mean([r[k] for r in rows])) if rows else None

    return {
        "N_train": N_train, "N_eval": N_eval, "n_train": n_train, "n_test": n_test, "eval_seeds": list(eval_seeds),
        "epochs": epochs, "batch": batch, "precision": precision, "tol": tol, "gen_tol": gen_tol,
        "network": {"width": width, "modes": modes, "layers": layers, "proj": proj, "params": ws.n_params, "d": 3},
        "loss_first_epoch": hist[0] if hist else None, "loss_last_epoch": hist[-1] if hist else None,
        "gen_iters_mean": float(np.mean(gen_iters)),
        "test_iters_zero_mean": mean(rows_test, "iters_zero"), "test_iters_warm_mean": mean(rows_test, "iters_warm"),
        "test_ms_zero_mean": mean(rows_test, "ms_zero"), "test_ms_warm_mean": mean(rows_test, "ms_warm_total"),
        "tight_tol": tight_tol,
        "test_iters_zero_tight_mean": mean(rows_test, "iters_zero_tight") if tight_tol else None,
        "test_iters_warm_tight_mean": mean(rows_test, "iters_warm_tight") if tight_tol else None,
        "test_max_rel_bound_diff": float(max(r["rel_bound_diff"] for r in rows_test)) if rows_test else None,
        "test_ordering_ok": all(r["ordering_ok"] and r["cross_ordering_ok"] and r.get("coarse_ordering_ok", True)
                                for r in rows_test + rows_eval),
        "test_net_only_gap_ratio_median": float(np.median([r["net_only_gap_ratio"] for r in rows_test]))
        if rows_test else None,
        "eval": rows_eval,
        "time_geometry_s": t_probs, "time_data_s": t_data, "time_train_s": t_train,
    }
