#!/usr/bin/env python
"""Benchmark: time to guaranteed bounds on the 3D cube cell, N = 41^3 (double grid 81^3).

One step = one hom_bounds call = the whole hot path: both double-grid coefficients
built from the closed-form inclusion coefficients, 3 primal and 3 dual CG solves (E =
e1, e2, e3) to a relative residual of 1e-4, FP64 re-projection and the exact
double-grid bound energies, upper and inv(lower) on the host.

Prints one JSON line (rank 0). Default: 1 GPU, plain FP64 CG (the workload's stated
precision), 10 timed steps after 3 warm-up steps, L2 flushed between steps. Extra
keys report the mixed-precision path (FP32 inner CG, FP64 outer) on the same
workload and single-matvec timings. ``--impl reference`` times the CPU oracle
instead (the reference arm of this comparison).

Multi-GPU: independent replicas (the path does not shard): under torchrun each rank
runs the same workload on its own GPU; timing is max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to bounds at 1e-4 rel. residual; matvec HBM GB/s; vs plain FP64 CG"
WORKLOAD = ("3D d=3, N=41^3 (double grid 81^3), centred cube inclusion side 0.5, contrast 100 "
            "(a=1 matrix, a=100 inclusion), plain CG, primal and dual bounds for E=e1,e2,e3, "
            "stop at ||r|| <= 1e-4 ||E||")
TOL = 1e-4
# FP64 CG iterations of this workload at 1e-4 (primal, dual), per right-hand side: a
# property of the problem (CG in exact arithmetic); measured by running the oracle's
# own CG to completion, pinned by tests/test_bench_host.py.
ORACLE_ITERS = {"primal": 46, "dual": 24}
HBM_PEAK_GBS = 6782.8       # measured copy bandwidth of the GB300s (MEASURED_PEAKS.json)
FP64_PEAK_TFLOPS = 1.25     # nominal GB300 FP64 (the recipe's table); a probe measured 1.256

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_xpass<double, 81> launch
# on the 3D N = 41 cube workload (3 fields, isotropic coefficient), from one ncu capture of
# the build whose kernel sources hash to `sha256_16`; reported only while they still do.
XPASS_TRAFFIC = {"sha256_16": "e18ef698bd254de5", "bytes": 24164352 + 26368, "fp64_pipe_active": 0.8375,
                 "sources": ("common.cuh", "kernels.cuh", "passes.cuh", "passes_f64.cu"),
                 "capture": "profiles/xpass_f64_cube3d_N41.md"}


def xpass_traffic(workload_name, precision):
    """Per-launch DRAM traffic of the FP64 row pass, or None once the kernel has changed."""
    import hashlib
    if workload_name != "cube3d_N41" or precision != "fp64":
        return None
    h = hashlib.sha256()
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1404_3614_gb300", "csrc")
    for f in XPASS_TRAFFIC["sources"]:
        with open(os.path.join(src, f), "rb") as fh:
            h.update(fh.read())
    return XPASS_TRAFFIC["bytes"] if h.hexdigest()[:16] == XPASS_TRAFFIC["sha256_16"] else None


WORKLOADS = {
    "cube3d_N41": "3D cube cell N=41^3 (double grid 81^3), contrast 100",
    "spheres3d_N113": "3D cell with 16 random balls, volume fraction 0.3, contrast 1000, N=113^3 (double grid 225^3), seed 0",
    "square2d_N23": "2D square inclusion side 0.6, a=1/10, N=23^2 (double grid 45^2)",
    "porous2d_N1199": "2D synthetic porous pixel image 1199^2 (pores: union of random disks, fraction 0.45), "
                      "a = 0.49 / 0.029, N = 1199 (double grid 2397^2)",
}


def workload(name: str = "cube3d_N41"):
    import microstructures as ms
    if name == "cube3d_N41":
        return ms.cube_inclusion_3d()
    if name == "spheres3d_N113":
        return ms.random_spheres_3d(0, N=113)
    if name == "square2d_N23":
        return ms.square_inclusion_2d()
    if name == "porous2d_N1199":
        return ms.bitmap_problem(ms.porous_bitmap_2d(0, P=1199))
    raise ValueError(name)


def run_learned(args):
    """The learned warm-start workload: train the Fourier-layer network on method-generated
    correctors of random-rectangle cells at N = 63, then compare CG from zero and from the
    projected prediction on held-out cells (one JSON line)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1404_3614_gb300 as hb
    from paper_1404_3614_gb300 import warmstart
    solver = hb.Bounds(0)
    res = warmstart.train_and_evaluate(N=args.learned_N, n_train=args.learned_train, n_test=args.learned_test,
                                       epochs=args.learned_epochs, batch=32, width=32, modes=12, layers=4,
                                       proj=128, tol=TOL, precision="mixed", solver=solver)
    print(json.dumps({"workload": "learned warm start, random-rectangle cells", **res}), flush=True)
    solver.close()
    return 0


def run_learned3d(args):
    """The 3D learned warm start: train on method-generated correctors of random-sphere cells
    (16 balls, volume fraction 0.3, contrast 1000) at N = 41, then time the 3D sphere workload
    (N = 113, seed 0) in mixed precision from zero and from the network's start (features,
    forward and transform included), plus held-out N = 41 cells (one JSON line)."""
    import __graft_entry__
    __graft_entry__.build()
    import paper_1404_3614_gb300 as hb
    from paper_1404_3614_gb300 import warmstart
    solver = hb.Bounds(0)
    res = warmstart.train_and_evaluate_3d(N_train=41, N_eval=113, n_train=args.learned_train3d,
                                          n_test=args.learned_test3d, eval_seeds=(0, 1), epochs=args.learned_epochs3d,
                                          batch=8, width=args.learned_width3d, modes=args.learned_modes3d, layers=4,
                                          proj=64, tol=TOL, precision="mixed", solver=solver, tight_tol=1e-8)
    print(json.dumps({"workload": "3D learned warm start, random-sphere cells, trained at N=41, "
                      "evaluated at N=113 (seed 0 = the 3D sphere workload)", **res}), flush=True)
    solver.close()
    return 0


def run_batched_only(args):
    """The batched workload alone (for kernel captures): `--batch-n` random-rectangle cells."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1404_3614_gb300 as hb
    solver = hb.Bounds(0)
    fixed = args.batch_threads > 0 or args.batch_cluster > 0
    if args.batch_threads:
        hb.binding.hom_set_batch_threads(solver.ctx, args.batch_threads)
    if args.batch_cluster:
        hb.binding.hom_set_batch_cluster(solver.ctx, args.batch_cluster, args.batch_coop_M)
    res = batched_timings(hb, solver, torch.device("cuda", 0), n=args.batch_n, n_seq=2, autotune=0 if fixed else 1)
    print(json.dumps({"batched": res}), flush=True)
    solver.close()
    return 0


def run_matvec_only(args):
    """Operator applications only (for kernel captures): `--reps` hom_matvec calls on d fields."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1404_3614_gb300 as hb
    problem = workload(args.workload)
    solver = hb.Bounds(0)
    stream = torch.cuda.current_stream()
    mv = matvec_timings(hb, solver, problem, torch.device("cuda", 0), stream, reps=args.reps,
                        precisions=(args.precision,) if args.precision != "mixed" else ("fp32",))
    print(json.dumps({"workload": WORKLOADS[args.workload], "matvec": mv}), flush=True)
    solver.close()
    return 0


def run_paper_grids(args):
    """The paper's square-inclusion study (Sec. 7, Eqs. S, S1, S2): for each contrast, the
    Galerkin (exact integration) bounds, the GaNi homogenized matrices A_{H,N}, B_{H,N}^{-1}
    and the bounds of the GaNi fields, on odd grids n = 5 3^j (cell S) and on even grids
    n = 2^j (cells S1 and S2). FP64, tol 1e-8. One JSON line per (cell, contrast, n)."""
    import numpy as np
    import __graft_entry__
    __graft_entry__.build()
    import microstructures as ms
    import paper_1404_3614_gb300 as hb
    solver = hb.Bounds(0)
    cases = [("S", False, n) for n in (5, 15, 45, 135, 405)] + \
            [(c, c == "S2", n) for n in (4, 8, 16, 32, 64, 128, 256, 512) for c in ("S1", "S2")]
    for rho in (10.0, 1000.0):
        for cell, closed, n in cases:
            p = ms.paper_square_2d(n, rho) if cell == "S" else ms.paper_square_even_2d(n, rho, closed=closed)
            t0 = time.perf_counter()
            ga = solver(p, precision=hb.HOM_FP64, tol=1e-8)
            gn = solver(p, precision=hb.HOM_FP64, tol=1e-8, discretization=1)
            print(json.dumps({"cell": cell, "rho": rho, "n": n,
                              "ga_upper": ga["upper"][0, 0], "ga_lower": ga["lower"][0, 0],
                              "gani_A": gn["gani_A"][0, 0], "gani_invB": float(np.linalg.inv(gn["gani_B"])[0, 0]),
                              "gani_upper": gn["upper"][0, 0], "gani_lower": gn["lower"][0, 0],
                              "iters_ga": int(np.asarray(ga["report"]["iters"]).sum()),
                              "iters_gani": int(np.asarray(gn["report"]["iters"]).sum()),
                              "s": time.perf_counter() - t0}), flush=True)
    solver.close()
    return 0


def run_even_grids(args):
    """The paper's even-grid cells S1/S2 (Sec. 7.2, Eqs. S1, S2) at n = 512 and 1024,
    rho = 10 and 10^3, tol 1e-8: Ga and GaNi in FP64 and in mixed precision. Each solve is
    timed on its second call (the first builds plans and captures graphs); one JSON line per
    (cell, rho, n, precision) with the bounds, so the precisions can be compared."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import microstructures as ms
    import paper_1404_3614_gb300 as hb
    solver = hb.Bounds(0)
    for n in (512, 1024):
        for rho in (10.0, 1000.0):
            for cell in ("S1", "S2"):
                p = ms.paper_square_even_2d(n, rho, closed=cell == "S2")
                for pname, prec in (("fp64", hb.HOM_FP64), ("mixed", hb.HOM_MIXED)):
                    line = {"cell": cell, "rho": rho, "n": n, "precision": pname, "tol": 1e-8}
                    for disc, tag in ((0, "ga"), (1, "gani")):
                        solver(p, precision=prec, tol=1e-8, discretization=disc)
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        o = solver(p, precision=prec, tol=1e-8, discretization=disc)
                        torch.cuda.synchronize()
                        line[tag + "_s"] = time.perf_counter() - t0
                        line[tag + "_upper"] = float(o["upper"][0, 0])
                        line[tag + "_lower"] = float(o["lower"][0, 0])
                        line[tag + "_iters"] = int(np.asarray(o["report"]["iters"]).sum())
                    print(json.dumps(line), flush=True)
    solver.close()
    return 0


def run_gemm_only(args):
    """The network's tensor-core GEMM alone (for kernel captures and its roofline): a 1x1
    channel-mixing layer of the 3D network, C = A B with A [M x K] FP32 (M = 2^20 grid points,
    4 MiB per channel column, larger than L2 at K = 64), B [K x N], `--reps` timed launches."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1404_3614_gb300 as hb
    M, N, K = 1 << 20, 64, 64
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn((M, K), generator=g, device="cuda")
    B = torch.randn((K, N), generator=g, device="cuda")
    C = torch.empty((M, N), device="cuda")
    ctx = hb.hom_create(0)
    stream = torch.cuda.current_stream().cuda_stream

    def run():
        hb.binding.hom_gemm_bf16(ctx, M, N, K, A.data_ptr(), K, 0, B.data_ptr(), N, 0, C.data_ptr(), N, 1.0, 0.0,
                                 stream)
    for _ in range(3):
        run()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(args.reps):
        run()
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / args.reps
    ref = (A[:4096].bfloat16().double() @ B.bfloat16().double())
    err = float((C[:4096].double() - ref).abs().max() / ref.abs().max())
    hb.hom_destroy(ctx)
    flops = 2.0 * M * N * K
    byt = 4.0 * (M * K + K * N + M * N)
    print(json.dumps({"gemm": {"M": M, "N": N, "K": K, "ms": ms, "tflops": flops / ms / 1e9,
                               "gbs": byt / ms / 1e6, "hbm_frac": byt / ms / 1e6 / HBM_PEAK_GBS,
                               "max_rel_err_vs_bf16_products": err}}), flush=True)
    return 0


# ------------------------------------------------------------------------------------
# distributed helpers (host logic; covered by CPU gloo tests)
# ------------------------------------------------------------------------------------
def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------
# algorithmic FLOP counts (conventional 5 M log2 M per complex length-M FFT)
# ------------------------------------------------------------------------------------
def fft_flops(M: int) -> float:
    return 5.0 * M * math.log2(M) if M > 1 else 0.0


def family_flops_per_launch(problem, family: str, nrhs: int) -> float:
    """FFT flops one launch of a kernel family performs on the operator of `problem`."""
    d = problem.d
    N = [int(n) for n in problem.N] + [1] * (3 - d)
    M = [2 * n - 1 for n in N]
    Nh = (N[0] + 1) // 2
    RC = nrhs * d
    if family == "xpass":
        return RC * M[1] * M[2] * fft_flops(M[0])          # pairs of real rows -> one complex FFT each way
    if family == "zpass":
        return RC * N[1] * Nh * fft_flops(M[2])
    if family == "final":
        return RC * (N[1] * Nh * fft_flops(M[2]) if d == 3 else Nh * fft_flops(M[1]))
    if family == "ypass":
        return RC * M[2] * Nh * fft_flops(M[1])
    if family == "slab":    # fused inverse y, x row pass and forward y
        return (2 * family_flops_per_launch(problem, "ypass", nrhs)
                + family_flops_per_launch(problem, "xpass", nrhs))
    return 0.0


# ------------------------------------------------------------------------------------
# CPU oracle leg
# ------------------------------------------------------------------------------------
def oracle_sample(problem, iters, n_matvec: int):
    """Time the oracle on a bounded sample and extrapolate to one full time to bounds.

    Sample: both double-grid coefficient builds (naive inverse DFT) + n_matvec
    double-grid matvecs per side on one right-hand side. Estimate: coefficient builds
    + (iters_side x d) matvecs per side + d/2 matvec-equivalents per side for the energies.
    """
    import numpy as np
    from oracle import matfree
    d = problem.d
    total = 0.0
    t_coef = 0.0
    t_mv = {}
    for side in ("primal", "dual"):
        t = time.perf_counter()
        op = matfree.MatFreeOperator(problem, side)
        t_coef += time.perf_counter() - t
        u = op.constant_field(np.eye(d)[0])
        u = op.apply(u)
        t = time.perf_counter()
        for _ in range(n_matvec):
            u = op.apply(u)
            u /= max(np.abs(u).max(), 1e-300)
        t_mv[side] = (time.perf_counter() - t) / n_matvec
    for side in ("primal", "dual"):
        total += (iters[side] * d + 0.5 * d) * t_mv[side]
    est = (t_coef + total) * 1e3
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    threads = int(os.environ.get("OPENBLAS_NUM_THREADS", os.environ.get("OMP_NUM_THREADS", cores)))
    sample = (f"oracle O2 (naive-DFT double-grid CG, numpy fp64): both coefficient builds + {n_matvec} "
              f"matvecs per side on one RHS, timed; extrapolated with {iters['primal']}/{iters['dual']} "
              f"CG iterations x {d} RHS per side + d/2 matvecs per side for the energies")
    return est, {"value": est, "unit": "ms", "cores": min(threads, cores), "kind": "oracle", "sample": sample,
                 "matvec_ms": {k: v * 1e3 for k, v in t_mv.items()}, "coef_ms": t_coef * 1e3}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    problem = workload()
    vals = []
    info = None
    for i in range(args.warmup + args.steps):
        v, info = oracle_sample(problem, ORACLE_ITERS, n_matvec=max(2, args.ref_matvecs // 3))
        if i >= args.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "impl": "CPU oracle (naive DFT double-grid CG)"},
            "cpu_baseline": info, "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0,
                                          "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------
# GPU leg
# ------------------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1404_3614_gb300 as hb

    problem = workload(args.workload)
    prec = hb.HOM_FP64 if args.precision == "fp64" else hb.HOM_MIXED
    solver = hb.Bounds(local)
    stream = torch.cuda.current_stream(dev)
    s_ptr = stream.cuda_stream
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > L2 (129 MB)

    def step(precision):
        return solver(problem, precision=precision, tol=TOL, stream=s_ptr)

    for _ in range(args.warmup):
        out = step(prec)
    torch.cuda.synchronize()

    # dominant kernel family: one untimed profiled step per family
    fam_ms = {}
    for fam in ("slab", "xpass", "ypass", "zpass", "final", "cg", "coef", "energy"):
        hb.hom_profile_kernel(solver.ctx, fam)
        step(prec)
        n, ms = hb.hom_kernel_timing(solver.ctx)
        fam_ms[fam] = (n, ms)
    hb.hom_profile_kernel(solver.ctx, "")
    dom = max(fam_ms, key=lambda f: fam_ms[f][1])

    # timed region: K steps, device time by CUDA events on the launching stream,
    # L2 flushed between steps (outside the events), dominant family timed live
    hb.hom_profile_kernel(solver.ctx, dom)
    times = []
    launches = 0
    reports = []
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = step(prec)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            reports.append(out["report"])
            launches += out["report"]["launches"]
    torch.cuda.synchronize()
    barrier(world)
    dom_n, dom_ms = hb.hom_kernel_timing(solver.ctx)
    hb.hom_profile_kernel(solver.ctx, "")
    ms_step = statistics.mean(times)
    ms_step = max_over_ranks(ms_step, world, dev)

    # end to end through the public API: host problem in, host bounds out, wall clock. Two
    # workspaces alternate, as for two requests in flight, so every step uploads its problem
    # tables (inclusions, twiddles) from the host again instead of finding them resident.
    opts_e2e = hb.make_opts(prec, TOL)
    nbytes = hb.hom_workspace_size(solver.ctx, problem, opts_e2e)
    wss = [torch.empty(nbytes, dtype=torch.uint8, device=dev) for _ in range(2)]

    def step_e2e(i):
        return hb.hom_bounds(solver.ctx, problem, opts_e2e, wss[i % 2].data_ptr(), nbytes, s_ptr)
    for i in range(2 * args.warmup):
        step_e2e(i)
    e2e = []
    for i in range(max(4, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        o = step_e2e(i)
        e2e.append((time.perf_counter() - t) * 1e3)
    e2e_ms = max_over_ranks(statistics.mean(e2e), world, dev)
    rep = o["report"]
    del wss

    # the other precision on the same workload (plain FP64 vs mixed)
    other = hb.HOM_MIXED if prec == hb.HOM_FP64 else hb.HOM_FP64
    alt = []
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        oo = step(other)
        e1.record(stream)
        e1.synchronize()
        alt.append(e0.elapsed_time(e1))
    alt_ms = statistics.mean(alt)

    # variants of the method on the same workload (FP64, same tolerance): the dual CG started
    # from the primal minimisers, and GaNi (the paper's algorithm: N-grid CG, double-grid
    # bounds) from zero and with the dual start, which is exact for GaNi on odd grids
    def timed(**kw):
        ts, o_ = [], None
        for _ in range(3):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            o_ = solver(problem, tol=TOL, stream=s_ptr, **kw)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.mean(ts), o_
    variants = {}
    F64, MIX = {"precision": hb.HOM_FP64}, {"precision": hb.HOM_MIXED}
    for name, kw in (("dual_start", {"dual_start": 1, **F64}), ("gani", {"discretization": 1, **F64}),
                     ("gani_dual_start", {"discretization": 1, "dual_start": 1, **F64}),
                     ("gani_mixed", {"discretization": 1, **MIX}),
                     ("gani_mixed_dual_start", {"discretization": 1, "dual_start": 1, **MIX})):
        timed(**kw)   # untimed first call (graph capture, tables)
        ms_v, o_v = timed(**kw)
        variants[name] = {"ms": ms_v, "iters": o_v["report"]["iters"], "upper_11": float(o_v["upper"][0, 0]),
                          "lower_11": float(o_v["lower"][0, 0])}
        if "gani_A" in o_v:
            variants[name]["gani_A_11"] = float(o_v["gani_A"][0, 0])
            variants[name]["gani_invB_11"] = float(np.linalg.inv(o_v["gani_B"])[0, 0])

    # one operator application (3 fields) per precision, through hom_matvec
    mv = matvec_timings(hb, solver, problem, dev, stream)
    # the 225^3 operator of the 16-ball cell, where the HBM fraction is claimed
    mv_large = None
    if args.workload != "spheres3d_N113":
        mv_large = matvec_timings(hb, solver, workload("spheres3d_N113"), dev, stream, reps=10)
        mv_large["workload"] = WORKLOADS["spheres3d_N113"]
    batched = None if args.no_batched else batched_timings(hb, solver, dev)
    image = None if args.no_batched else image_timings(hb, solver, stream, flush)

    # roofline of the dominant kernel family
    nrhs = problem.d
    per_launch_ms = dom_ms / max(dom_n, 1)
    flops = family_flops_per_launch(problem, dom, nrhs)
    roof = None
    if flops > 0 and per_launch_ms > 0:
        achieved = flops / (per_launch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": xpass_traffic(args.workload, args.precision) if dom == "xpass" else None,
                "flops_per_launch": flops, "launches": dom_n, "avg_launch_ms": per_launch_ms,
                "peak_note": "FP64 nominal 1.25 TFLOP/s (recipe table); FMA probe measured 1.256"}
        if prec != hb.HOM_FP64:
            roof["note"] = "mixed: dominant family mixes FP32 inner and FP64 outer launches"
        if roof["traffic"] is not None:
            roof["traffic_note"] = ("ncu DRAM bytes per launch (" + XPASS_TRAFFIC["capture"] + "): the "
                                    "input fields and coefficient are read once; the in-place output "
                                    "stays in L2 during the launch")
            # the same capture: the FP64 pipe is busy this fraction of the active cycles; the
            # conventional 5 M log2 M flop count undercounts an add-heavy radix-3 FFT, so frac
            # reads well below the pipe's own occupancy
            roof["fp64_pipe_active_ncu"] = XPASS_TRAFFIC["fp64_pipe_active"]

    line = {
        "metric": METRIC, "value": ms_step, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == hb.HOM_FP64 else "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if args.workload == "cube3d_N41" else WORKLOADS[args.workload],
                   "precision": args.precision, "tol": TOL,
                   "l2": "flushed between steps (256 MiB write, outside the timed region)",
                   "launch": "CG iterations in blocks of 8 replayed from captured CUDA graphs",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "bounds": {"upper_11": float(out["upper"][0, 0]), "lower_11": float(out["lower"][0, 0])},
        "iters": reports[-1]["iters"], "matvecs": reports[-1]["matvecs"],
        "gpu_launches": launches,
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": rep["h2d_bytes"],
                "d2h_bytes_per_step": rep["d2h_bytes"],
                "note": "hom_bounds wall clock: host problem in (tables uploaded every step, two workspaces "
                        "alternating), host bounds out"},
        "alt_precision": {"precision": "mixed" if other == hb.HOM_MIXED else "fp64", "ms": alt_ms,
                          "speedup_vs_this": ms_step / alt_ms if alt_ms > 0 else None,
                          "upper_11": float(oo["upper"][0, 0]), "lower_11": float(oo["lower"][0, 0])},
        "variants": variants,
        "matvec": mv,
        "matvec_225": mv_large,
        "batched": batched,
        "image": image,
        "kernel_families_ms_one_step": {k: v[1] for k, v in fam_ms.items()},
        "roofline": roof,
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        iters = {"primal": max(reports[-1]["iters"][0]), "dual": max(reports[-1]["iters"][1])}
        _, info = oracle_sample(problem, iters, n_matvec=args.ref_matvecs)
        line["cpu_baseline"] = info
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def batched_timings(hb, solver, dev, n=256, reps=3, n_seq=8, autotune=1):
    """The batched workload: n seeded random-rectangle 2D cells (N from {23, 63, 113, 203}),
    FP32 inner CG / FP64 bounds, tol 1e-4, one persistent launch replayed as a CUDA graph
    after an autotuning pass (threads per CTA, chunk capacity, radix schedule, cluster size
    for the largest cells); against plain FP64 hom_bounds one cell at a time on the same
    GPU (a sample of n_seq cells, extrapolated to n)."""
    import statistics as st_
    import torch
    import microstructures as ms
    probs = [ms.random_rectangles_2d(s) for s in range(n)]
    stream = torch.cuda.Stream(device=dev)
    out = solver.batched(probs, precision=hb.HOM_MIXED, tol=TOL, autotune=autotune, graph=1,
                         stream=stream.cuda_stream)
    times = []
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    for _ in range(reps):
        with torch.cuda.stream(stream):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        out = solver.batched(probs, precision=hb.HOM_MIXED, tol=TOL, graph=1, stream=stream.cuda_stream)
        with torch.cuda.stream(stream):
            e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms_batch = st_.mean(times)
    seq = []
    for p in probs[:n_seq]:
        torch.cuda.synchronize()
        t = time.perf_counter()
        solver(p, precision=hb.HOM_FP64, tol=TOL)
        seq.append((time.perf_counter() - t) * 1e3)
    seq_ms = st_.mean(seq) * n
    return {"workload": f"{n} random-rectangle 2D cells, N from {{23,63,113,203}}, FP32 inner CG, FP64 bounds, tol {TOL:g}",
            "ms": ms_batch, "problems_per_s": n / (ms_batch * 1e-3), "launches": out["report"]["launches"],
            "launch_config": out["report"]["config"],
            "max_iters": int(out["iters"].max()), "status_nonzero": int((out["status"] != 0).sum()),
            "sequential_fp64_ms_est": seq_ms, "speedup_vs_sequential_fp64": seq_ms / ms_batch,
            "sequential_note": f"plain FP64 hom_bounds per cell, mean of the first {n_seq} cells x {n}"}


def image_timings(hb, solver, stream, flush):
    """The pixel-image workload (the paper's Sec. 7.3 type, synthetic stand-in): a 1199^2
    porous two-phase image at N = 1199, tol 1e-4: Ga in FP64 and mixed, GaNi (the paper's
    algorithm) with and without the dual start. One untimed call, then one timed call each."""
    import torch
    import microstructures as ms
    p = workload("porous2d_N1199")
    out = {"workload": WORKLOADS["porous2d_N1199"]}
    for name, kw in (("ga_fp64", {"precision": hb.HOM_FP64}), ("ga_mixed", {"precision": hb.HOM_MIXED}),
                     ("gani_fp64", {"precision": hb.HOM_FP64, "discretization": 1}),
                     ("gani_fp64_dual_start", {"precision": hb.HOM_FP64, "discretization": 1, "dual_start": 1}),
                     ("smoothed_ga_mixed", {"precision": hb.HOM_MIXED}),
                     ("smoothed_gani_fp64", {"precision": hb.HOM_FP64, "discretization": 1})):
        if name.startswith("smoothed") and "smoothed_image" not in out:
            out["smoothed_image"] = "the same image with the paper's 4/2/1 local average of the solid phase"
            p = ms.bitmap_problem(ms.porous_bitmap_2d(0, P=1199), smooth=True)
        solver(p, tol=TOL, stream=stream.cuda_stream, **kw)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        o = solver(p, tol=TOL, stream=stream.cuda_stream, **kw)
        e1.record(stream)
        e1.synchronize()
        out[name] = {"ms": e0.elapsed_time(e1), "iters": o["report"]["iters"],
                     "upper": o["upper"].tolist(), "lower": o["lower"].tolist()}
    return out


def matvec_bytes(problem, elem_bytes: int) -> float:
    """Algorithmic bytes of one operator application on d fields in the pass structure used
    (z inverse, y inverse, x rows, y forward, z forward + projection + p.Cp): every pass reads
    and writes its input and output once, the coefficient is read once per field set."""
    d = problem.d
    N = [int(n) for n in problem.N] + [1] * (3 - d)
    M = [2 * n - 1 for n in N]
    Nh = (N[0] + 1) // 2
    if d == 3:
        per = Nh * (2 * N[2] * N[1] + 4 * M[2] * N[1] + 4 * M[2] * M[1])
    else:
        per = Nh * (2 * N[1] + 4 * M[1])
    cplx = 2 * elem_bytes
    fields = d * d
    coef = M[0] * M[1] * M[2] * elem_bytes * d      # read once per right-hand side
    return fields * per * cplx + coef


def matvec_timings(hb, solver, problem, dev, stream, reps=20, precisions=("fp64", "fp32")):
    """Device time of one operator application on d fields, FP64 and FP32."""
    import torch
    ctx = solver.ctx
    info = hb.hom_problem_info(ctx, problem)
    d = problem.d
    nws = hb.hom_step_workspace_size(ctx, problem, d)
    ws = torch.empty(nws, dtype=torch.uint8, device=dev)
    shape = (d, d, int(problem.N[2]), int(problem.N[1]), (int(problem.N[0]) + 1) // 2)
    out = {}
    for name, prec, cdt, rdt in (("fp64", hb.HOM_FP64, torch.complex128, torch.float64),
                                 ("fp32", hb.HOM_FP32, torch.complex64, torch.float32)):
        if name not in precisions:
            continue
        coef = torch.empty((info["ncomp"],) + tuple(info["M"][::-1]), dtype=rdt, device=dev)
        hb.hom_coefficient(ctx, problem, 0, prec, coef.data_ptr(), ws.data_ptr(), nws, stream.cuda_stream)
        x = torch.randn(shape, dtype=cdt, device=dev)
        y = torch.empty_like(x)
        for _ in range(3):
            hb.hom_matvec(ctx, problem, 0, prec, 1, d, coef.data_ptr(), x.data_ptr(), y.data_ptr(),
                          ws.data_ptr(), nws, stream.cuda_stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            hb.hom_matvec(ctx, problem, 0, prec, 1, d, coef.data_ptr(), x.data_ptr(), y.data_ptr(),
                          ws.data_ptr(), nws, stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        flops = sum(family_flops_per_launch(problem, f, d) * (2 if f == "ypass" else 1)
                    for f in ("zpass", "ypass", "xpass", "final"))
        nbytes = matvec_bytes(problem, 8 if name == "fp64" else 4)
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "matvecs_per_s": 1e3 / ms, "fft_tflops": flops / (ms * 1e-3) / 1e12, "fields": d,
                     "model_bytes": nbytes, "model_gbs": gbs, "model_hbm_frac": gbs / HBM_PEAK_GBS}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--ref-matvecs", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--workload", default="cube3d_N41", choices=sorted(WORKLOADS))
    ap.add_argument("--matvec-only", action="store_true", help="operator applications only")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--batched-only", action="store_true", help="the batched workload only")
    ap.add_argument("--batch-n", type=int, default=256, help="cells in the batched workload")
    ap.add_argument("--batch-threads", type=int, default=0, help="fix the threads per CTA (no autotune)")
    ap.add_argument("--batch-cluster", type=int, default=0, help="fix the cluster size (no autotune)")
    ap.add_argument("--batch-coop-M", type=int, default=225, help="with --batch-cluster: cooperative 2N-1")
    ap.add_argument("--learned", action="store_true", help="learned warm-start workload only")
    ap.add_argument("--learned-N", type=int, default=63)
    ap.add_argument("--learned-train", type=int, default=20000)
    ap.add_argument("--learned-test", type=int, default=1024)
    ap.add_argument("--learned-epochs", type=int, default=20)
    ap.add_argument("--learned3d", action="store_true", help="3D learned warm-start workload only")
    ap.add_argument("--gemm-only", action="store_true", help="the network's tensor-core GEMM alone")
    ap.add_argument("--paper-grids", action="store_true",
                    help="the paper's square-inclusion study on odd and even grids (Ga and GaNi)")
    ap.add_argument("--even-grids", action="store_true",
                    help="the paper's even-grid cells S1/S2 at n = 512, 1024: Ga and GaNi, FP64 and mixed")
    ap.add_argument("--learned-train3d", type=int, default=1000)
    ap.add_argument("--learned-test3d", type=int, default=16)
    ap.add_argument("--learned-epochs3d", type=int, default=30)
    ap.add_argument("--learned-width3d", type=int, default=24)
    ap.add_argument("--learned-modes3d", type=int, default=8)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.matvec_only:
        return run_matvec_only(args)
    if args.batched_only:
        return run_batched_only(args)
    if args.learned:
        return run_learned(args)
    if args.learned3d:
        return run_learned3d(args)
    if args.gemm_only:
        return run_gemm_only(args)
    if args.paper_grids:
        return run_paper_grids(args)
    if args.even_grids:
        return run_even_grids(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
