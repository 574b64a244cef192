#!/usr/bin/env python
"""Benchmark: time to guaranteed bounds on the 3D cell with 16 random balls, N = 113^3.

One step = one hom_bounds call = the whole hot path: both double-grid coefficients built
from the closed-form ball coefficients, 3 primal and 3 dual CG solves (E = e1, e2, e3) to a
relative residual of 1e-4 with FP32 inner CG and FP64 outer refinement, FP64 re-projection
and the exact double-grid bound energies, upper and inv(lower) on the host.

Prints one JSON line (rank 0). Default: 1 GPU, mixed precision (the workload's stated
"FP32 inner CG with FP64 bounds"), 10 timed steps after 3 warm-up steps, L2 flushed between
steps. The same line carries plain FP64 CG on the same cell (the "vs plain FP64 CG" part of
the metric), the roofline of the dominant kernel (the fused FP32 slab pass of the operator,
against the measured HBM bandwidth), the measured FMA peaks, the 3D cube cell, the 256-cell
batched launch against all 256 cells solved one by one in FP64, and the CPU oracle timed on
a bounded sample. ``--impl reference`` times the CPU oracle instead (the reference arm).

Multi-GPU: independent replicas (the path does not shard): under torchrun each rank runs the
same workload on its own GPU; timing is max over ranks.
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
WORKLOAD = ("3D d=3, N=113^3 (double grid 225^3), 16 random non-overlapping balls (seed 0), volume "
            "fraction 0.3, contrast 1000 (a=1 matrix, a=1000 balls), FP32 inner CG with FP64 refinement "
            "(residuals in float-float arithmetic on FP64 data), FP64 re-projection and bounds, primal and dual "
            "bounds for E=e1,e2,e3, stop at ||r|| <= 1e-4 ||E||")
CUBE_WORKLOAD = ("3D d=3, N=41^3 (double grid 81^3), centred cube inclusion side 0.5, contrast 100 "
                 "(a=1 matrix, a=100 inclusion), plain FP64 CG")
TOL = 1e-4
# FP64 CG iterations of the cube cell at 1e-4 (primal, dual), per right-hand side: a property
# of the problem (CG in exact arithmetic), from the oracle's own CG, pinned by
# tests/test_bench_host.py.
ORACLE_ITERS = {"primal": 46, "dual": 24}
GOLDEN = os.path.join(ROOT, "tests", "golden", "fullsize_bounds.json")
FALLBACK_HBM_GBS = 6800.0     # used only when MEASURED_PEAKS.json is absent ("of fallback")


def measured_peaks():
    """The measured peaks of the GB300s (copy bandwidth, bf16 GEMM)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "of measured (MEASURED_PEAKS.json)"}
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "source": "of fallback (recipe: 6.8 TB/s)"}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_slab<float, 15> launch on
# the 16-ball cell (9 fields, 3 right-hand sides), from one ncu capture of the build whose
# kernel sources (the kernel's file, the device helpers it calls and its argument struct) hash
# to `sha256_16`; reported only while they still do.
SLAB_TRAFFIC = {"sha256_16": "54945fc3d6ddd343", "bytes": 149977344 + 48060672,
                "sources": ("common.cuh", "kernels.cuh:SlabArgs", "slab.cuh"),
                "capture": "profiles/slab_f32_spheres3d_N113.md"}


def source_hash(files) -> str:
    """SHA-256 (16 hex digits) of kernel sources: whole files, or "file:Name" for the text of
    one `struct Name { ... };` of that file (the argument block a kernel takes from a shared
    header, without the header's unrelated declarations)."""
    import hashlib
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_1404_3614_gb300", "csrc")
    for f in files:
        name, _, struct = f.partition(":")
        with open(os.path.join(src, name), "rb") as fh:
            data = fh.read()
        if struct:
            start = data.index(("struct %s {" % struct).encode())
            data = data[start:data.index(b"};", start) + 2]
        h.update(data)
    return h.hexdigest()[:16]


def slab_traffic():
    """Per-launch DRAM traffic of the slab pass from ncu, or None once the kernel has changed."""
    if SLAB_TRAFFIC["sha256_16"] is None:
        return None
    return SLAB_TRAFFIC["bytes"] if source_hash(SLAB_TRAFFIC["sources"]) == SLAB_TRAFFIC["sha256_16"] else None


WORKLOADS = {
    "spheres3d_N113": "3D cell with 16 random balls, volume fraction 0.3, contrast 1000, N=113^3 (double grid 225^3), seed 0",
    "cube3d_N41": "3D cube cell N=41^3 (double grid 81^3), contrast 100",
    "square2d_N23": "2D square inclusion side 0.6, a=1/10, N=23^2 (double grid 45^2)",
    "porous2d_N1199": "2D synthetic porous pixel image 1199^2 (pores: union of random disks, fraction 0.45), "
                      "a = 0.49 / 0.029, N = 1199 (double grid 2397^2)",
}


def workload(name: str = "spheres3d_N113"):
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


def oracle_iters_c5():
    """CG iterations per right-hand side to 1e-4 of the 16-ball cell, read off the residual
    history of the oracle's own CG (tests/golden/make_fullsize_goldens.py); None if absent."""
    try:
        with open(GOLDEN) as f:
            it = json.load(f)["spheres3d_N113"]["iters_to_1e-4"]
        return {"primal": it[0], "dual": it[1]}
    except Exception:
        return None


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
    res = batched_timings(hb, solver, torch.device("cuda", 0), n=args.batch_n, autotune=0 if fixed else 1)
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
    prec = args.matvec_precision or ("fp32" if args.precision == "mixed" else args.precision)
    mv = matvec_timings(hb, solver, problem, torch.device("cuda", 0), stream, reps=args.reps, precisions=(prec,))
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
                               "gbs": byt / ms / 1e6, "hbm_frac": byt / ms / 1e6 / measured_peaks()["hbm_gbs"],
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
def oracle_sample(problem, iters, n_matvec: int = 2, n_slabs: int = 8):
    """Time the oracle on a bounded sample and extrapolate to one full time to bounds.

    The oracle: O2 (matrix DFTs) for grids up to 81 points per axis, O3 (the same steps with
    library FFTs, pinned to O2) beyond. Sample per side: the closed-form coefficient of
    `n_slabs` of the M first-axis slabs of Z_M (O3; O2 builds it whole), one inverse FFT of
    the whole grid, and `n_matvec` operator applications on one right-hand side. Estimate per
    side: the coefficient (slabs scaled to M) + (iters x d + d for the right-hand sides + d for
    the energies) matvecs, with iters the CG iteration counts per right-hand side.
    """
    import numpy as np
    from oracle import fftcg, matfree
    d = problem.d
    M = [2 * int(n) - 1 for n in problem.N]
    use_o3 = max(M) > 81
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    t_coef, t_mv = {}, {}
    for side in ("primal", "dual"):
        t = time.perf_counter()
        if use_o3:
            import scipy.fft as sfft
            for i0 in range(n_slabs):
                fftcg.coefficient_slab(problem, side, M, i0)
            t_slab = (time.perf_counter() - t) / n_slabs
            t = time.perf_counter()
            grid = sfft.ifftn(np.zeros(M, dtype=np.complex128), workers=cores).real
            t_coef[side] = t_slab * M[0] + (time.perf_counter() - t)
            # the operator with a stand-in coefficient of the same shape: a matvec costs the
            # same whatever the values
            op = fftcg.FFTOperator(problem, side, workers=cores, A_grid=grid + 1.0)
        else:
            op = matfree.MatFreeOperator(problem, side)
            t_coef[side] = time.perf_counter() - t
        u = op.constant_field(np.eye(d)[0])
        u = op.apply(u)
        t = time.perf_counter()
        for _ in range(n_matvec):
            u = op.apply(u)
            u /= max(np.abs(u).max(), 1e-300)
        t_mv[side] = (time.perf_counter() - t) / n_matvec
    total = sum(t_coef.values())
    for side in ("primal", "dual"):
        it = iters[side]
        total += (sum(it) if isinstance(it, (list, tuple)) else it * d) * t_mv[side] + 2 * d * t_mv[side]
    est = total * 1e3
    which = "O3 (library-FFT double-grid CG, scipy.fft, numpy fp64)" if use_o3 else \
        "O2 (matrix-DFT double-grid CG, numpy fp64)"
    sample = (f"oracle {which}: per side the closed-form coefficient of "
              f"{n_slabs if use_o3 else M[0]} of {M[0]} slabs and {n_matvec} matvecs on one RHS, timed; "
              f"extrapolated with the CG iteration counts {iters} + 2d matvecs per side (right-hand sides, "
              f"energies)")
    return est, {"value": est, "unit": "ms", "cores": cores, "kind": "oracle", "sample": sample,
                 "extrapolated": True, "matvec_ms": {k: v * 1e3 for k, v in t_mv.items()},
                 "coef_ms": {k: v * 1e3 for k, v in t_coef.items()}}


def reference_iters(problem, name):
    if name == "spheres3d_N113":
        it = oracle_iters_c5()
        if it is not None:
            return it
        # not yet in the golden file: the GPU FP64 counts of this cell (primal, dual per rhs)
        return {"primal": [176, 176, 176], "dual": [49, 51, 49]}
    return dict(ORACLE_ITERS)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    problem = workload(args.workload)
    iters = reference_iters(problem, args.workload)
    vals = []
    info = None
    for i in range(args.warmup + args.steps):
        v, info = oracle_sample(problem, iters, n_matvec=1 if i < args.warmup else 2, n_slabs=4)
        if i >= args.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.workload == "spheres3d_N113" else WORKLOADS[args.workload],
                       "impl": "CPU oracle (double-grid CG, FP64), bounded sample, extrapolated"},
            "extrapolated": True,
            "cpu_baseline": info, "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0,
                                          "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------
# GPU leg
# ------------------------------------------------------------------------------------
def timed_steps(stream, flush, fn, n):
    """n calls of fn, each bracketed by CUDA events on `stream`, L2 flushed before each
    (outside the events); returns the per-call device times (ms) and the last result."""
    import torch
    ts, out = [], None
    for _ in range(n):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return ts, out


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
    peaks = measured_peaks()

    def step(precision, p=problem):
        return solver(p, precision=precision, tol=TOL, stream=s_ptr)

    for _ in range(args.warmup):
        out = step(prec)
    torch.cuda.synchronize()

    # timed region: K steps, device time by CUDA events on the launching stream, L2 flushed
    # between steps (outside the events), no per-kernel instrumentation
    reports = []
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        times, out = timed_steps(stream, flush, lambda: step(prec), args.steps)
    torch.cuda.synchronize()
    barrier(world)
    launches = out["report"]["launches"] * args.steps
    ms_step = max_over_ranks(statistics.mean(times), world, dev)

    # end to end through the public API: host problem in, host bounds out, wall clock. Two
    # workspaces alternate, as for two requests in flight, so every step uploads its problem
    # tables (inclusions, twiddles) from the host again instead of finding them resident.
    opts_e2e = hb.make_opts(prec, TOL)
    nbytes = hb.hom_workspace_size(solver.ctx, problem, opts_e2e)
    wss = [torch.empty(nbytes, dtype=torch.uint8, device=dev) for _ in range(2)]

    def step_e2e(i):
        return hb.hom_bounds(solver.ctx, problem, opts_e2e, wss[i % 2].data_ptr(), nbytes, s_ptr)
    for i in range(2):
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

    line = {
        "metric": METRIC, "value": ms_step, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == hb.HOM_FP64 else "f32+f32x2+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.workload == "spheres3d_N113" else WORKLOADS[args.workload],
                   "precision": args.precision, "tol": TOL,
                   "l2": "flushed between steps (256 MiB write, outside the timed region)",
                   "launch": "CG iterations in blocks of 8 replayed from captured CUDA graphs",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "bounds": {"upper": out["upper"].tolist(), "lower": out["lower"].tolist()},
        "iters": out["report"]["iters"], "matvecs": out["report"]["matvecs"],
        "gpu_launches": launches,
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": rep["h2d_bytes"],
                "d2h_bytes_per_step": rep["d2h_bytes"],
                "note": "hom_bounds wall clock: host problem in (tables uploaded every step, two workspaces "
                        "alternating), host bounds out"},
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.headline_only:
        line.update(extras(args, hb, solver, problem, prec, dev, stream, flush, peaks, ms_step))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        _, info = oracle_sample(problem, reference_iters(problem, args.workload))
        line["cpu_baseline"] = info
    barrier(world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def extras(args, hb, solver, problem, prec, dev, stream, flush, peaks, ms_step):
    """Everything the line reports beside the headline (rank 0, after the timed region)."""
    import numpy as np
    s_ptr = stream.cuda_stream
    res = {}
    # plain FP64 CG on the same cell (the metric's comparison)
    other = hb.HOM_FP64 if prec == hb.HOM_MIXED else hb.HOM_MIXED
    solver(problem, precision=other, tol=TOL, stream=s_ptr)
    ts, oo = timed_steps(stream, flush, lambda: solver(problem, precision=other, tol=TOL, stream=s_ptr),
                         args.fp64_steps)
    res["alt_precision"] = {"precision": "fp64" if other == hb.HOM_FP64 else "mixed", "ms": statistics.mean(ts),
                            "steps": len(ts), "iters": oo["report"]["iters"],
                            "upper": oo["upper"].tolist(), "lower": oo["lower"].tolist()}
    if other == hb.HOM_FP64:
        res["alt_precision"]["mixed_speedup_vs_fp64"] = statistics.mean(ts) / ms_step
    # kernel families of one step (separate, instrumented steps: the timed steps carry no events)
    fam_ms = {}
    for fam in ("slab", "xpass", "ypass", "zpass", "final", "cg", "coef", "energy"):
        hb.hom_profile_kernel(solver.ctx, fam)
        solver(problem, precision=prec, tol=TOL, stream=s_ptr)
        n, ms = hb.hom_kernel_timing(solver.ctx)
        fam_ms[fam] = {"launches": n, "ms": ms}
    hb.hom_profile_kernel(solver.ctx, "")
    res["kernel_families_one_step"] = fam_ms
    # the operator: one application on d fields per precision; the slab pass timed per launch
    mv = matvec_timings(hb, solver, problem, dev, stream, reps=20, profile="slab")
    res["matvec"] = mv
    # measured FMA peaks (the denominators of the ALU-bound passes)
    p32 = hb.binding.hom_peak_probe(solver.ctx, hb.HOM_FP32, s_ptr)
    p64 = hb.binding.hom_peak_probe(solver.ctx, hb.HOM_FP64, s_ptr)
    res["fma_peaks_tflops"] = {"fp32": p32, "fp64": p64, "how": "hom_peak_probe: 8 FMA chains per thread, "
                               "4 x 512 threads per SM, best of 5"}
    # roofline of the dominant kernel of the step
    dom = max(fam_ms, key=lambda f: fam_ms[f]["ms"])
    res["dominant_family"] = dom
    f32 = mv.get("fp32", {})
    if problem.d == 3 and f32.get("profiled_launch_ms"):
        byt = slab_model_bytes(problem, 4, problem.d)
        ms_l = f32["profiled_launch_ms"]
        achieved = byt / (ms_l * 1e-3) / 1e9
        res["roofline"] = {
            "bound": "hbm", "kernel": "k_slab<float,15>", "achieved": achieved, "peak": peaks["hbm_gbs"],
            "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": slab_traffic(),
            "algorithmic_bytes_per_launch": byt, "avg_launch_ms": ms_l, "launches_timed": f32["profiled_launches"],
            "peak_note": peaks["source"],
            "bytes_note": "passes 2-4 of the unfused 5-pass operator model (inverse y with padding, x rows with "
                          "the coefficient, forward y with truncation) for 9 field components + one coefficient "
                          "read per right-hand side; the fused kernel keeps the double-grid slab on chip, so "
                          "its DRAM traffic is far below these bytes",
            "fft_tflops": slab_flops(problem, problem.d) / (ms_l * 1e-3) / 1e12,
            "fp32_fma_peak_tflops": p32,
            "operator_3field_ms": f32["ms"], "operator_model_frac": f32["model_hbm_frac"]}
    # the 3D cube cell (FP64 plain CG and mixed)
    if not args.no_cube:
        cube = workload("cube3d_N41")
        cres = {"workload": CUBE_WORKLOAD}
        for name, pr in (("fp64", hb.HOM_FP64), ("mixed", hb.HOM_MIXED)):
            solver(cube, precision=pr, tol=TOL, stream=s_ptr)
            ts, oc = timed_steps(stream, flush, lambda: solver(cube, precision=pr, tol=TOL, stream=s_ptr), 5)
            cres[name] = {"ms": statistics.mean(ts), "iters": oc["report"]["iters"],
                          "upper_11": float(oc["upper"][0, 0]), "lower_11": float(oc["lower"][0, 0])}
        res["cube3d_N41"] = cres
    if not args.no_batched:
        res["batched"] = batched_timings(hb, solver, dev)
    if args.image:
        res["image"] = image_timings(hb, solver, stream, flush)
    return res


def batched_timings(hb, solver, dev, n=256, reps=3, autotune=1):
    """The batched workload: n seeded random-rectangle 2D cells (N from {23, 63, 113, 203}),
    FP32 inner CG / FP64 bounds, tol 1e-4, one persistent launch replayed as a CUDA graph
    after an autotuning pass (threads per CTA, chunk capacity, radix schedule, cluster size
    for the largest cells); against plain FP64 hom_bounds one cell at a time on the same
    GPU, all n cells, wall clock."""
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
    for p in probs[:4]:                      # warm: plans and graphs of the four grid sizes
        solver(p, precision=hb.HOM_FP64, tol=TOL)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for p in probs:
        solver(p, precision=hb.HOM_FP64, tol=TOL)
    torch.cuda.synchronize()
    seq_ms = (time.perf_counter() - t) * 1e3
    return {"workload": f"{n} random-rectangle 2D cells, N from {{23,63,113,203}}, FP32 inner CG, FP64 bounds, tol {TOL:g}",
            "ms": ms_batch, "problems_per_s": n / (ms_batch * 1e-3), "launches": out["report"]["launches"],
            "launch_config": out["report"]["config"],
            "max_iters": int(out["iters"].max()), "status_nonzero": int((out["status"] != 0).sum()),
            "sequential_fp64_ms": seq_ms, "speedup_vs_sequential_fp64": seq_ms / ms_batch,
            "sequential_note": f"plain FP64 hom_bounds per cell, all {n} cells one after another, wall clock"}


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


def slab_model_bytes(problem, elem_bytes: int, nrhs: int) -> float:
    """Algorithmic bytes of one slab launch (3D): passes 2-4 of the operator model (inverse y
    with zero padding, x rows with the coefficient, forward y with truncation) for nrhs x d
    field components, each pass reading and writing its input and output once, plus one
    coefficient read per right-hand side."""
    N = [int(n) for n in problem.N]
    M = [2 * n - 1 for n in N]
    Nh = (N[0] + 1) // 2
    per = Nh * (2 * M[2] * N[1] + 4 * M[2] * M[1])
    return nrhs * problem.d * per * 2 * elem_bytes + nrhs * M[0] * M[1] * M[2] * elem_bytes


def slab_flops(problem, nrhs: int) -> float:
    return family_flops_per_launch(problem, "slab", nrhs)


def matvec_timings(hb, solver, problem, dev, stream, reps=20, precisions=("fp64", "ff", "fp32"), profile=None):
    """Device time of one operator application on d fields, FP64, float-float (FP64 fields,
    the residual arithmetic of the mixed refinement) and FP32; with `profile` a kernel
    family, its FP32 launches are timed too (in separate, instrumented applications)."""
    import torch
    ctx = solver.ctx
    info = hb.hom_problem_info(ctx, problem)
    d = problem.d
    nws = hb.hom_step_workspace_size(ctx, problem, d)
    ws = torch.empty(nws, dtype=torch.uint8, device=dev)
    shape = (d, d, int(problem.N[2]), int(problem.N[1]), (int(problem.N[0]) + 1) // 2)
    out = {}
    for name, prec, cdt, rdt in (("fp64", hb.HOM_FP64, torch.complex128, torch.float64),
                                 ("ff", hb.HOM_FF, torch.complex128, torch.float32),
                                 ("fp32", hb.HOM_FP32, torch.complex64, torch.float32)):
        if name not in precisions:
            continue
        coef = torch.empty((info["ncomp"],) + tuple(info["M"][::-1]) + ((2,) if name == "ff" else ()), dtype=rdt,
                           device=dev)
        hb.hom_coefficient(ctx, problem, 0, prec, coef.data_ptr(), ws.data_ptr(), nws, stream.cuda_stream)
        x = torch.randn(shape, dtype=cdt, device=dev)
        y = torch.empty_like(x)

        def apply():
            hb.hom_matvec(ctx, problem, 0, prec, 1, d, coef.data_ptr(), x.data_ptr(), y.data_ptr(),
                          ws.data_ptr(), nws, stream.cuda_stream)
        for _ in range(3):
            apply()
        n_rep = reps if name == "fp32" else max(3, reps // 6)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n_rep):
            apply()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / n_rep
        flops = sum(family_flops_per_launch(problem, f, d) * (2 if f == "ypass" else 1)
                    for f in ("zpass", "ypass", "xpass", "final"))
        nbytes = matvec_bytes(problem, 4 if name == "fp32" else 8)
        gbs = nbytes / (ms * 1e-3) / 1e9
        hbm = measured_peaks()["hbm_gbs"]
        out[name] = {"ms": ms, "matvecs_per_s": 1e3 / ms, "fft_tflops": flops / (ms * 1e-3) / 1e12, "fields": d,
                     "model_bytes": nbytes, "model_gbs": gbs, "model_hbm_frac": gbs / hbm}
        if profile and name == "fp32":
            hb.hom_profile_kernel(ctx, profile)
            for _ in range(n_rep):
                apply()
            torch.cuda.synchronize()
            n, tot = hb.hom_kernel_timing(ctx)
            hb.hom_profile_kernel(ctx, "")
            if n:
                out[name]["profiled_family"] = profile
                out[name]["profiled_launches"] = n
                out[name]["profiled_launch_ms"] = tot / n
    return out


def run_peak_probe(args):
    """The FMA peak probe alone, with the clocks sampled while it runs."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1404_3614_gb300 as hb
    ctx = hb.hom_create(0)
    s = torch.cuda.current_stream().cuda_stream
    with ClockSampler(0) as clk:
        r = {"fp32_tflops": [hb.binding.hom_peak_probe(ctx, hb.HOM_FP32, s) for _ in range(5)],
             "fp64_tflops": [hb.binding.hom_peak_probe(ctx, hb.HOM_FP64, s) for _ in range(5)]}
    hb.hom_destroy(ctx)
    r["clocks"] = clk.summary()
    print(json.dumps({"fma_peak_probe": r}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed steps of the other precision")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-cube", action="store_true")
    ap.add_argument("--image", action="store_true", help="add the 1199^2 pixel-image timings")
    ap.add_argument("--headline-only", action="store_true", help="only the timed steps and e2e")
    ap.add_argument("--workload", default="spheres3d_N113", choices=sorted(WORKLOADS))
    ap.add_argument("--matvec-only", action="store_true", help="operator applications only")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--matvec-precision", default="", choices=["", "fp64", "ff", "fp32"],
                    help="with --matvec-only: that arithmetic alone (default: the inner solves' FP32, or FP64)")
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
    ap.add_argument("--peak-probe", action="store_true", help="the FMA peak probe alone, with clocks")
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
    if args.peak_probe:
        return run_peak_probe(args)
    if args.paper_grids:
        return run_paper_grids(args)
    if args.even_grids:
        return run_even_grids(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
