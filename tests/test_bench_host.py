"""Host-side logic of bench.py (no GPU): the oracle iteration counts it extrapolates
with, the FLOP model, and the max-over-ranks reduction on 2 gloo ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench
import microstructures as ms
from oracle import matfree


def test_oracle_iteration_counts_pinned():
    """bench.ORACLE_ITERS are the oracle CG's own iteration counts at 1e-4 on the cube cell (E = e1)."""
    p = bench.workload("cube3d_N41")
    for side in ("primal", "dual"):
        op = matfree.MatFreeOperator(p, side)
        _, it, res = matfree.cg_solve(op, [1.0, 0.0, 0.0], tol=bench.TOL)
        assert it == bench.ORACLE_ITERS[side] and res <= bench.TOL


def test_traffic_reported_only_for_the_captured_kernel(monkeypatch):
    """The ncu DRAM figure is tied to the slab-pass sources it was captured on."""
    monkeypatch.setitem(bench.SLAB_TRAFFIC, "sha256_16", "0" * 16)
    monkeypatch.setitem(bench.SLAB_TRAFFIC, "bytes", 123)
    assert bench.slab_traffic() is None
    monkeypatch.setitem(bench.SLAB_TRAFFIC, "sha256_16", bench.source_hash(bench.SLAB_TRAFFIC["sources"]))
    assert bench.slab_traffic() == 123


def test_reference_arm_uses_the_oracles_own_iteration_counts():
    """The oracle arm extrapolates the 16-ball cell with the oracle CG's own iteration counts to
    1e-4, read off the residual history of the full-size golden run (equal to the GPU's FP64
    counts on this cell)."""
    it = bench.oracle_iters_c5()
    assert it is not None
    assert it == {"primal": [176, 176, 176], "dual": [49, 51, 49]}
    assert bench.reference_iters(bench.workload("spheres3d_N113"), "spheres3d_N113") == it


def test_slab_byte_model():
    """Passes 2-4 of the 5-pass model on the 16-ball cell (N = 113, M = 225, Nh = 57), 9 FP32
    field components and 3 coefficient reads."""
    p = bench.workload("spheres3d_N113")
    want = 9 * 57 * (2 * 225 * 113 + 4 * 225 * 225) * 8 + 3 * 225 ** 3 * 4
    assert bench.slab_model_bytes(p, 4, 3) == want
    # with passes 1 and 5 (the z transforms) it is the whole-operator model
    z = 9 * 57 * (2 * 113 * 113 + 2 * 225 * 113) * 8
    assert bench.matvec_bytes(p, 4) == want + z


def test_oracle_sample_extrapolates_a_bounded_sample():
    p = ms.cube_inclusion_3d(N=9)
    est, info = bench.oracle_sample(p, {"primal": 5, "dual": 3}, n_matvec=1)
    assert est > 0 and info["extrapolated"] and info["kind"] == "oracle" and info["cores"] >= 1


def test_flop_model():
    p = ms.cube_inclusion_3d()
    assert bench.fft_flops(1) == 0.0
    assert bench.fft_flops(81) == pytest.approx(5 * 81 * np.log2(81))
    x = bench.family_flops_per_launch(p, "xpass", 3)
    assert x == pytest.approx(9 * 81 * 81 * bench.fft_flops(81))
    assert bench.family_flops_per_launch(p, "cg", 3) == 0.0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    v = bench.max_over_ranks(10.0 + rank * 3.5, world)
    bench.barrier(world)
    q.put((rank, v))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 13.5), (1, 13.5)]
