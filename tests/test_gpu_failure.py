"""Failure detection through the C ABI, in the forms that fault no GPU.

* The tensor-core GEMM's bounded wait on its completion barrier: a test aid limits the
  polls so the wait gives up at once; the kernel records the timeout in the context's flag,
  drains its committed MMAs, frees its tensor memory and returns; the call returns
  HOM_ERR_TIMEOUT. The same context then computes the right result with the default limit,
  and another context never sees the first one's timeout.
* CG breakdown from host-made bad input: a starting field holding a NaN, given to
  hom_bounds_io (FP64 and mixed) and to the batched launch, returns HOM_ERR_BREAKDOWN (a
  per-cell status in the batch) instead of bounds, and the context stays usable.
"""
import numpy as np
import pytest

import microstructures as ms

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hb():
    import paper_1404_3614_gb300 as hb
    return hb


def gemm(hb, ctx, A, B):
    M, K = A.shape
    N = B.shape[1]
    C = torch.full((M, N), float("nan"), device="cuda")
    hb.binding.hom_gemm_bf16(ctx, M, N, K, A.data_ptr(), K, 0, B.data_ptr(), N, 0, C.data_ptr(), N, 1.0, 0.0)
    return C


def test_gemm_wait_timeout_returns_status_and_context_recovers(hb):
    ctx = hb.hom_create(0)
    other = hb.hom_create(0)
    try:
        g = torch.Generator(device="cuda").manual_seed(0)
        A = torch.randn((4096, 256), generator=g, device="cuda")
        B = torch.randn((256, 64), generator=g, device="cuda")
        ref = A.bfloat16().double() @ B.bfloat16().double()
        hb.binding.hom_set_gemm_spin_limit(ctx, 1)
        for _ in range(2):
            with pytest.raises(hb.HombError) as e:
                gemm(hb, ctx, A, B)
            assert e.value.status == hb.binding.HOM_ERR_TIMEOUT
            assert "timed out" in hb.hom_last_error(ctx)
        # the other context's GEMMs are unaffected and do not inherit the timeout
        C = gemm(hb, other, A, B)
        assert (C.double() - ref).abs().max() <= 1e-3 * ref.abs().max()
        hb.binding.hom_set_gemm_spin_limit(ctx, 0)
        C = gemm(hb, ctx, A, B)
        torch.cuda.synchronize()
        assert (C.double() - ref).abs().max() <= 1e-3 * ref.abs().max()
    finally:
        hb.hom_destroy(ctx)
        hb.hom_destroy(other)


def test_network_forward_timeout(hb):
    ctx = hb.hom_create(0)
    try:
        cfg = hb.binding.net_config(N=15, cin=1, width=16, modes=4, layers=2, proj=32, cout=8)
        npar, wsb = hb.binding.hom_net_sizes(ctx, cfg, 4)
        params = torch.empty(npar, dtype=torch.float32, device="cuda")
        hb.binding.hom_net_init(ctx, cfg, 1, params.data_ptr())
        x = torch.randn((4, 15, 15, 1), device="cuda")
        y = torch.empty((4, 15, 15, 8), device="cuda")
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        hb.binding.hom_set_gemm_spin_limit(ctx, 1)
        with pytest.raises(hb.HombError) as e:
            hb.binding.hom_net_forward(ctx, cfg, params.data_ptr(), 4, x.data_ptr(), y.data_ptr(), ws.data_ptr(), wsb)
        assert e.value.status == hb.binding.HOM_ERR_TIMEOUT
        hb.binding.hom_set_gemm_spin_limit(ctx, 0)
        hb.binding.hom_net_forward(ctx, cfg, params.data_ptr(), 4, x.data_ptr(), y.data_ptr(), ws.data_ptr(), wsb)
        torch.cuda.synchronize()
        assert torch.isfinite(y).all()
    finally:
        hb.hom_destroy(ctx)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nan_start_breaks_down(hb, precision):
    solver = hb.Bounds(0)
    try:
        p = ms.cube_inclusion_3d(N=9)
        prec = hb.HOM_FP64 if precision == "fp64" else hb.HOM_MIXED
        shape = (2, 3, 3, 9, 9, 5)
        x0 = torch.zeros(shape, dtype=torch.complex128, device="cuda")
        x0[0, 1, 0, 2, 3, 1] = complex(float("nan"), 0.0)          # one poisoned coefficient
        with pytest.raises(hb.HombError) as e:
            solver(p, precision=prec, tol=1e-8, x0=x0)
        assert e.value.status == hb.binding.HOM_ERR_BREAKDOWN
        good = solver(p, precision=prec, tol=1e-8, x0=torch.zeros_like(x0))
        assert np.isfinite(good["upper"]).all() and np.isfinite(good["lower"]).all()
    finally:
        solver.close()


def test_nan_start_in_a_batch_marks_only_that_cell(hb):
    """The batched launch reports a breakdown per cell (status -2, the call returns a
    warning): the other cells of the same launch keep their bounds."""
    solver = hb.Bounds(0)
    try:
        probs = [ms.square_inclusion_2d(N=9), ms.random_rectangles_2d(3, N=9), ms.laminate_2d(9)]
        x0 = torch.zeros((3, 2, 2, 2, 9, 5), dtype=torch.complex128, device="cuda")
        clean = solver.batched(probs, precision=hb.HOM_FP64, tol=1e-10, x0=x0)
        x0[1, 0, 0, 1, 2, 1] = complex(float("nan"), 0.0)
        out = solver.batched(probs, precision=hb.HOM_FP64, tol=1e-10, x0=x0)
        assert out["code"] == hb.binding.HOM_WARN_NOT_CONVERGED
        assert list(out["status"]) == [0, -2, 0]
        assert "broke down" in hb.hom_last_error(solver.ctx)
        for i in (0, 2):
            assert np.array_equal(out["upper"][i], clean["upper"][i])
        x0.zero_()
        out = solver.batched(probs, precision=hb.HOM_FP64, tol=1e-10, x0=x0)
        assert (out["status"] == 0).all()
    finally:
        solver.close()
