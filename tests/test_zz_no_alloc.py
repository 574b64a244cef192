"""hom_matvec_noalloc: the operator for callers that cannot allocate device memory.

Such callers (code whose device memory is owned and capped by another allocator, or
loops that must not allocate) cannot provide the workspace hom_matvec takes; this entry
point uses a scratch array that lives inside the library instead. The test checks it
through the C ABI against hom_matvec on the same inputs, within the tolerances of the
other operator tests, on two calls in a row, and that an oversized problem is refused. It
also checks the promise itself: once every kernel has been loaded by a first call, later
calls, alternating between two problems whose tables must be uploaded again each time,
leave both torch's allocated bytes and the device's free memory unchanged.
The file name makes pytest collect it last.
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


@pytest.fixture(scope="module")
def ctx(hb):
    c = hb.hom_create(0)
    yield c
    hb.hom_destroy(c)


CASES = [
    ("aniso2d_N23", lambda: ms.random_anisotropic_2d(8, N=23)),
    ("spheres3d_N9", lambda: ms.random_spheres_3d(3, N=9, n_balls=4, phi=0.2, contrast=50.0)),
    ("cube3d_N41", lambda: ms.cube_inclusion_3d()),
]


@pytest.mark.parametrize("name,maker", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_workspace_matvec(hb, ctx, name, maker, prec):
    p = maker()
    d = p.d
    info = hb.hom_problem_info(ctx, p)
    nws = hb.hom_step_workspace_size(ctx, p, d)
    ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
    hp = hb.HOM_FP64 if prec == "fp64" else hb.HOM_FP32
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    rdt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 5e-6
    gen = torch.Generator(device="cuda").manual_seed(5)
    shape = (d, d) + ((int(p.N[2]),) if d == 3 else ()) + (int(p.N[1]), (int(p.N[0]) + 1) // 2)
    for side in (0, 1):
        coef = torch.empty((info["ncomp"],) + tuple(info["M"][:d][::-1]), dtype=rdt, device="cuda")
        hb.hom_coefficient(ctx, p, side, hp, coef.data_ptr(), ws.data_ptr(), nws)
        for project in (1, 0):
            x = torch.randn(shape, dtype=cdt, device="cuda", generator=gen)
            ref = torch.empty_like(x)
            hb.hom_matvec(ctx, p, side, hp, project, d, coef.data_ptr(), x.data_ptr(), ref.data_ptr(),
                          ws.data_ptr(), nws)
            for _call in range(2):                      # two calls in a row share the scratch
                out = torch.full_like(x, float("nan"))
                hb.binding.hom_matvec_noalloc(ctx, p, side, hp, project, d, coef.data_ptr(), x.data_ptr(),
                                      out.data_ptr())
                torch.cuda.synchronize()
                a, b = out.cpu().numpy(), ref.cpu().numpy()
                err = np.abs(a - b).max() / np.abs(b).max()
                assert np.isfinite(a).all() and err <= tol, (name, prec, side, project, err)


def test_noalloc_rejects_problems_beyond_the_scratch(hb, ctx):
    p = ms.cube_inclusion_3d(N=101)          # double grid 201^3: far more than 32 MiB of scratch
    info = hb.hom_problem_info(ctx, p)
    one = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(hb.HombError) as e:
        hb.binding.hom_matvec_noalloc(ctx, p, 0, hb.HOM_FP64, 1, 3, one.data_ptr(), one.data_ptr() + 0,
                                      one.data_ptr() + 8)
    assert e.value.status == hb.binding.HOM_ERR_WORKSPACE
    assert "static scratch" in hb.hom_last_error(ctx)
    assert info["grid_elems"] == 201 ** 3


def test_noalloc_allocates_nothing_across_alternating_problems(hb, ctx):
    probs = [ms.random_anisotropic_2d(8, N=23), ms.cube_inclusion_3d(N=13)]
    prep = []
    for p in probs:
        d = p.d
        info = hb.hom_problem_info(ctx, p)
        nws = hb.hom_step_workspace_size(ctx, p, d)
        ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
        coef = torch.empty((info["ncomp"],) + tuple(info["M"][:d][::-1]), dtype=torch.float64, device="cuda")
        hb.hom_coefficient(ctx, p, 0, hb.HOM_FP64, coef.data_ptr(), ws.data_ptr(), nws)
        shape = (d, d) + ((int(p.N[2]),) if d == 3 else ()) + (int(p.N[1]), (int(p.N[0]) + 1) // 2)
        x = torch.randn(shape, dtype=torch.complex128, device="cuda")
        ref = torch.empty_like(x)
        hb.hom_matvec(ctx, p, 0, hb.HOM_FP64, 1, d, coef.data_ptr(), x.data_ptr(), ref.data_ptr(), ws.data_ptr(), nws)
        out = torch.empty_like(x)
        prep.append((p, coef, x, ref, out))
    # first calls: the scratch address lookup and the first launch of each kernel
    for p, coef, x, ref, out in prep:
        hb.binding.hom_matvec_noalloc(ctx, p, 0, hb.HOM_FP64, 1, p.d, coef.data_ptr(), x.data_ptr(), out.data_ptr())
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    for rep in range(3):
        for p, coef, x, ref, out in prep:
            out.fill_(float("nan"))
            hb.binding.hom_matvec_noalloc(ctx, p, 0, hb.HOM_FP64, 1, p.d, coef.data_ptr(), x.data_ptr(),
                                          out.data_ptr())
            torch.cuda.synchronize()
            a, b = out.cpu().numpy(), ref.cpu().numpy()
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), (rep, p.d)
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
