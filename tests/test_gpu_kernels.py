"""Step-level parity of the CUDA path against the CPU oracle (through the C ABI).

Each test runs a library entry point on seeded inputs and compares element by element
with the oracle (FP64: 1e-12 relative to the largest entry; FP32: 2e-6). The FFT is
checked against numpy's FFT, which is the textbook DFT up to rounding.
"""
import zlib

import numpy as np
import pytest

import microstructures as ms
from oracle import matfree

from layout import coef_to_dev, full_to_half, half_to_full, random_real_field

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


PROBLEMS = {
    "square2d_N9": lambda: ms.square_inclusion_2d(N=9),
    "aniso2d_N7": lambda: ms.random_anisotropic_2d(1, N=7),
    "aniso3d_N5": lambda: ms.random_anisotropic_3d(2, N=5),
    "cube3d_N7": lambda: ms.cube_inclusion_3d(N=7),
    "rect2d_N11": lambda: ms.random_rectangles_2d(5, N=11),
    "spheres3d_N9": lambda: ms.random_spheres_3d(1, N=9, n_balls=4, phi=0.2, contrast=50.0),
    "aniso2d_N13_rect": lambda: ms.make_problem(2, (13, 9), (1.0, 0.7), np.array([[2.0, 0.3], [0.3, 1.0]]),
                                                 [ms.box((0.1, 0.05), (0.3, 0.2), 7.0, 2),
                                                  ms.ball((-0.25, -0.2), 0.12, 0.2, 2)]),
    # grids whose double grid has a compile-time specialised FFT length (45, 81, 125, 225, 405)
    "rect2d_N63_M125": lambda: ms.random_rectangles_2d(21, N=63),
    "rect2d_N113_M225": lambda: ms.random_rectangles_2d(22, N=113),
    "aniso2d_N203x41_M405x81": lambda: ms.make_problem(2, (203, 41), (1.0, 0.5), np.array([[1.5, 0.2], [0.2, 0.8]]),
                                                       [ms.box((0.0, 0.1), (0.4, 0.2), 9.0, 2)]),
    "cube3d_N23_M45": lambda: ms.cube_inclusion_3d(N=23),
    # isotropic 3D cells with M = R^2 on x and y: the fused y-x-y slab pass
    "spheres3d_N5_M9": lambda: ms.random_spheres_3d(3, N=5, n_balls=3, phi=0.2, contrast=20.0),
    "cube3d_N13_M25": lambda: ms.cube_inclusion_3d(N=13),
    "spheres3d_N41_M81": lambda: ms.random_spheres_3d(4, N=41, n_balls=6, phi=0.25, contrast=100.0),
    # double-grid length 225 along z only: the persistent pipelined z passes (FP32) with ragged
    # last chunks (55 positions per z plane), the separate y and x passes
    "balls3d_N9x11x113_Mz225": lambda: ms.make_problem(3, (9, 11, 113), (1.0, 0.8, 1.2), 1.0,
                                                       [ms.ball((0.1, 0.0, 0.05), 0.3, 30.0, 3),
                                                        ms.box((-0.3, 0.25, -0.4), (0.2, 0.2, 0.3), 0.1, 3)]),
}


@pytest.mark.parametrize("M", [1, 3, 5, 7, 9, 13, 15, 21, 37, 45, 73, 81, 125, 225, 405, 243, 343, 2, 8, 12, 34, 64])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fft_matches_numpy(hb, ctx, M, prec):
    rng = np.random.default_rng(M)
    howmany = 37
    x = rng.normal(size=(howmany, M)) + 1j * rng.normal(size=(howmany, M))
    dt = np.complex128 if prec == "fp64" else np.complex64
    p = hb.HOM_FP64 if prec == "fp64" else hb.HOM_FP32
    xin = dev(x.astype(dt))
    ws = torch.empty(16 * M + 256, dtype=torch.uint8, device="cuda")
    for direction, ref in ((-1, np.fft.fft(x, axis=1)), (1, np.fft.ifft(x, axis=1) * M)):
        out = torch.empty_like(xin)
        hb.hom_fft(ctx, M, p, direction, howmany, xin.data_ptr(), out.data_ptr(), ws.data_ptr(), ws.numel())
        torch.cuda.synchronize()
        tol = 1e-13 if prec == "fp64" else 3e-6
        assert relerr(out.cpu().numpy(), ref) < tol * max(1.0, np.log2(M))


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("side", [0, 1])
def test_coefficient_matches_oracle(hb, ctx, name, side):
    p = PROBLEMS[name]()
    info = hb.hom_problem_info(ctx, p)
    op = matfree.MatFreeOperator(p, "primal" if side == 0 else "dual")
    ref = coef_to_dev(op.A_grid, p.d, info["ncomp"] == 1)
    nws = hb.hom_step_workspace_size(ctx, p, 1)
    ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
    for prec, dt, tol in ((hb.HOM_FP64, torch.float64, 1e-13), (hb.HOM_FP32, torch.float32, 1e-6)):
        coef = torch.empty(ref.size, dtype=dt, device="cuda")
        hb.hom_coefficient(ctx, p, side, prec, coef.data_ptr(), ws.data_ptr(), nws)
        torch.cuda.synchronize()
        got = coef.cpu().numpy().astype(np.float64).reshape(ref.shape)
        assert relerr(got, ref) < tol, (name, side, prec)


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("side", [0, 1])
def test_rhs_matches_oracle(hb, ctx, name, side):
    p = PROBLEMS[name]()
    d = p.d
    op = matfree.MatFreeOperator(p, "primal" if side == 0 else "dual")
    nws = hb.hom_step_workspace_size(ctx, p, d)
    ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
    refs = [full_to_half(-op.apply(op.constant_field(np.eye(d)[a])), d) for a in range(d)]
    ref = np.stack(refs)
    for prec, dt, tol in ((hb.HOM_FP64, torch.complex128, 1e-12), (hb.HOM_FP32, torch.complex64, 2e-6)):
        b = torch.empty(ref.shape, dtype=dt, device="cuda")
        hb.hom_rhs(ctx, p, side, prec, d, b.data_ptr(), ws.data_ptr(), nws)
        torch.cuda.synchronize()
        assert relerr(b.cpu().numpy().astype(np.complex128), ref) < tol, (name, side, prec)


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("project", [0, 1])
def test_matvec_matches_oracle(hb, ctx, name, side, project):
    p = PROBLEMS[name]()
    d = p.d
    N = tuple(int(n) for n in p.N)
    rng = np.random.default_rng([zlib.crc32(name.encode()), side, project])
    op = matfree.MatFreeOperator(p, "primal" if side == 0 else "dual")
    info = hb.hom_problem_info(ctx, p)
    nws = hb.hom_step_workspace_size(ctx, p, d)
    ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
    fields = [random_real_field(rng, d, N) for _ in range(d)]
    ref = np.stack([full_to_half(op.apply(u, project=bool(project)), d) for u in fields])
    uin = np.stack([full_to_half(u, d) for u in fields])
    # HOM_FF: float-float arithmetic (about 48 bits) between FP64 input and output, the
    # coefficient as (hi, lo) float pairs; its bar is FP64's
    for prec, cdt, rdt, tol in ((hb.HOM_FP64, torch.complex128, torch.float64, 1e-12),
                                (hb.HOM_FF, torch.complex128, torch.float32, 1e-12),
                                (hb.HOM_FP32, torch.complex64, torch.float32, 5e-6)):
        cshape = (info["ncomp"],) + tuple(info["M"][:d][::-1]) + ((2,) if prec == hb.HOM_FF else ())
        coef = torch.empty(cshape, dtype=rdt, device="cuda")
        hb.hom_coefficient(ctx, p, side, prec, coef.data_ptr(), ws.data_ptr(), nws)
        x = dev(uin.astype(np.complex128)).to(cdt)
        y = torch.zeros_like(x)
        hb.hom_matvec(ctx, p, side, prec, project, d, coef.data_ptr(), x.data_ptr(), y.data_ptr(),
                      ws.data_ptr(), nws)
        torch.cuda.synchronize()
        got = y.cpu().numpy().astype(np.complex128)
        assert relerr(got, ref) < tol, (name, side, project, prec, relerr(got, ref))
        # and the full Hermitian field agrees too
        if prec == hb.HOM_FP64:
            full = np.stack([half_to_full(g, d, N[0]) for g in got])
            reff = np.stack([op.apply(u, project=bool(project)) for u in fields])
            assert relerr(full, reff) < 1e-12


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("add_constant", [0, 1])
def test_energy_matches_oracle(hb, ctx, name, add_constant):
    p = PROBLEMS[name]()
    d = p.d
    N = tuple(int(n) for n in p.N)
    rng = np.random.default_rng(7)
    info = hb.hom_problem_info(ctx, p)
    nws = hb.hom_step_workspace_size(ctx, p, d)
    ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
    for side in (0, 1):
        op = matfree.MatFreeOperator(p, "primal" if side == 0 else "dual")
        fields = [random_real_field(rng, d, N) for _ in range(d)]
        if add_constant:
            ofields = [op.constant_field(np.eye(d)[a]) + fields[a] for a in range(d)]
        else:
            ofields = fields
        ref = op.energy_matrix(ofields)
        coef = torch.empty((info["ncomp"],) + tuple(info["M"][:d][::-1]), dtype=torch.float64, device="cuda")
        hb.hom_coefficient(ctx, p, side, hb.HOM_FP64, coef.data_ptr(), ws.data_ptr(), nws)
        x = dev(np.stack([full_to_half(u, d) for u in fields]))
        W = hb.hom_energy(ctx, p, d, add_constant, coef.data_ptr(), x.data_ptr(), ws.data_ptr(), nws)
        assert relerr(W, ref) < 1e-12, (name, side, W, ref)


def test_invalid_inputs_rejected(hb, ctx):
    p = ms.square_inclusion_2d(N=5).with_N(0)
    with pytest.raises(hb.HombError) as e:
        hb.hom_problem_info(ctx, p)
    assert e.value.status == hb.binding.HOM_ERR_INVALID_ARG
    # even grids are general grids: FP64 only
    p8 = ms.square_inclusion_2d(N=8)
    hb.hom_problem_info(ctx, p8)
    nws = hb.hom_step_workspace_size(ctx, p8, 2)
    wsb = torch.empty(nws, dtype=torch.uint8, device="cuda")
    b = torch.empty((2, 2, 8, 4), dtype=torch.complex64, device="cuda")
    with pytest.raises(hb.HombError):
        hb.hom_rhs(ctx, p8, 0, hb.HOM_FP32, 2, b.data_ptr(), wsb.data_ptr(), nws)
    q = ms.make_problem(2, 5, 1.0, 1.0, [ms.box(0.0, 0.4, 2.0, 2), ms.box(0.1, 0.4, 3.0, 2)])
    with pytest.raises(hb.HombError):
        hb.hom_problem_info(ctx, q)
    r = ms.make_problem(3, 5, 1.0, 1.0, [ms.ball(0.0, 0.6, 2.0, 3)])
    with pytest.raises(hb.HombError):
        hb.hom_problem_info(ctx, r)
    s = ms.make_problem(2, 5, 1.0, np.array([[1.0, 2.0], [2.0, 1.0]]), [])
    with pytest.raises(hb.HombError):
        hb.hom_problem_info(ctx, s)
    # workspace too small
    p5 = ms.square_inclusion_2d(N=5)
    opts = hb.make_opts()
    n = hb.hom_workspace_size(ctx, p5, opts)
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    with pytest.raises(hb.HombError) as e:
        hb.hom_bounds(ctx, p5, opts, ws.data_ptr(), n - 1024)
    assert e.value.status == hb.binding.HOM_ERR_WORKSPACE


@pytest.mark.parametrize("N,prec", [(5, "fp32"), (13, "fp32"), (41, "fp32"), (113, "fp32"), (41, "fp64")])
def test_slab_pass_matches_separate_passes(hb, ctx, N, prec):
    """The fused y-x-y slab pass (FP32) and the three separate passes compute the same
    operator: equal to rounding (2e-6 relative to the largest entry) at M = 9, 25, 81, 225.
    FP64 always takes the separate passes: switching the slab pass makes no difference."""
    p = ms.random_spheres_3d(7, N=N, n_balls=5, phi=0.2, contrast=100.0)
    d = 3
    rng = np.random.default_rng([zlib.crc32(b"slab"), N])
    info = hb.hom_problem_info(ctx, p)
    nws = hb.hom_step_workspace_size(ctx, p, d)
    ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
    precision = hb.HOM_FP64 if prec == "fp64" else hb.HOM_FP32
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    rdt = torch.float64 if prec == "fp64" else torch.float32
    Nh = (N + 1) // 2
    x = torch.from_numpy(rng.normal(size=(d, d, N, N, Nh)) + 1j * rng.normal(size=(d, d, N, N, Nh))).to(cdt).cuda()
    out = {}
    try:
        for side in (0, 1):
            coef = torch.empty((info["ncomp"],) + tuple(info["M"][:d][::-1]), dtype=rdt, device="cuda")
            hb.hom_coefficient(ctx, p, side, precision, coef.data_ptr(), ws.data_ptr(), nws)
            # automatic, two fixed warp counts of the persistent kernel (different CTA counts and
            # slabs per CTA), and the separate passes
            variants = (1, 8, 20, 0) if N >= 41 and prec == "fp32" else (1, 0)
            for slab in variants:
                hb.hom_set_slab_pass(ctx, slab)
                y = torch.zeros_like(x)
                hb.hom_matvec(ctx, p, side, precision, 1, d, coef.data_ptr(), x.data_ptr(), y.data_ptr(),
                              ws.data_ptr(), nws)
                torch.cuda.synchronize()
                out[side, slab] = y.cpu().numpy()
            tol = 1e-13 if prec == "fp64" else 2e-6
            for slab in variants[:-1]:
                assert relerr(out[side, slab], out[side, 0]) < tol, (N, prec, side, slab,
                                                                     relerr(out[side, slab], out[side, 0]))
    finally:
        hb.hom_set_slab_pass(ctx, 1)


@pytest.mark.parametrize("name", ["balls3d_N9x11x113_Mz225", "spheres3d_N113"])
def test_pipe_passes_match_chunked_passes(hb, ctx, name):
    """The persistent pipelined FP32 z passes (length 225; each of the two, both, and the last
    pass with 16 positions per chunk) and the
    chunked passes compute the same operator (2e-6 relative to the largest entry) on both
    sides, with and without Gamma;
    through hom_bounds (mixed: the CG prologue p = r + beta p and the partial sums p.Cp) they
    give the same bounds to the solver's tolerance."""
    p = PROBLEMS[name]() if name in PROBLEMS else ms.random_spheres_3d(0, N=113)
    d = 3
    N = tuple(int(n) for n in p.N)
    rng = np.random.default_rng([zlib.crc32(name.encode()), 3])
    info = hb.hom_problem_info(ctx, p)
    nws = hb.hom_step_workspace_size(ctx, p, d)
    ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
    shape = (d, d, N[2], N[1], (N[0] + 1) // 2)
    x = torch.from_numpy(rng.normal(size=shape) + 1j * rng.normal(size=shape)).to(torch.complex64).cuda()
    try:
        for side in (0, 1):
            coef = torch.empty((info["ncomp"],) + tuple(info["M"][:d][::-1]), dtype=torch.float32, device="cuda")
            hb.hom_coefficient(ctx, p, side, hb.HOM_FP32, coef.data_ptr(), ws.data_ptr(), nws)
            for project in (0, 1):
                out = {}
                for pipe in (3, 2, 1, 5, 0):
                    hb.binding.hom_set_pipe_passes(ctx, pipe)
                    y = torch.full_like(x, float("nan"))
                    hb.hom_matvec(ctx, p, side, hb.HOM_FP32, project, d, coef.data_ptr(), x.data_ptr(),
                                  y.data_ptr(), ws.data_ptr(), nws)
                    torch.cuda.synchronize()
                    out[pipe] = y.cpu().numpy()
                for pipe in (3, 2, 1, 5):
                    assert np.isfinite(out[pipe]).all()
                    assert relerr(out[pipe], out[0]) < 2e-6, (name, side, project, pipe, relerr(out[pipe], out[0]))
        if name in PROBLEMS:
            solver = hb.Bounds(0)
            try:
                res = {}
                for pipe in (3, 0):
                    hb.binding.hom_set_pipe_passes(solver.ctx, pipe)
                    res[pipe] = solver(p, precision=hb.HOM_MIXED, tol=1e-7)
                for key in ("upper", "lower"):
                    assert relerr(res[3][key], res[0][key]) < 1e-6, key
            finally:
                solver.close()
    finally:
        hb.binding.hom_set_pipe_passes(ctx, 1)


@pytest.mark.parametrize("N,prec", [(41, "fp64"), (23, "fp64"), (41, "fp32")])
def test_pass_chunks_do_not_change_the_operator(hb, ctx, N, prec):
    """hom_set_pass_chunks only regroups pencils and planes into CTAs. The y-pass pencils keep
    their arithmetic; the row pass packs two real rows per complex FFT, and the partner row
    changes with the plane count, so results agree to rounding (1e-13 FP64, 2e-6 FP32)."""
    p = ms.random_spheres_3d(3, N=N, n_balls=5, phi=0.2, contrast=100.0)
    d = 3
    rng = np.random.default_rng([zlib.crc32(b"chunks"), N])
    info = hb.hom_problem_info(ctx, p)
    nws = hb.hom_step_workspace_size(ctx, p, d)
    ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
    precision = hb.HOM_FP64 if prec == "fp64" else hb.HOM_FP32
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    rdt = torch.float64 if prec == "fp64" else torch.float32
    Nh = (N + 1) // 2
    x = torch.from_numpy(rng.normal(size=(d, d, N, N, Nh)) + 1j * rng.normal(size=(d, d, N, N, Nh))).to(cdt).cuda()
    coef = torch.empty((info["ncomp"],) + tuple(info["M"][:d][::-1]), dtype=rdt, device="cuda")
    hb.hom_coefficient(ctx, p, 0, precision, coef.data_ptr(), ws.data_ptr(), nws)
    outs = []
    try:
        for yc, yb in ((0, 0), (1, 1), (3, 5), (7, 10), (100, 100)):
            hb.binding.hom_set_pass_chunks(ctx, yc, yb)
            y = torch.zeros_like(x)
            hb.hom_matvec(ctx, p, 0, precision, 1, d, coef.data_ptr(), x.data_ptr(), y.data_ptr(), ws.data_ptr(), nws)
            torch.cuda.synchronize()
            outs.append(y.cpu().numpy())
        tol = 1e-13 if prec == "fp64" else 2e-6
        for o in outs[1:]:
            assert relerr(o, outs[0]) < tol
        with pytest.raises(hb.HombError):
            hb.binding.hom_set_pass_chunks(ctx, -1, 0)
    finally:
        hb.binding.hom_set_pass_chunks(ctx, 0, 0)
