"""Whole-pipeline parity of hom_bounds against the oracle, and properties at full size.

FP64: upper and lower bounds within 1e-10 relative (Frobenius-scaled max entry error)
of the dense oracle (the Galerkin definition) on small grids; mixed precision (FP32
inner CG, FP64 re-projection and energies) within 1e-6 with lower <= upper kept.
The full-size 3D N = 41 cube cell is checked on sampled operator rows (computed one
by one by the oracle from the Fourier convolution of Lemma Ga_full) and on the
properties that hold at any size.
"""
import numpy as np
import pytest

import microstructures as ms
import oracle
from oracle import matfree

from layout import full_to_half, half_to_full, random_real_field

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hb():
    import paper_1404_3614_gb300 as hb
    return hb


@pytest.fixture(scope="module")
def solver(hb):
    s = hb.Bounds(0)
    yield s
    s.close()


def rel(a, b):
    return np.abs(a - b).max() / np.linalg.norm(b)


def loewner_ge(A, B, tol=1e-12):
    S = 0.5 * ((A - B) + (A - B).T)
    return np.linalg.eigvalsh(S).min() >= -tol * max(1.0, np.abs(A).max())


CASES = {
    "square2d_N9": lambda: ms.square_inclusion_2d(N=9),
    "square2d_N23": lambda: ms.square_inclusion_2d(N=23),
    "paper_rho1000_N15": lambda: ms.paper_square_2d(15, 1000.0),
    "aniso2d_N9": lambda: ms.random_anisotropic_2d(3, N=9),
    "aniso3d_N5": lambda: ms.random_anisotropic_3d(4, N=5),
    "cube3d_N7": lambda: ms.cube_inclusion_3d(N=7),
    "rect2d_N15": lambda: ms.random_rectangles_2d(11, N=15),
    "spheres3d_N7": lambda: ms.random_spheres_3d(2, N=7, n_balls=6, phi=0.25, contrast=30.0),
    "laminate_N11": lambda: ms.laminate_2d(11),
    "homogeneous3d": lambda: ms.homogeneous(3, 5, np.array([[2.0, 0.1, 0.0], [0.1, 1.5, 0.2], [0.0, 0.2, 1.0]])),
    "N1_voigt_reuss": lambda: ms.random_anisotropic_2d(5, N=1),
}


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_bounds_match_dense_oracle(hb, solver, name):
    p = CASES[name]()
    ref = oracle.dense_bounds(p)
    out = solver(p, precision=hb.HOM_FP64, tol=1e-12)
    for key in ("upper", "lower", "mean", "D"):
        scale = np.linalg.norm(ref["upper"])
        assert np.abs(out[key] - ref[key]).max() <= 1e-10 * scale, (name, key, out[key], ref[key])
    assert out["status"] == 0


@pytest.mark.parametrize("name", [n for n in CASES if n != "homogeneous3d"])
def test_mixed_bounds_within_1e6_and_ordered(hb, solver, name):
    p = CASES[name]()
    ref = oracle.dense_bounds(p)
    out = solver(p, precision=hb.HOM_MIXED, tol=1e-6)
    for key in ("upper", "lower"):
        assert rel(out[key], ref[key]) <= 1e-6, (name, key, rel(out[key], ref[key]))
    assert loewner_ge(out["upper"], out["lower"])
    # guaranteed: any conforming field bounds from the correct side
    assert loewner_ge(out["upper"], ref["upper"], 1e-9)
    assert loewner_ge(ref["lower"], out["lower"], 1e-9)


@pytest.mark.parametrize("name", ["square2d_N23", "paper_rho1000_N15", "aniso2d_N9", "aniso3d_N5", "cube3d_N7",
                                  "spheres3d_N7", "laminate_N11", "homogeneous3d"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_dual_start_from_primal(hb, solver, name, prec):
    """Dual CG started from the primal minimisers (Remark "Avoiding the solution of dual
    formulation"): converged bounds equal the oracle's (1e-10 FP64, 1e-6 mixed) and, at a
    loose tolerance, the lower bound is still a guaranteed one (below the exact Galerkin
    lower bound) however good or bad the start."""
    precision = hb.HOM_FP64 if prec == "fp64" else hb.HOM_MIXED
    p = CASES[name]()
    ref = oracle.dense_bounds(p)
    out = solver(p, precision=precision, tol=1e-12 if prec == "fp64" else 1e-7, dual_start=1)
    for key in ("upper", "lower"):
        assert rel(out[key], ref[key]) <= (1e-10 if prec == "fp64" else 1e-6), (key, rel(out[key], ref[key]))
    loose = solver(p, precision=precision, tol=1e-2, dual_start=1)
    assert loewner_ge(ref["lower"], loose["lower"], 1e-9)
    assert loewner_ge(loose["upper"], ref["upper"], 1e-9)


def test_dual_start_iterations(hb, solver):
    """On the 3D N = 41 cube cell at 1e-4 the dual solve from the primal minimisers needs
    no more CG iterations than from zero (24 -> 23 measured: with the exact double-grid
    integration the superposition of the primal minimisers is not the dual minimiser,
    its residual is 14-30 % of |b| on the oracle's small cells), and the primal side is
    untouched."""
    p = ms.cube_inclusion_3d()
    zero = solver(p, precision=hb.HOM_FP64, tol=1e-4)
    warm = solver(p, precision=hb.HOM_FP64, tol=1e-4, dual_start=1)
    iz, iw = max(zero["report"]["iters"][1]), max(warm["report"]["iters"][1])
    print("dual iterations from zero", iz, "from the primal minimisers", iw)
    assert iw <= iz
    assert zero["report"]["iters"][0] == warm["report"]["iters"][0]
    assert np.array_equal(zero["upper"], warm["upper"])
    assert rel(warm["lower"], zero["lower"]) < 1e-4


def test_double_grid_cg_oracle_at_mid_size(hb, solver):
    """2D N = 45 (double grid 89): O2 (naive DFT + CG) against the FP64 CUDA path."""
    p = ms.random_rectangles_2d(17, N=45)
    ref = oracle.matfree_bounds(p, tol=1e-11)
    out = solver(p, precision=hb.HOM_FP64, tol=1e-11)
    for key in ("upper", "lower"):
        assert rel(out[key], ref[key]) <= 1e-10, (key, rel(out[key], ref[key]))


def test_repeatable_bitwise(hb, solver):
    p = ms.random_anisotropic_3d(9, N=7)
    a = solver(p, precision=hb.HOM_FP64, tol=1e-10)
    b = solver(p, precision=hb.HOM_FP64, tol=1e-10)
    assert np.array_equal(a["upper"], b["upper"]) and np.array_equal(a["lower"], b["lower"])
    assert a["report"]["iters"] == b["report"]["iters"]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_replay_matches_direct_launches(hb, solver, prec):
    """CG iteration blocks replayed from captured graphs run the same kernels in the same
    order as direct launches: bitwise equal bounds, equal iterations and launch counts,
    also for a check interval that does not divide the iteration count and when the
    kernel timing records event nodes inside the graphs."""
    precision = hb.HOM_FP64 if prec == "fp64" else hb.HOM_MIXED
    p = ms.random_anisotropic_3d(5, N=9)
    for every in (8, 5):
        d = solver(p, precision=precision, tol=1e-9, check_every=every, graph=-1)
        g1 = solver(p, precision=precision, tol=1e-9, check_every=every, graph=0)
        g2 = solver(p, precision=precision, tol=1e-9, check_every=every, graph=0)
        for out in (g1, g2):
            assert np.array_equal(out["upper"], d["upper"]) and np.array_equal(out["lower"], d["lower"])
            assert out["report"]["iters"] == d["report"]["iters"]
            assert out["report"]["launches"] == d["report"]["launches"]
    counts = {}
    for graph in (-1, 0, 0):
        hb.hom_profile_kernel(solver.ctx, "xpass")
        solver(p, precision=precision, tol=1e-9, graph=graph)
        n, ms_ = hb.hom_kernel_timing(solver.ctx)
        hb.hom_profile_kernel(solver.ctx, "")
        assert ms_ > 0
        counts.setdefault(graph, []).append(n)
    assert counts[0] == [counts[-1][0]] * 2


def test_not_converged_still_bounds(hb, solver):
    """max_iter reached: HOM_WARN_NOT_CONVERGED, the bounds stay guaranteed (Lemma bounds)."""
    p = ms.paper_square_2d(15, 1000.0)
    ref = oracle.dense_bounds(p)
    out = solver(p, precision=hb.HOM_FP64, tol=1e-14, max_iter=3, check_every=1)
    assert out["status"] == hb.binding.HOM_WARN_NOT_CONVERGED
    assert loewner_ge(out["upper"], ref["upper"], 1e-12)
    assert loewner_ge(ref["lower"], out["lower"], 1e-12)


def test_homogeneous_takes_no_iterations(hb, solver):
    p = CASES["homogeneous3d"]()
    out = solver(p, precision=hb.HOM_FP64)
    assert out["report"]["matvecs"] == 0
    assert np.abs(out["upper"] - p.A0).max() < 1e-14 and np.abs(out["lower"] - p.A0).max() < 1e-14


# ------------------------------------------------------------------------------------
# full size: the 3D N = 41 cube cell (double grid 81^3), the bench workload
# ------------------------------------------------------------------------------------
def test_full_size_cube_matvec_sampled_rows(hb):
    p = ms.cube_inclusion_3d()
    d = 3
    N = tuple(int(n) for n in p.N)
    ctx = hb.hom_create(0)
    try:
        rng = np.random.default_rng(123)
        info = hb.hom_problem_info(ctx, p)
        nws = hb.hom_step_workspace_size(ctx, p, d)
        ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
        fields = [random_real_field(rng, d, N) for _ in range(d)]
        uin = torch.from_numpy(np.stack([full_to_half(u, d) for u in fields])).cuda()
        ls = np.array([[0, 0, 0], [1, 0, 0], [0, -3, 2], [20, 20, -20], [-7, 13, 5], [3, -20, 11]])
        for side in (0, 1):
            coef = torch.empty((info["ncomp"],) + tuple(info["M"][::-1]), dtype=torch.float64, device="cuda")
            hb.hom_coefficient(ctx, p, side, hb.HOM_FP64, coef.data_ptr(), ws.data_ptr(), nws)
            out = torch.zeros_like(uin)
            hb.hom_matvec(ctx, p, side, hb.HOM_FP64, 1, d, coef.data_ptr(), uin.data_ptr(), out.data_ptr(),
                          ws.data_ptr(), nws)
            got = out.cpu().numpy()
            for r in range(d):
                full = half_to_full(got[r], d, N[0])
                rows = matfree.matvec_sampled(p, "primal" if side == 0 else "dual", fields[r], ls)
                for i, l in enumerate(ls):
                    idx = tuple(l + (np.array(N) - 1) // 2)
                    v = full[(slice(None),) + idx]
                    assert np.abs(v - rows[i]).max() <= 1e-11 * max(1.0, np.abs(rows[i]).max()), (side, r, l)
    finally:
        hb.hom_destroy(ctx)


def test_full_size_cube_bounds_properties(hb, solver):
    p = ms.cube_inclusion_3d()
    f = p.volume_fraction()
    voigt = (1 - f) * 1.0 + f * 100.0
    reuss = 1.0 / ((1 - f) / 1.0 + f / 100.0)
    out64 = solver(p, precision=hb.HOM_FP64, tol=1e-8)
    outmx = solver(p, precision=hb.HOM_MIXED, tol=1e-6)
    for out in (out64, outmx):
        up, lo = out["upper"], out["lower"]
        assert loewner_ge(up, lo) and loewner_ge(voigt * np.eye(3), up) and loewner_ge(lo, reuss * np.eye(3))
        # centred cube + isotropic phases: bounds proportional to I (Sec. 7)
        assert np.abs(up - up[0, 0] * np.eye(3)).max() < 1e-9 * up[0, 0]
        assert np.abs(lo - lo[0, 0] * np.eye(3)).max() < 1e-9 * lo[0, 0]
    assert rel(outmx["upper"], out64["upper"]) < 1e-6 and rel(outmx["lower"], out64["lower"]) < 1e-6
    # bounds tighten from N = 21 to N = 41 (nested spaces, exact integration)
    small = solver(p.with_N(21), precision=hb.HOM_FP64, tol=1e-8)
    assert out64["upper"][0, 0] <= small["upper"][0, 0] + 1e-9
    assert out64["lower"][0, 0] >= small["lower"][0, 0] - 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["aniso3d_N5", "cube3d_N7", "square2d_N23", "spheres3d_N7"])
def test_starting_fields_and_fields_out(hb, solver, name, prec):
    """hom_bounds_io: the converged fields come back out; restarting from them (any scale:
    Rayleigh-Ritz rescales the start) needs almost no iterations; a random start gives the
    same converged bounds; all bounds stay guaranteed."""
    precision = hb.HOM_FP64 if prec == "fp64" else hb.HOM_MIXED
    tol = 1e-10 if prec == "fp64" else 1e-6
    p = CASES[name]()
    d = p.d
    N = [int(n) for n in p.N] + [1] * (3 - d)
    shape = (2, d, d, N[2], N[1], (N[0] + 1) // 2)
    fields = torch.zeros(shape, dtype=torch.complex128, device="cuda")
    ref = solver(p, precision=precision, tol=tol, fields=fields)
    it0 = ref["report"]["iters"]
    start = 3.0 * fields
    again = solver(p, precision=precision, tol=tol, x0=start)
    # FP64: within two iterations; mixed: the Rayleigh-Ritz factor of an inexact field is not
    # exactly 1, so one short refinement may follow
    limit = 2 if prec == "fp64" else max(2, 0.2 * max(max(r) for r in it0))
    assert max(max(r) for r in again["report"]["iters"]) <= limit, (it0, again["report"]["iters"])
    for key in ("upper", "lower"):
        assert rel(again[key], ref[key]) <= (1e-9 if prec == "fp64" else 1e-6)
    g = torch.Generator(device="cuda").manual_seed(3)
    rnd = torch.randn(shape, dtype=torch.complex128, device="cuda", generator=g)
    out = solver(p, precision=precision, tol=tol, x0=rnd)
    dense = oracle.dense_bounds(p)
    for key in ("upper", "lower"):
        assert rel(out[key], dense[key]) <= (1e-9 if prec == "fp64" else 1e-6)
    assert loewner_ge(out["upper"], dense["upper"], 1e-9) and loewner_ge(dense["lower"], out["lower"], 1e-9)


@pytest.mark.parametrize("N", [5, 9])
def test_element_bounds_match_oracle_and_contain_the_laminate(hb, N):
    """Entry intervals of A_H (Lemma bounds): equal to the oracle's, and they contain the exact
    homogenized tensor of an anisotropic laminate (closed form)."""
    import sys
    import os
    sys.path.insert(0, os.path.dirname(__file__))
    from test_oracle_pins import _anisotropic_laminate, _laminate_exact
    p, A0, A1, w = _anisotropic_laminate(N)
    ref = oracle.dense_bounds(p)
    s = hb.Bounds(0)
    try:
        out = s(p, precision=hb.HOM_FP64, tol=1e-12)
    finally:
        s.close()
    for key in ("elem_lo", "elem_hi"):
        assert np.abs(out[key] - ref[key]).max() <= 1e-10 * np.abs(ref["upper"]).max(), key
    exact = _laminate_exact(A0, A1, w)
    assert np.all(out["elem_lo"] <= exact + 1e-12) and np.all(exact <= out["elem_hi"] + 1e-12)


def test_full_size_spheres_matvec_sampled_rows(hb):
    """The 3D 16-ball cell at N = 113 (double grid 225^3), the mixed-precision workload: rows
    of the FP64 and FP32 operators at full size against the oracle's one-by-one rows
    (Lemma Ga_full), 1e-11 (FP64) and 2e-6 (FP32) relative to the largest entry."""
    p = ms.random_spheres_3d(0)
    d = 3
    N = tuple(int(n) for n in p.N)
    ctx = hb.hom_create(0)
    try:
        rng = np.random.default_rng(7)
        info = hb.hom_problem_info(ctx, p)
        nws = hb.hom_step_workspace_size(ctx, p, d)
        ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
        fields = [random_real_field(rng, d, N) for _ in range(d)]
        uin = np.stack([full_to_half(u, d) for u in fields])
        cases = {0: np.array([[0, 0, 0], [1, -2, 3], [56, -56, 10]]), 1: np.array([[5, 0, -1], [-40, 33, 56]])}
        for side, ls in cases.items():
            rows = matfree.matvec_sampled(p, "primal" if side == 0 else "dual", fields[0], ls)
            for prec, cdt, rdt, tol in ((hb.HOM_FP64, torch.complex128, torch.float64, 1e-11),
                                        (hb.HOM_FP32, torch.complex64, torch.float32, 2e-6)):
                coef = torch.empty((info["ncomp"],) + tuple(info["M"][::-1]), dtype=rdt, device="cuda")
                hb.hom_coefficient(ctx, p, side, prec, coef.data_ptr(), ws.data_ptr(), nws)
                x = torch.from_numpy(uin).to(cdt).cuda()
                out = torch.zeros_like(x)
                hb.hom_matvec(ctx, p, side, prec, 1, d, coef.data_ptr(), x.data_ptr(), out.data_ptr(),
                              ws.data_ptr(), nws)
                full = half_to_full(out.cpu().numpy().astype(np.complex128)[0], d, N[0])
                scale = max(1.0, np.abs(rows).max())
                for i, l in enumerate(ls):
                    idx = tuple(l + (np.array(N) - 1) // 2)
                    v = full[(slice(None),) + idx]
                    assert np.abs(v - rows[i]).max() <= tol * scale, (side, prec, l, v, rows[i])
    finally:
        hb.hom_destroy(ctx)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_laminate_at_the_largest_2d_grid(hb, solver, precision):
    """The largest 2D grid hom_bounds takes: N = 1348 (double grid 2695 = 5 * 7^2 * 11, whose
    FP64 energy pass holds the four rows of a plane in 220 KB). The laminate's closed forms
    hold at every N (layers normal to x1: upper[1,1] is the arithmetic mean and lower[0,0] the
    harmonic mean, exactly; the other diagonal entries are strict bounds)."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "laminate_2d.json")))
    p = ms.laminate_2d(1348, width=g["width"], a_matrix=g["a_matrix"], a_incl=g["a_incl"])
    prec = hb.HOM_FP64 if precision == "fp64" else hb.HOM_MIXED
    out = solver(p, precision=prec, tol=1e-6)
    up, lo = np.asarray(out["upper"]), np.asarray(out["lower"])
    assert up[1, 1] == pytest.approx(g["arithmetic"], rel=1e-10)
    assert lo[0, 0] == pytest.approx(g["harmonic"], rel=1e-10)
    assert abs(up[0, 1]) < 1e-10 and abs(lo[0, 1]) < 1e-10
    assert up[0, 0] > g["harmonic"] and lo[1, 1] < g["arithmetic"]
    assert loewner_ge(up, lo)


def test_oversize_grids_rejected_before_any_work(hb, solver):
    """One step past the largest grids (2D N = 1349: double grid 2835; 3D N = 615: 1287) the
    energy pass cannot hold a plane of rows: hom_workspace_size refuses with
    HOM_ERR_INVALID_ARG, so no workspace is ever allocated; the largest grids are accepted."""
    ctx = solver.ctx
    for prec in (hb.HOM_FP64, hb.HOM_MIXED):
        opts = hb.make_opts(precision=prec)
        assert hb.hom_workspace_size(ctx, ms.laminate_2d(1348), opts) > 0
        assert hb.hom_workspace_size(ctx, ms.cube_inclusion_3d(N=613), opts) > 0
        for p in (ms.laminate_2d(1349), ms.laminate_2d(1350), ms.cube_inclusion_3d(N=615)):
            with pytest.raises(hb.HombError) as e:
                hb.hom_workspace_size(ctx, p, opts)
            assert e.value.status == hb.binding.HOM_ERR_INVALID_ARG
            assert "too large" in str(e.value)


def test_one_context_per_thread(hb):
    """Contexts are independent: two host threads, each with its own context and stream,
    solve at the same time (ctypes releases the interpreter lock during the calls; graph
    captures are thread-local) and reproduce the results of the same solves run one after
    the other."""
    import threading
    cells = [ms.square_inclusion_2d(N=23), ms.cube_inclusion_3d(N=9)]
    precs = [hb.HOM_FP64, hb.HOM_MIXED]
    ref = {}
    s0 = hb.Bounds(0)
    try:
        for i, p in enumerate(cells):
            for prec in precs:
                o = s0(p, precision=prec, tol=1e-8)
                ref[i, prec] = (np.asarray(o["upper"]), np.asarray(o["lower"]))
    finally:
        s0.close()
    errors, got = [], {}

    def work(i):
        try:
            s = hb.Bounds(0)
            st = torch.cuda.Stream()
            try:
                with torch.cuda.stream(st):
                    for rep in range(3):
                        for prec in precs:
                            o = s(cells[i], precision=prec, tol=1e-8)
                            got[i, prec, rep] = (np.asarray(o["upper"]), np.asarray(o["lower"]))
            finally:
                st.synchronize()
                s.close()
        except Exception as e:  # reported by the main thread
            errors.append(repr(e))

    threads = [threading.Thread(target=work, args=(i,)) for i in range(len(cells))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=600)
    assert not any(t.is_alive() for t in threads)
    assert not errors, errors
    assert len(got) == len(cells) * len(precs) * 3
    for (i, prec, rep), (up, lo) in got.items():
        ru, rl = ref[i, prec]
        assert np.abs(up - ru).max() <= 1e-12 * np.abs(ru).max(), (i, prec, rep)
        assert np.abs(lo - rl).max() <= 1e-12 * np.abs(rl).max(), (i, prec, rep)
