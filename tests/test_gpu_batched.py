"""hom_bounds_batched: many 2D cells of uneven N in one persistent launch.

Parity: every problem's bounds against the oracle (dense O1 for small N, double-grid
CG O2 for larger N): FP64 within 1e-10, mixed within 1e-6 with lower <= upper. The
random-rectangle batch of the benchmark (256 seeds, N in {23, 63, 113, 203}) is
checked for properties at full size and, on a sample, against single hom_bounds solves.
"""
import numpy as np
import pytest

import microstructures as ms
import oracle

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


def small_batch():
    probs = [ms.square_inclusion_2d(N=9), ms.random_anisotropic_2d(3, N=7), ms.laminate_2d(11),
             ms.random_rectangles_2d(4, N=13), ms.paper_square_2d(15, 1000.0), ms.checkerboard_2d(5),
             ms.random_anisotropic_2d(8, N=1), ms.homogeneous(2, 5, np.array([[2.0, 0.3], [0.3, 1.0]])),
             ms.make_problem(2, (13, 9), (1.0, 0.7), np.array([[2.0, 0.3], [0.3, 1.0]]),
                             [ms.box((0.1, 0.05), (0.3, 0.2), 7.0, 2), ms.ball((-0.25, -0.2), 0.12, 0.2, 2)]),
             ms.square_inclusion_2d(N=23)]
    return probs


def rel(a, b):
    return np.abs(a - b).max() / np.linalg.norm(b)


def loewner_ge(A, B, tol=1e-12):
    S = 0.5 * ((A - B) + (A - B).T)
    return np.linalg.eigvalsh(S).min() >= -tol * max(1.0, np.abs(A).max())


@pytest.fixture(scope="module")
def refs():
    return [oracle.dense_bounds(p) for p in small_batch()]


def test_batched_fp64_matches_oracle(hb, solver, refs):
    probs = small_batch()
    out = solver.batched(probs, precision=hb.HOM_FP64, tol=1e-12)
    assert (out["status"] == 0).all(), out["status"]
    for i, ref in enumerate(refs):
        for key in ("upper", "lower"):
            assert rel(out[key][i], ref[key]) <= 1e-10, (i, key, out[key][i], ref[key])


def test_batched_mixed_matches_oracle(hb, solver, refs):
    probs = small_batch()
    out = solver.batched(probs, precision=hb.HOM_MIXED, tol=1e-6)
    for i, ref in enumerate(refs):
        for key in ("upper", "lower"):
            assert rel(out[key][i], ref[key]) <= 1e-6, (i, key, rel(out[key][i], ref[key]))
        assert loewner_ge(out["upper"][i], out["lower"][i])
        assert loewner_ge(out["upper"][i], ref["upper"], 1e-9) and loewner_ge(ref["lower"], out["lower"][i], 1e-9)


def test_batched_equals_single_solves_mid_size(hb, solver):
    probs = [ms.random_rectangles_2d(s, N=n) for s, n in ((31, 45), (32, 63), (33, 23), (34, 113))]
    out = solver.batched(probs, precision=hb.HOM_FP64, tol=1e-11)
    for i, p in enumerate(probs):
        single = solver(p, precision=hb.HOM_FP64, tol=1e-11)
        for key in ("upper", "lower"):
            assert rel(out[key][i], single[key]) <= 1e-10, (i, key)
    ref = oracle.matfree_bounds(probs[0], tol=1e-11)
    for key in ("upper", "lower"):
        assert rel(out[key][0], ref[key]) <= 1e-10


def test_graph_replay_and_autotune(hb, solver):
    a = [ms.random_rectangles_2d(s, N=23) for s in range(6)]
    b = [ms.random_rectangles_2d(s + 100, N=23) for s in range(6)]
    stream = torch.cuda.Stream()
    plain_a = solver.batched(a, precision=hb.HOM_MIXED, tol=1e-5)
    plain_b = solver.batched(b, precision=hb.HOM_MIXED, tol=1e-5)
    ga = solver.batched(a, precision=hb.HOM_MIXED, tol=1e-5, graph=1, stream=stream.cuda_stream)
    gb = solver.batched(b, precision=hb.HOM_MIXED, tol=1e-5, graph=1, stream=stream.cuda_stream)   # replay
    tb = solver.batched(b, precision=hb.HOM_MIXED, tol=1e-5, autotune=1)
    for x, y in ((plain_a, ga), (plain_b, gb)):
        assert np.array_equal(x["upper"], y["upper"]) and np.array_equal(x["lower"], y["lower"])
    # a different chunk capacity changes only the order of the partial sums
    assert np.allclose(tb["upper"], plain_b["upper"], rtol=1e-9, atol=0)
    assert np.allclose(tb["lower"], plain_b["lower"], rtol=1e-9, atol=0)
    assert gb["report"]["launches"] == 1


def test_benchmark_batch_properties(hb, solver):
    """256 seeded random-rectangle cells, N drawn from {23, 63, 113, 203}: one launch."""
    probs = [ms.random_rectangles_2d(s) for s in range(256)]
    out = solver.batched(probs, precision=hb.HOM_MIXED, tol=1e-4)
    assert (out["status"] >= 0).all()
    for i, p in enumerate(probs):
        f = p.volume_fraction()
        a = p.inclusions[0].A[0, 0]
        voigt = (1 - f) + f * a
        reuss = 1.0 / ((1 - f) + f / a)
        up, lo = out["upper"][i], out["lower"][i]
        assert loewner_ge(up, lo, 1e-9), i
        assert loewner_ge(voigt * np.eye(2), up, 1e-9) and loewner_ge(lo, reuss * np.eye(2), 1e-9), i
    # a sample against single FP64 solves at a tight tolerance
    for i in range(0, 256, 37):
        single = solver(probs[i], precision=hb.HOM_FP64, tol=1e-9)
        for key in ("upper", "lower"):
            assert rel(out[key][i], single[key]) <= 2e-5, (i, key, rel(out[key][i], single[key]))


def test_batched_rejects_3d(hb, solver):
    with pytest.raises(hb.HombError):
        solver.batched([ms.cube_inclusion_3d(N=5)])


@pytest.mark.parametrize("cluster", [2, 4, 8])
@pytest.mark.parametrize("threads", [256, 1024])
def test_cluster_cooperative_cells(hb, solver, refs, cluster, threads):
    """The largest cells worked on by a whole thread-block cluster (every pass and
    reduction split over its CTAs) give the oracle's bounds like single-CTA cells: FP64
    within 1e-10 at tol 1e-12, also with ragged splits (cells of N 9, 13, 15, 23 mixed,
    the cooperative ones N >= 13 here), and mixed precision within 1e-6."""
    probs = small_batch()
    try:
        hb.binding.hom_set_batch_threads(solver.ctx, threads)
        hb.binding.hom_set_batch_cluster(solver.ctx, cluster, 25)
        out = solver.batched(probs, precision=hb.HOM_FP64, tol=1e-12)
        assert (out["status"] == 0).all(), out["status"]
        for i, ref in enumerate(refs):
            for key in ("upper", "lower"):
                assert rel(out[key][i], ref[key]) <= 1e-10, (i, key, rel(out[key][i], ref[key]))
        mixed = solver.batched(probs, precision=hb.HOM_MIXED, tol=1e-6)
        for i, ref in enumerate(refs):
            for key in ("upper", "lower"):
                assert rel(mixed[key][i], ref[key]) <= 1e-6, (i, key)
            assert loewner_ge(mixed["upper"][i], mixed["lower"][i])
    finally:
        hb.binding.hom_set_batch_threads(solver.ctx, 0)
        hb.binding.hom_set_batch_cluster(solver.ctx, 0, 0)


def test_cluster_cooperative_benchmark_cells(hb, solver):
    """Cluster-cooperative N = 113 and 203 cells of the benchmark batch equal the same
    cells solved one CTA each (FP64, tol 1e-10: 1e-9 relative), with the graph replayed."""
    probs = [ms.random_rectangles_2d(s) for s in range(24)]
    base = solver.batched(probs, precision=hb.HOM_FP64, tol=1e-10)
    try:
        hb.binding.hom_set_batch_cluster(solver.ctx, 4, 225)
        stream = torch.cuda.Stream()
        for _ in range(2):
            out = solver.batched(probs, precision=hb.HOM_FP64, tol=1e-10, graph=1, stream=stream.cuda_stream)
        for i in range(len(probs)):
            for key in ("upper", "lower"):
                assert rel(out[key][i], base[key][i]) <= 1e-9, (i, key)
    finally:
        hb.binding.hom_set_batch_cluster(solver.ctx, 0, 0)


@pytest.mark.parametrize("cluster,threads", [(1, 512), (4, 512), (1, 1024)])
def test_warp_passes_match_block_passes(hb, solver, cluster, threads):
    """The warp-owned pencil passes of the FP32 iterations (double-grid lengths 45, 125,
    225, 405) and the chunked block-level passes solve the same problems: cells of the
    benchmark batch with every N of its mix (23, 63, 113, 203) and a rectangular cell that
    takes the warp passes along one axis only (N = 23 x 13), single-CTA and cluster-split:
    at tol 1e-6 both are within 1e-5 of FP64 single solves at tol 1e-10 (the FP32 floor of
    the batched solve on its high-contrast cells: seed 2 ends near 4e-6 either way), the
    warp passes no further off than the block passes (up to 1e-6), with lower <= upper."""
    probs = [ms.random_rectangles_2d(s) for s in (0, 1, 2, 3, 5, 6, 9, 11)]
    probs.append(ms.make_problem(2, (23, 13), (1.0, 0.6), 1.0, [ms.box((0.1, 0.0), (0.4, 0.3), 50.0, 2)]))
    assert {int(p.N[0]) for p in probs} >= {23, 63, 113, 203}
    out = {}
    try:
        hb.binding.hom_set_batch_threads(solver.ctx, threads)
        hb.binding.hom_set_batch_cluster(solver.ctx, cluster, 225)
        for wp in (1, 0):
            hb.binding.hom_set_batch_warp_passes(solver.ctx, wp)
            out[wp] = solver.batched(probs, precision=hb.HOM_MIXED, tol=1e-6)
            assert (out[wp]["status"] >= 0).all()
        for i, p in enumerate(probs):
            assert loewner_ge(out[1]["upper"][i], out[1]["lower"][i])
            ref = solver(p, precision=hb.HOM_FP64, tol=1e-10)
            for key in ("upper", "lower"):
                e1, e0 = rel(out[1][key][i], ref[key]), rel(out[0][key][i], ref[key])
                assert e1 <= 1e-5 and e0 <= 1e-5 and e1 <= e0 + 1e-6, (i, key, e1, e0)
    finally:
        hb.binding.hom_set_batch_warp_passes(solver.ctx, 1)
        hb.binding.hom_set_batch_threads(solver.ctx, 0)
        hb.binding.hom_set_batch_cluster(solver.ctx, 0, 0)
