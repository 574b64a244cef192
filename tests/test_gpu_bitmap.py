"""Pixel-image coefficients (the paper's Sec. 7.3 workload type) through the C ABI.

The image's Fourier coefficients are computed on the GPU (DFT of the image, pixel sinc and
centring phase) and zero-padded to the double grid; the right-hand side is the operator
applied to the constant field. Parity against the oracle (which sums the pixel boxes
directly): the double-grid coefficient to 1e-12, FP64 bounds to 1e-10, mixed to 1e-6, GaNi
on the image grid to 1e-10; images of odd and even size, N equal to and different from the
image size, 2D and 3D. The paper's local average of the image (Sec. 7.3) is a flag of the
problem: the library smooths the uploaded image on the device, the oracle by its own
circulant-matrix products (oracle/image.py); both start from the same raw image.
"""
import numpy as np
import pytest

import microstructures as ms
import oracle
from oracle import gani, matfree

from layout import coef_to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def two_phase(seed, shape, p=0.4, a=(0.49, 0.029)):
    rng = np.random.default_rng(seed)
    return np.where(rng.uniform(size=shape) < p, a[1], a[0])


CELLS = {
    "box_image_P9_N9": lambda: ms.bitmap_problem(ms.box_bitmap(9, 2, 7, 10.0)),
    "two_phase_P9_N9": lambda: ms.bitmap_problem(two_phase(1, (9, 9))),
    "two_phase_P9_N5": lambda: ms.bitmap_problem(two_phase(2, (9, 9)), N=5),
    "two_phase_P8_N11": lambda: ms.bitmap_problem(two_phase(3, (8, 8)), N=11),
    "rect_cell_P7x5_N7x5": lambda: ms.bitmap_problem(two_phase(4, (7, 5)), N=(7, 5), Y=(1.0, 0.6)),
    "image3d_P5_N5": lambda: ms.bitmap_problem(two_phase(5, (5, 5, 5)), N=5),
    "image3d_P4_N7": lambda: ms.bitmap_problem(two_phase(6, (4, 4, 4), a=(3.0, 0.5)), N=7),
    "smoothed_P9_N9": lambda: ms.bitmap_problem(two_phase(7, (9, 9)), smooth=True),
    "smoothed_P10x7_N5x7": lambda: ms.bitmap_problem(two_phase(8, (10, 7)), N=(5, 7), Y=(1.0, 0.7), smooth=True),
    "smoothed3d_P5_N5": lambda: ms.bitmap_problem(two_phase(9, (5, 5, 5), a=(3.0, 0.5)), N=5, smooth=True),
}


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


@pytest.mark.parametrize("name", list(CELLS))
@pytest.mark.parametrize("side", [0, 1])
def test_image_coefficient_matches_oracle(hb, solver, name, side):
    p = CELLS[name]()
    d = p.d
    op = matfree.MatFreeOperator(p, "primal" if side == 0 else "dual")
    ctx = solver.ctx
    info = hb.hom_problem_info(ctx, p)
    nws = hb.hom_step_workspace_size(ctx, p, d)
    ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
    ref = coef_to_dev(op.A_grid, d, True)
    coef = torch.empty(ref.size, dtype=torch.float64, device="cuda")
    hb.hom_coefficient(ctx, p, side, hb.HOM_FP64, coef.data_ptr(), ws.data_ptr(), nws)
    torch.cuda.synchronize()
    got = coef.cpu().numpy().reshape(ref.shape)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("name", list(CELLS))
def test_image_bounds_match_dense_oracle(hb, solver, name):
    p = CELLS[name]()
    ref = oracle.dense_bounds(p)
    out = solver(p, precision=hb.HOM_FP64, tol=1e-12)
    assert out["status"] == 0
    for key in ("upper", "lower"):
        assert rel(out[key], ref[key]) <= 1e-10, (key, rel(out[key], ref[key]))
    mixed = solver(p, precision=hb.HOM_MIXED, tol=1e-7)
    for key in ("upper", "lower"):
        assert rel(mixed[key], ref[key]) <= 1e-6, (key, rel(mixed[key], ref[key]))


@pytest.mark.parametrize("name", ["two_phase_P9_N9", "rect_cell_P7x5_N7x5", "image3d_P5_N5", "two_phase_P9_N5",
                                  "smoothed_P9_N9", "smoothed3d_P5_N5"])
def test_image_gani_matches_oracle(hb, solver, name):
    p = CELLS[name]()
    ref = gani.gani_bounds(p)
    out = solver(p, precision=hb.HOM_FP64, tol=1e-12, discretization=1)
    assert rel(out["gani_A"], ref["A_HN"]) <= 1e-10
    assert rel(out["gani_B"], ref["B_HN"]) <= 1e-10
    for key in ("upper", "lower"):
        assert rel(out[key], ref[key]) <= 1e-10, key


def test_porous_image_against_double_grid_cg_oracle(hb, solver):
    """A 63 x 63 synthetic porous image at N = 63 (double grid 125): O2 (naive DFTs + CG)."""
    p = ms.bitmap_problem(ms.porous_bitmap_2d(7, P=63, r_min=0.03, r_max=0.1))
    ref = oracle.matfree_bounds(p, tol=1e-11)
    out = solver(p, precision=hb.HOM_FP64, tol=1e-11)
    for key in ("upper", "lower"):
        assert rel(out[key], ref[key]) <= 1e-9, (key, rel(out[key], ref[key]))


def test_smoothed_porous_image_against_double_grid_cg_oracle(hb, solver):
    """The same kind of 63 x 63 porous image with the paper's smoothing applied by the library
    (FP64 and mixed) against O2 on the oracle's own smoothing of the raw image; the smoothing
    moves the bounds by far more than the tolerance."""
    img = ms.porous_bitmap_2d(8, P=63, r_min=0.03, r_max=0.1)
    p = ms.bitmap_problem(img, smooth=True)
    ref = oracle.matfree_bounds(p, tol=1e-11)
    out = solver(p, precision=hb.HOM_FP64, tol=1e-11)
    mixed = solver(p, precision=hb.HOM_MIXED, tol=1e-8)
    raw = solver(ms.bitmap_problem(img), precision=hb.HOM_FP64, tol=1e-11)
    for key in ("upper", "lower"):
        assert rel(out[key], ref[key]) <= 1e-9, (key, rel(out[key], ref[key]))
        assert rel(mixed[key], ref[key]) <= 1e-6, (key, rel(mixed[key], ref[key]))
        assert rel(raw[key], ref[key]) > 1e-4


def test_smoothing_needs_an_image(hb, solver):
    p = ms.square_inclusion_2d(N=9)
    import dataclasses
    with pytest.raises(hb.HombError) as e:
        solver(dataclasses.replace(p, smooth=True), precision=hb.HOM_FP64)
    assert e.value.status == hb.binding.HOM_ERR_INVALID_ARG


def test_image_rejected_where_not_supported(hb, solver):
    p = CELLS["two_phase_P9_N9"]()
    with pytest.raises(hb.HombError):
        solver.batched([p])
    ctx = solver.ctx
    nws = hb.hom_step_workspace_size(ctx, p, 2)
    ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
    b = torch.empty((2, 2, 9, 5), dtype=torch.complex128, device="cuda")
    with pytest.raises(hb.HombError):
        hb.hom_rhs(ctx, p, 0, hb.HOM_FP64, 2, b.data_ptr(), ws.data_ptr(), nws)
