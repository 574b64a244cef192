"""Seeded synthetic microstructures for the periodic scalar-conductivity cell problem.

This module only describes and samples geometry: a periodic cell, an odd grid size
N, a matrix phase A0 and a list of non-overlapping inclusions (boxes, balls/disks)
with absolute SPD phase tensors. It holds none of the homogenisation arithmetic
(no Fourier coefficients, no projections, no bounds). Both the CPU oracle and the
GPU library's Python binding read these descriptions.

Geometry model (Vondrejc-Zeman-Marek, Sec. 6, Eq. A_with_inclusions):
    A(x) = A0 + sum_j f_j(x - x_j) (A_j - A0)
with f_j the indicator of a box (Remark "inclusion") or a ball, extended
periodically. The phases are given as absolute tensors A_j (a reading of the
paper's increments, which are A_j - A0).

Workload recipes (the paper uses no public dataset for these workloads):
  * square_inclusion_2d  - centred square, side 0.6 of a unit cell, a = 1 / 10, N = 23.
  * cube_inclusion_3d    - centred cube, side 0.5 of a unit cell, a = 1 / 100, N = 41.
  * random_rectangles_2d - 1..16 non-overlapping axis-aligned rectangles, volume
                           fraction U(0.1, 0.5), inclusion conductivity log-uniform in
                           [1e-2, 1e3] over a matrix of 1, N drawn from {23, 63, 113, 203}.
  * random_spheres_3d    - 16 equal non-overlapping balls, volume fraction 0.3,
                           contrast 1000, N = 113.
  * paper_square_2d      - the paper's Sec. 7 cell (-1, 1)^2 with |x_a| < 3/5 and
                           A = (1 + rho f) I.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

BOX = "box"
BALL = "ball"   # a disk when d == 2


@dataclasses.dataclass
class Inclusion:
    shape: str                 # BOX or BALL
    center: np.ndarray         # (d,)
    size: np.ndarray           # BOX: side lengths h (d,); BALL: (radius,)
    A: np.ndarray              # (d, d) absolute SPD phase tensor inside the inclusion

    def volume(self) -> float:
        d = self.center.shape[0]
        if self.shape == BOX:
            return float(np.prod(self.size))
        r = float(self.size[0])
        return math.pi * r * r if d == 2 else 4.0 / 3.0 * math.pi * r ** 3


@dataclasses.dataclass
class Problem:
    d: int
    Y: np.ndarray              # (d,) cell side lengths, cell = prod (-Y/2, Y/2)
    N: np.ndarray              # (d,) grid sizes (odd; even sizes give the general grids)
    A0: np.ndarray             # (d, d) matrix phase
    inclusions: List[Inclusion]
    # optional pixel image of an isotropic scalar coefficient, shape (P_1, ..., P_d): pixel
    # (i_1, ..., i_d) covers prod_a (-Y_a/2 + i_a h_a, -Y_a/2 + (i_a + 1) h_a), h_a = Y_a / P_a,
    # and holds the conductivity a (A = a I there). When set, A0 and inclusions are unused.
    bitmap: np.ndarray = None
    # where GaNi samples a grid point lying exactly on an inclusion boundary: False puts it in
    # the matrix (strict membership, the paper's Eq. S and S1), True in the inclusion
    # (non-strict, Eq. S2). Galerkin with exact integration does not depend on it.
    closed: bool = False
    # pixel images only: True asks for the paper's local average of the image (Sec. 7.3)
    # before the coefficient is formed; a flag of the problem statement, applied by the
    # solver (and independently by the oracle), never by this module
    smooth: bool = False

    @property
    def M(self) -> np.ndarray:
        """Double-grid size 2N - 1 per axis."""
        return 2 * self.N - 1

    def with_N(self, N) -> "Problem":
        N = np.broadcast_to(np.asarray(N, dtype=np.int64), (self.d,)).copy()
        return dataclasses.replace(self, N=N)

    def is_bitmap(self) -> bool:
        return self.bitmap is not None

    def volume_fraction(self) -> float:
        return sum(inc.volume() for inc in self.inclusions) / float(np.prod(self.Y))

    def is_isotropic(self) -> bool:
        if self.bitmap is not None:
            return True

        def iso(A):
            return np.allclose(A, A[0, 0] * np.eye(self.d), rtol=0, atol=0)
        return iso(self.A0) and all(iso(inc.A) for inc in self.inclusions)


def _vec(x, d):
    return np.broadcast_to(np.asarray(x, dtype=np.float64), (d,)).copy()


def make_problem(d, N, Y=1.0, a0=1.0, inclusions=()) -> Problem:
    A0 = np.asarray(a0, dtype=np.float64)
    if A0.ndim == 0:
        A0 = float(A0) * np.eye(d)
    return Problem(d=d, Y=_vec(Y, d), N=np.broadcast_to(np.asarray(N, dtype=np.int64), (d,)).copy(),
                   A0=A0, inclusions=list(inclusions))


def box(center, h, a, d) -> Inclusion:
    A = np.asarray(a, dtype=np.float64)
    if A.ndim == 0:
        A = float(A) * np.eye(d)
    return Inclusion(BOX, _vec(center, d), _vec(h, d), A)


def ball(center, radius, a, d) -> Inclusion:
    A = np.asarray(a, dtype=np.float64)
    if A.ndim == 0:
        A = float(A) * np.eye(d)
    return Inclusion(BALL, _vec(center, d), np.array([float(radius)]), A)


# ----------------------------------------------------------------------------------
# fixed workloads
# ----------------------------------------------------------------------------------
def square_inclusion_2d(N=23, side=0.6, a_matrix=1.0, a_incl=10.0) -> Problem:
    """Unit cell, one centred square inclusion (2D, d = 2)."""
    return make_problem(2, N, 1.0, a_matrix, [box(0.0, side, a_incl, 2)])


def cube_inclusion_3d(N=41, side=0.5, a_matrix=1.0, a_incl=100.0) -> Problem:
    """Unit cell, one centred cube inclusion (3D, d = 3)."""
    return make_problem(3, N, 1.0, a_matrix, [box(0.0, side, a_incl, 3)])


def paper_square_2d(N, rho) -> Problem:
    """Cell (-1, 1)^2 with A = (1 + rho f) I and f the indicator of |x_a| < 3/5 (Sec. 7)."""
    return make_problem(2, N, 2.0, 1.0, [box(0.0, 1.2, 1.0 + rho, 2)])


def paper_square_even_2d(N, rho, closed=False) -> Problem:
    """Cell (-1, 1)^2 with A = (1 + rho f) I and f the indicator of |x_a| < 3/4 (Eq. S1,
    closed=False) or |x_a| <= 3/4 (Eq. S2, closed=True), the even-grid cells of Sec. 7."""
    p = make_problem(2, N, 2.0, 1.0, [box(0.0, 1.5, 1.0 + rho, 2)])
    return dataclasses.replace(p, closed=bool(closed))


def laminate_2d(N, width=0.4, a_matrix=1.0, a_incl=10.0, Y=1.0) -> Problem:
    """A stripe of the inclusion phase across the whole cell height: layers normal to x1."""
    Yv = _vec(Y, 2)
    return make_problem(2, N, Yv, a_matrix, [box(0.0, (width * Yv[0], Yv[1]), a_incl, 2)])


def checkerboard_2d(N, a1=1.0, a2=5.0, Y=1.0) -> Problem:
    """Two-phase checkerboard: two quarter-cell squares of phase a2 on a matrix a1."""
    Yv = _vec(Y, 2)
    q = Yv / 4.0
    return make_problem(2, N, Yv, a1, [box(-q, Yv / 2, a2, 2), box(q, Yv / 2, a2, 2)])


def homogeneous(d, N, A0) -> Problem:
    return make_problem(d, N, 1.0, A0, [])


# ----------------------------------------------------------------------------------
# periodic overlap tests (geometry only)
# ----------------------------------------------------------------------------------
def _pdist(a, b, Y):
    """Periodic (minimum-image) per-axis distance."""
    t = np.abs(np.asarray(a) - np.asarray(b))
    return np.minimum(t, Y - t)


def inclusions_overlap(p: Inclusion, q: Inclusion, Y, gap=0.0) -> bool:
    """True when two inclusions share an open set in the periodic cell.

    Touching is allowed (the interface has measure zero). ``gap`` widens both
    inclusions, so that ``gap > 0`` also rejects near-contacts.
    """
    Y = np.asarray(Y, dtype=np.float64)
    dist = _pdist(p.center, q.center, Y)
    if p.shape == BOX and q.shape == BOX:
        return bool(np.all(dist < 0.5 * (p.size + q.size) + gap))
    if p.shape == BALL and q.shape == BALL:
        return bool(np.sqrt(np.sum(dist ** 2)) < p.size[0] + q.size[0] + gap)
    bx, bl = (p, q) if p.shape == BOX else (q, p)
    dist = _pdist(bx.center, bl.center, Y)
    outside = np.maximum(dist - 0.5 * bx.size, 0.0)
    return bool(np.sqrt(np.sum(outside ** 2)) < bl.size[0] + gap)


def fits_cell(inc: Inclusion, Y) -> bool:
    """An inclusion must not overlap its own periodic images."""
    Y = np.asarray(Y, dtype=np.float64)
    if inc.shape == BOX:
        return bool(np.all(inc.size <= Y))
    return bool(2.0 * inc.size[0] <= np.min(Y))


# ----------------------------------------------------------------------------------
# random workloads
# ----------------------------------------------------------------------------------
RANDOM_RECT_N = (23, 63, 113, 203)


def random_rectangles_2d(seed: int, N=None, max_restarts=200) -> Problem:
    """Seeded random-rectangle cell (matrix a = 1, unit cell).

    Draws, in this order: N from {23, 63, 113, 203} (unless given), the number of
    rectangles J ~ U{1..16}, the volume fraction phi ~ U(0.1, 0.5), one inclusion
    conductivity a ~ 10^U(-2, 3) shared by all rectangles, a Dirichlet(1) split of
    phi over the J rectangles, and per rectangle an aspect ratio log-uniform in
    [1/4, 4] and a uniform centre. Rectangles are placed by rejection with a
    periodic clearance of 1e-3; a failed layout restarts with a new split.
    """
    rng = np.random.default_rng(np.random.SeedSequence([0x5EC7, int(seed)]))
    if N is None:
        N = int(rng.choice(RANDOM_RECT_N))
    J = int(rng.integers(1, 17))
    phi = float(rng.uniform(0.1, 0.5))
    a_incl = float(10.0 ** rng.uniform(-2.0, 3.0))
    Y = np.ones(2)
    for _ in range(max_restarts):
        w = rng.dirichlet(np.ones(J))
        areas = phi * w
        placed: List[Inclusion] = []
        ok = True
        for area in sorted(areas, reverse=True):
            rho = float(np.exp(rng.uniform(np.log(0.25), np.log(4.0))))
            h = np.array([math.sqrt(area * rho), math.sqrt(area / rho)])
            h = np.minimum(h, 0.95)
            for _attempt in range(400):
                c = rng.uniform(-0.5, 0.5, size=2)
                cand = box(c, h, a_incl, 2)
                if not any(inclusions_overlap(cand, o, Y, gap=1e-3) for o in placed):
                    placed.append(cand)
                    break
            else:
                ok = False
                break
        if ok:
            return make_problem(2, N, Y, 1.0, placed)
    raise RuntimeError(f"random_rectangles_2d: no layout found for seed {seed}")


def random_spheres_3d(seed: int, N=113, n_balls=16, phi=0.3, contrast=1000.0,
                      max_restarts=200) -> Problem:
    """Seeded random sequential addition of equal balls in the unit cube.

    Radius R = (3 phi / (4 pi n))^(1/3); periodic centre distance >= 2R + 1e-3;
    matrix a = 1, balls a = contrast.
    """
    rng = np.random.default_rng(np.random.SeedSequence([0xB411, int(seed)]))
    R = (3.0 * phi / (4.0 * math.pi * n_balls)) ** (1.0 / 3.0)
    Y = np.ones(3)
    for _ in range(max_restarts):
        placed: List[Inclusion] = []
        for _i in range(n_balls):
            for _attempt in range(2000):
                cand = ball(rng.uniform(-0.5, 0.5, size=3), R, contrast, 3)
                if not any(inclusions_overlap(cand, o, Y, gap=1e-3) for o in placed):
                    placed.append(cand)
                    break
            else:
                break
        if len(placed) == n_balls:
            return make_problem(3, N, Y, 1.0, placed)
    raise RuntimeError(f"random_spheres_3d: no packing found for seed {seed}")


def random_anisotropic_2d(seed: int, N=7, n_boxes=2) -> Problem:
    """Small anisotropic test cell: SPD A0 and SPD box phases with random rotations."""
    rng = np.random.default_rng(np.random.SeedSequence([0xA150, int(seed)]))

    def spd():
        t = rng.uniform(0, math.pi)
        Rm = np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]])
        lam = 10.0 ** rng.uniform(-1, 1, size=2)
        return Rm @ np.diag(lam) @ Rm.T

    Y = np.array([1.0, float(rng.uniform(0.7, 1.4))])
    placed: List[Inclusion] = []
    while len(placed) < n_boxes:
        h = rng.uniform(0.15, 0.45, size=2) * Y
        cand = box(rng.uniform(-0.5, 0.5, size=2) * Y, h, spd(), 2)
        if not any(inclusions_overlap(cand, o, Y, gap=1e-3) for o in placed):
            placed.append(cand)
    return make_problem(2, N, Y, spd(), placed)


def random_anisotropic_3d(seed: int, N=5, n_incl=2) -> Problem:
    """Small anisotropic 3D test cell with one box and one ball (when n_incl >= 2)."""
    rng = np.random.default_rng(np.random.SeedSequence([0xA153, int(seed)]))

    def spd():
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        lam = 10.0 ** rng.uniform(-1, 1, size=3)
        return Q @ np.diag(lam) @ Q.T

    Y = np.array([1.0, float(rng.uniform(0.8, 1.25)), float(rng.uniform(0.8, 1.25))])
    placed: List[Inclusion] = []
    k = 0
    while len(placed) < n_incl:
        if k % 2 == 0:
            cand = box(rng.uniform(-0.5, 0.5, size=3) * Y, rng.uniform(0.2, 0.45, size=3) * Y, spd(), 3)
        else:
            cand = ball(rng.uniform(-0.5, 0.5, size=3) * Y, float(rng.uniform(0.1, 0.2)), spd(), 3)
        if not any(inclusions_overlap(cand, o, Y, gap=1e-3) for o in placed):
            placed.append(cand)
            k += 1
    return make_problem(3, N, Y, spd(), placed)


def batch_rectangles_2d(seeds: Sequence[int], N=None) -> List[Problem]:
    return [random_rectangles_2d(s, N=N) for s in seeds]


# ----------------------------------------------------------------------------------
# pixel images (the paper's Sec. 7.3 workload type: a coefficient given per pixel)
# ----------------------------------------------------------------------------------
def bitmap_problem(bitmap, N=None, Y=1.0, smooth=False) -> Problem:
    """A cell whose isotropic conductivity is the pixel image `bitmap` (values > 0).
    N defaults to the image size (the grid points then sit at the pixel centres for odd
    sizes). smooth=True asks the solver to replace the image by the paper's local
    average (Sec. 7.3) first; the image itself is stored raw."""
    b = np.ascontiguousarray(np.asarray(bitmap, dtype=np.float64))
    d = b.ndim
    if d not in (2, 3) or np.any(~(b > 0)):
        raise ValueError("bitmap: 2D or 3D array of positive conductivities")
    Nv = np.asarray(b.shape if N is None else np.broadcast_to(N, (d,)), dtype=np.int64)
    Yv = _vec(Y, d)
    return Problem(d, Yv, Nv.copy(), float(b.mean()) * np.eye(d), [], bitmap=b, smooth=bool(smooth))


def box_bitmap(P, lo, hi, a_in, a_out=1.0, d=2) -> np.ndarray:
    """A P^d image holding a_in on the pixels [lo, hi) of every axis and a_out elsewhere."""
    b = np.full((P,) * d, float(a_out))
    b[tuple(slice(lo, hi) for _ in range(d))] = float(a_in)
    return b


def porous_bitmap_2d(seed: int, P=1199, porosity=0.45, r_min=0.01, r_max=0.04, a_solid=0.49,
                     a_pore=0.029) -> np.ndarray:
    """A synthetic porous two-phase P x P image standing in for a micrograph: pores are the
    union of periodic disks (centres uniform, radii log-uniform in [r_min, r_max] of the cell),
    added until the pore fraction reaches `porosity`; conductivities a_solid / a_pore (the
    paper's Sec. 7.3 phase values). The raw image: the paper's smoothing is a flag of the
    problem (bitmap_problem(..., smooth=True)), applied by the solver."""
    rng = np.random.default_rng(seed)
    c = (np.arange(P) + 0.5) / P - 0.5
    X, Yg = np.meshgrid(c, c, indexing="ij")
    pore = np.zeros((P, P), dtype=bool)
    while pore.mean() < porosity:
        cx, cy = rng.uniform(-0.5, 0.5, size=2)
        r = math.exp(rng.uniform(math.log(r_min), math.log(r_max)))
        dx = X - cx
        dy = Yg - cy
        dx -= np.round(dx)
        dy -= np.round(dy)
        pore |= dx * dx + dy * dy < r * r
    solid = (~pore).astype(np.float64)
    return a_pore + (a_solid - a_pore) * solid

