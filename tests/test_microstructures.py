"""The seeded input generators: determinism and the stated distributions (no GPU)."""
import itertools
import math

import numpy as np

import microstructures as ms


def test_random_rectangles_deterministic_and_valid():
    for seed in range(40):
        p = ms.random_rectangles_2d(seed)
        q = ms.random_rectangles_2d(seed)
        assert p.N[0] == q.N[0] and len(p.inclusions) == len(q.inclusions)
        for a, b in zip(p.inclusions, q.inclusions):
            assert np.array_equal(a.center, b.center) and np.array_equal(a.size, b.size)
        assert int(p.N[0]) in ms.RANDOM_RECT_N
        assert 1 <= len(p.inclusions) <= 16
        assert 0.1 - 1e-12 <= p.volume_fraction() <= 0.5 + 1e-12
        a = p.inclusions[0].A[0, 0]
        assert 1e-2 <= a <= 1e3
        assert all(inc.A[0, 0] == a for inc in p.inclusions)
        for i, j in itertools.combinations(p.inclusions, 2):
            assert not ms.inclusions_overlap(i, j, p.Y)
        assert all(ms.fits_cell(i, p.Y) for i in p.inclusions)


def test_random_spheres_packing():
    p = ms.random_spheres_3d(0, N=113)
    assert len(p.inclusions) == 16
    assert abs(p.volume_fraction() - 0.3) < 1e-12
    R = p.inclusions[0].size[0]
    assert abs(R - (3 * 0.3 / (4 * math.pi * 16)) ** (1 / 3)) < 1e-15
    for i, j in itertools.combinations(p.inclusions, 2):
        dist = np.abs(i.center - j.center)
        dist = np.minimum(dist, 1.0 - dist)
        assert np.sqrt(np.sum(dist ** 2)) >= 2 * R + 1e-3 - 1e-12


def test_fixed_workloads():
    c1 = ms.square_inclusion_2d()
    assert c1.d == 2 and list(c1.N) == [23, 23] and list(c1.M) == [45, 45]
    assert abs(c1.volume_fraction() - 0.36) < 1e-15 and c1.is_isotropic()
    c2 = ms.cube_inclusion_3d()
    assert c2.d == 3 and list(c2.M) == [81, 81, 81] and abs(c2.volume_fraction() - 0.125) < 1e-15
    assert not ms.random_anisotropic_3d(0).is_isotropic()


def test_overlap_rules():
    Y = np.ones(2)
    a = ms.box([0.0, 0.0], [0.4, 0.4], 2.0, 2)
    touching = ms.box([0.4, 0.0], [0.4, 0.4], 2.0, 2)
    wrapped = ms.box([0.45, 0.0], [0.4, 0.4], 2.0, 2)   # overlaps a through the periodic boundary? no
    assert not ms.inclusions_overlap(a, touching, Y)
    assert ms.inclusions_overlap(a, ms.box([0.3, 0.1], [0.4, 0.4], 2.0, 2), Y)
    assert not ms.inclusions_overlap(a, wrapped, Y)
    b = ms.box([0.49, 0.0], [0.3, 0.3], 2.0, 2)
    c = ms.box([-0.49, 0.0], [0.3, 0.3], 2.0, 2)          # periodic neighbours
    assert ms.inclusions_overlap(b, c, Y)
    d1 = ms.ball([0.0, 0.0], 0.2, 2.0, 2)
    assert ms.inclusions_overlap(d1, ms.box([0.25, 0.0], [0.2, 0.2], 2.0, 2), Y)
    assert not ms.inclusions_overlap(d1, ms.box([0.35, 0.0], [0.2, 0.2], 2.0, 2), Y)


def test_porous_image_is_raw_and_smoothing_is_a_flag():
    b = ms.porous_bitmap_2d(1, P=101, porosity=0.4)
    assert set(np.unique(b)) <= {0.029, 0.49} and abs((b == 0.029).mean() - 0.4) < 0.05
    p = ms.bitmap_problem(b, smooth=True)
    assert p.smooth and np.array_equal(p.bitmap, b)       # the image is stored unsmoothed
    assert not ms.bitmap_problem(b).smooth
    assert not hasattr(ms, "smooth_indicator_2d")         # no method step in the input module
