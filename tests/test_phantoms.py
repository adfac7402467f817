"""The seeded input generators are deterministic and give the stated shapes and contrasts."""
import numpy as np

import phantoms as ph


def test_sphere_centre_and_radius():
    s = ph.sphere((32, 32, 32), 10.0, 0.02)
    # grid origin voxel (centred index 0) is array index n/2 - 1
    assert s[15, 15, 15] == 0.02
    assert s[15, 15, 15 + 10] == 0.02 and s[15, 15, 15 + 11] == 0.0
    assert set(np.unique(s)) == {0.0, 0.02}


def test_ellipsoids_deterministic_and_bounded():
    a = ph.random_ellipsoids((48, 48, 48), count=5, rmin=3, rmax=8)
    b = ph.random_ellipsoids((48, 48, 48), count=5, rmin=3, rmax=8)
    assert np.array_equal(a, b)
    assert a.min() >= 0.0 and a.max() <= 0.05 and a.max() > 0.0
    # nothing touches the 2-voxel margin
    assert np.all(a[:2] == 0) and np.all(a[-2:] == 0)


def test_cell_phantom_levels():
    c = ph.cell((48, 64, 64), scale=0.5)
    vals = set(np.round(np.unique(c), 6))
    assert vals <= {0.0, 0.03, 0.05, 0.08}
    assert {0.03, 0.05, 0.08} <= vals


def test_cone_directions_are_unit_on_the_cone():
    d = ph.cone_directions(60, 0.8, 1.333)
    assert d.shape == (60, 3)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0)
    assert np.allclose(np.hypot(d[:, 0], d[:, 1]), 0.8 / 1.333)
