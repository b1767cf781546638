"""Sanity of the seeded input generators (CPU)."""
import math

import numpy as np

from workloads import configs, geometry


def test_c1_c2_c3_sizes():
    assert configs.c1().geom.m == 242
    g = configs.c2().geom
    assert g.m == 3525 and abs(g.extra["perimeter"] - 2.294863) < 1e-6
    assert abs(configs.c3().geom.m - 38038) <= 1


def test_star_points_are_equispaced_in_arclength_with_unit_outward_normals():
    g = geometry.star(512, 0.3, 0.2, 5)
    d = np.linalg.norm(np.diff(np.vstack([g.X, g.X[:1]]), axis=0), axis=1)
    assert d.max() / d.min() < 1.0001
    assert np.allclose(np.linalg.norm(g.normals, axis=1), 1.0)
    out = np.sum((g.X - 0.5) * g.normals, axis=1)
    assert np.all(out > 0)
    assert abs(g.weights.sum() - g.extra["perimeter"]) < 1e-12


def test_sphere_weights_sum_to_area():
    g = geometry.sphere(64, 0.3)
    assert abs(g.weights.sum() - 4 * math.pi * 0.09) < 1e-12
    e = geometry.ellipsoid(64, (0.2, 0.3, 0.25))
    assert np.all(np.sum((e.X - 0.5) * e.normals, axis=1) > 0)


def test_seeded_data_is_deterministic():
    g = configs.c2(n=256).geom
    from workloads import data
    a = data.fourier_data(g.param, 0)
    b = data.fourier_data(g.param, 0)
    assert np.array_equal(a, b)
