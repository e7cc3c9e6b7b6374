"""Pins of the Shrake-Rupley oracle (numerical SASA): exact special cases and convergence to
the exact (inclusion-exclusion) areas as the point count grows."""
import math

import numpy as np
import pytest

from oracle import shrake_rupley as sr

P = 1.4


def test_points_are_unit_and_balanced():
    pts = sr.sphere_points(960).astype(np.float64)
    assert np.allclose(np.linalg.norm(pts, axis=1), 1.0, atol=1e-6)
    # golden-spiral points have a nearly zero centroid and cover both hemispheres equally
    assert np.abs(pts.mean(0)).max() < 2e-3
    assert (pts[:, 2] > 0).sum() == 480


def test_isolated_sphere_all_exposed():
    pts = sr.sphere_points(960)
    c = sr.exposed_counts(np.zeros((1, 3)), np.array([1.7]), pts)
    assert c[0] == 960


def test_buried_atom_none_exposed():
    # a small ball at the centre of a large one: every point of the small sphere is inside
    pts = sr.sphere_points(500)
    c = sr.exposed_counts(np.array([[0.0, 0, 0], [0.2, 0, 0]]), np.array([2.0, 1.0]), pts)
    assert c[1] == 0 and c[0] == 500


@pytest.mark.parametrize("d", [1.5, 3.0, 5.0])
def test_two_spheres_converge_to_the_cap_formula(d):
    r = np.array([1.5, 1.7])
    R1, R2 = r + P
    dd = math.sqrt(d * d + 0.3 ** 2 + 0.2 ** 2)
    t1 = (dd * dd + R1 * R1 - R2 * R2) / (2 * dd)
    exact = 4 * math.pi * R1 * R1 - 2 * math.pi * R1 * (R1 - t1)
    errs = [abs(sr.areas(np.array([[0.0, 0, 0], [d, 0.3, -0.2]]), r, m)[0] - exact) for m in (960, 15360)]
    assert errs[1] < 0.05 * 4 * math.pi * R1 * R1 / math.sqrt(960)
    assert errs[1] <= errs[0] + 1e-12


def test_globule_converges_to_the_exact_areas(orc, gen):
    m = gen.globule(200, 1)
    ex = orc.sasa(m.coords, m.radii, grad=False)[0]
    e1 = np.abs(sr.areas(m.coords, m.radii, 240) - ex).mean()
    e2 = np.abs(sr.areas(m.coords, m.radii, 3840) - ex).mean()
    assert e2 < 0.35 * e1
    assert abs(sr.areas(m.coords, m.radii, 3840).sum() - ex.sum()) < 2e-3 * ex.sum()
