"""Pins of the Shrake-Rupley oracle (numerical SASA): exact special cases, every decision
against rational arithmetic on small inputs, an exact tie, and convergence to the exact
(inclusion-exclusion) areas as the point count grows."""
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


def _brute_exposed(coords, radii, pts, i, probe):
    """Every point of atom i decided in rational arithmetic against every other ball."""
    out = []
    for s in pts:
        ok = True
        for j in range(len(radii)):
            if j != i and sr._exact_margin_sign(coords[i], coords[j], radii[i], radii[j], s, probe) <= 0:
                ok = False
                break
        out.append(ok)
    return np.array(out)


def test_every_decision_matches_rational_arithmetic(gen):
    m = gen.globule(12, 4)
    pts = sr.sphere_points(64)
    for i in range(m.n):
        assert np.array_equal(sr.exposed_mask(m.coords, m.radii, pts, i), _brute_exposed(m.coords, m.radii, pts, i, P))


def test_exact_tie_is_covered_and_near_ties_are_exact():
    # probe 0 so that R = r exactly.  The point (0, 0, 2) of the sphere of radius 2 at the
    # origin lies on the sphere of radius 1 centred at (0, 0, 3): not strictly outside.
    pts = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0]], dtype=np.float32)
    xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 3.0]])
    mask = sr.exposed_mask(xyz, np.array([2.0, 1.0]), pts, 0, probe=0.0)
    assert not mask[0] and mask[1]
    # near-ties: the ball moved by one ulp of its centre either way
    for z, exposed in ((np.nextafter(3.0, 4.0), True), (np.nextafter(3.0, 2.0), False)):
        xyz[1, 2] = z
        assert sr.exposed_mask(xyz, np.array([2.0, 1.0]), pts, 0, probe=0.0)[0] == exposed
