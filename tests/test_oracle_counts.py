"""Pins of the oracle's bookkeeping functions that the benchmark relies on.

term_counts (the work model of bench.py's roofline) counts the terms of Eq. (sainexclu) that
the area evaluation takes: one vertex term per exposed sphere, one solid angle per (tetrahedron
of C, vertex) and three dihedral angles per such pair, two edge caps per exterior edge (one for
each end) and three triangle terms per triangle whose coefficient is not zero.  On tiny inputs
these are known by hand.  areas_parallel (the all-core CPU baseline) splits the same per-atom
evaluation over threads, so every atom's area must equal areas()'s exactly; a gradient entry
gathers contributions of several atoms, in an order that the threads change, so it agrees to
rounding."""
import math

import numpy as np
import pytest


def _counts(orc, x, r):
    return orc.Oracle(np.array(x, float), np.array(r, float)).term_counts()


def test_term_counts_by_hand(orc):
    assert _counts(orc, [[0, 0, 0]], [1.5]) == dict(vertex_constants=1, solid_angles=0, dihedrals=0,
                                                     edge_caps=0, triangles=0)
    # two overlapping spheres: two exposed vertices, one exterior edge
    assert _counts(orc, [[0, 0, 0], [3, 0, 0]], [1.5, 1.5]) == dict(vertex_constants=2, solid_angles=0, dihedrals=0,
                                                                      edge_caps=2, triangles=0)
    # three pairwise overlapping spheres with a triple intersection: a triangle of C, no tetrahedron
    assert _counts(orc, [[0, 0, 0], [3, 0, 0], [1.5, 2.6, 0]], [1.5] * 3) == dict(
        vertex_constants=3, solid_angles=0, dihedrals=0, edge_caps=6, triangles=3)
    # four spheres on a regular tetrahedron of edge 2 A (R = 2.6 A > circumradius 1.22 A): the
    # tetrahedron is in C; every face has one tetrahedron (coefficient 1/2), every edge is exterior
    a = 2.0
    tet = [[0, 0, 0], [a, 0, 0], [a / 2, a * math.sqrt(3) / 2, 0], [a / 2, a * math.sqrt(3) / 6, a * math.sqrt(2 / 3)]]
    assert _counts(orc, tet, [1.2] * 4) == dict(vertex_constants=4, solid_angles=4, dihedrals=12, edge_caps=12,
                                                 triangles=12)
    # a fifth sphere well apart adds one vertex term only
    assert _counts(orc, tet + [[20, 0, 0]], [1.2] * 5)["vertex_constants"] == 5


def test_term_counts_scale_with_the_complex(orc, gen):
    """On a globule: solid angles are at most 4 per tetrahedron of C, dihedral angles at most
    12 (both ends of each of its 6 edges, an even number), edge caps at most 2 per edge of C,
    triangle terms 3 per counted triangle."""
    m = gen.globule(304, 0)
    o = orc.Oracle(m.coords, m.radii)
    t, c = o.term_counts(), o.counts()
    assert t["solid_angles"] <= 4 * c["K3"]
    assert t["dihedrals"] <= 12 * c["K3"] and t["dihedrals"] % 2 == 0
    assert t["edge_caps"] <= 2 * c["K1"] and t["edge_caps"] % 2 == 0
    assert t["triangles"] <= 3 * c["K2"] and t["triangles"] % 3 == 0
    assert 0 < t["vertex_constants"] <= c["K0"]


def test_parallel_area_stage_equals_the_serial_one(orc, gen):
    m = gen.globule(304, 3)
    o = orc.Oracle(m.coords, m.radii)
    a, tot, g = o.areas(grad=True)
    ap, totp, gp, used = o.areas_parallel(4, grad=True)
    assert np.array_equal(a, ap)
    assert np.max(np.abs(g - gp)) <= 1e-12 * np.max(np.abs(g))
    assert totp == pytest.approx(tot, rel=1e-13)
    assert used >= 1
