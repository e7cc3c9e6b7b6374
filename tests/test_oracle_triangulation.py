"""Pins of the oracle's Steps 1-2: exact predicates against rational arithmetic,
brute-force regularity of the triangulation, Euler characteristics of the dual complex
and the paper's simplex counts."""
import json
import math
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
PAPER = json.load(open(os.path.join(HERE, "golden", "paper_values.json")))
P = 1.4


# ---------------------------------------------------------------- predicates vs Fractions
def _fr_orient(p):
    a, b, c, d = [[Fr(x) for x in q[:3]] for q in p]
    m = [[b[k] - a[k] for k in range(3)], [c[k] - a[k] for k in range(3)], [d[k] - a[k] for k in range(3)]]
    return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
            + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))


def _fr_det(M):
    M = [row[:] for row in M]
    n = len(M)
    det = Fr(1)
    for c in range(n):
        piv = next((r for r in range(c, n) if M[r][c] != 0), None)
        if piv is None:
            return Fr(0)
        if piv != c:
            M[c], M[piv] = M[piv], M[c]
            det = -det
        det *= M[c][c]
        for r in range(c + 1, n):
            f = M[r][c] / M[c][c]
            for k in range(c, n):
                M[r][k] -= f * M[c][k]
    return det


def _fr_power(p):
    """Sign of the power of p[4] w.r.t. the orthosphere of p[0..3] (positively oriented)
    from the lifted 5x5 determinant, written independently with Gaussian elimination."""
    rows = []
    for q in p:
        x, y, z, R = [Fr(v) for v in q]
        rows.append([x, y, z, x * x + y * y + z * z - R * R, Fr(1)])
    # for a positively oriented tetrahedron, det < 0 <=> p4 strictly inside the orthosphere
    o = _fr_orient(p[:4])
    d5 = _fr_det(rows)
    return d5, o


def test_predicates_match_rational_arithmetic(orc):
    rng = np.random.default_rng(7)
    for t in range(300):
        pts = np.concatenate([rng.normal(scale=3, size=(5, 3)), rng.uniform(1.2, 3.3, size=(5, 1))], 1)
        if t % 3 == 0:   # near-degenerate: nudge p4 onto the orthosphere of p0..p3
            pts[4, :3] = pts[0, :3] + 1e-13 * rng.normal(size=3)
            pts[4, 3] = pts[0, 3]
        o = orc.predicate(0, pts, [0, 1, 2, 3])
        fo = _fr_orient(pts[:4])
        assert o == (fo > 0) - (fo < 0)
        if fo == 0:
            continue
        order = [0, 1, 2, 3] if fo > 0 else [1, 0, 2, 3]
        d5, o4 = _fr_power(pts[order + [4]])
        c = orc.predicate(1, pts, order + [4])
        if d5 != 0:
            # negative lifted determinant (with positive orientation) <=> conflict
            assert (c == -1) == ((d5 * (1 if o4 > 0 else -1)) < 0), (t, d5, c)


def test_exact_on_cospherical_points(orc):
    """Five points on one sphere with equal weights: power determinant exactly 0, the
    oracle resolves it by SoS and still yields a valid triangulation of a lattice."""
    # cubic lattice with identical radii: massively degenerate (co-spherical, co-planar)
    g = np.stack(np.meshgrid(np.arange(4), np.arange(4), np.arange(3), indexing="ij"), -1).reshape(-1, 3) * 2.5
    r = np.full(len(g), 1.5)
    o = orc.Oracle(g.astype(float), r)
    tets = o.simplices(4)
    vol = 0.0
    for t in tets:
        a, b, c, d = g[t]
        vol += abs(np.linalg.det(np.stack([b - a, c - a, d - a]))) / 6
    assert vol == pytest.approx(7.5 * 7.5 * 5.0, rel=1e-12)
    assert o.counts()["sos"] > 0
    # areas still agree with the independent per-sphere computation except where the
    # lattice makes the arc arrangement itself degenerate
    a, _, _ = o.areas(grad=False)
    assert np.all(a >= -1e-12) and np.all(a <= 4 * math.pi * 2.9 ** 2 + 1e-9)


# ---------------------------------------------------------------- brute-force regularity
def _orthosphere(pts, R):
    # centre z with |z - p|^2 - R^2 equal for all 4 points; returns z, psi
    p0 = pts[0]
    A = 2 * (pts[1:] - p0)
    b = (pts[1:] ** 2).sum(1) - R[1:] ** 2 - (p0 ** 2).sum() + R[0] ** 2
    z = np.linalg.solve(A, b)
    return z, ((z - p0) ** 2).sum() - R[0] ** 2


@pytest.mark.parametrize("seed", range(5))
def test_triangulation_is_regular_bruteforce(orc, seed):
    rng = np.random.default_rng(seed)
    n = 40
    xyz = rng.uniform(-5, 5, size=(n, 3))
    r = rng.choice([1.2, 1.52, 1.55, 1.7, 1.8], size=n)
    R = r + P
    o = orc.Oracle(xyz, r)
    tets = o.simplices(4)
    red = o.redundant()
    # 1) no point has negative power w.r.t. any tetrahedron's orthosphere
    for t in tets:
        z, psi = _orthosphere(xyz[t], R[t])
        pw = ((xyz - z) ** 2).sum(1) - R ** 2 - psi
        pw[t] = 1.0
        scale = 1.0 + np.abs(((xyz - z) ** 2).sum(1)) + np.abs(psi)
        assert np.all(pw > -1e-9 * scale)
    # 2) the tetrahedra do not overlap and fill the convex hull up to flat hull slivers
    #    (the four far bounding points, weight 0, can hide huge-orthosphere slivers on the
    #    hull; they never touch a simplex of the dual complex, whose orthospheres have
    #    non-positive power)
    from scipy.spatial import ConvexHull
    vol = sum(abs(np.linalg.det(np.stack([xyz[t[1]] - xyz[t[0]], xyz[t[2]] - xyz[t[0]], xyz[t[3]] - xyz[t[0]]]))) / 6
              for t in tets)
    hull = ConvexHull(xyz).volume
    assert hull * (1 - 1e-3) <= vol <= hull * (1 + 1e-12)
    samples = rng.uniform(-5, 5, size=(4000, 3))
    inside = np.zeros(len(samples), int)
    for t in tets:
        T = np.stack([xyz[t[1]] - xyz[t[0]], xyz[t[2]] - xyz[t[0]], xyz[t[3]] - xyz[t[0]]], 1)
        lam = np.linalg.solve(T, (samples - xyz[t[0]]).T).T
        bary = np.concatenate([1 - lam.sum(1, keepdims=True), lam], 1)
        inside += np.all(bary > 1e-9, 1)
    assert inside.max() <= 1
    # 3) a point is absent from the triangulation iff its power cell is empty (LP)
    from scipy.optimize import linprog
    for i in range(n):
        A = 2 * (xyz - xyz[i])
        b = (xyz ** 2).sum(1) - R ** 2 - (xyz[i] ** 2).sum() + R[i] ** 2
        A = np.delete(A, i, 0)
        b = np.delete(b, i)
        res = linprog(np.zeros(3), A_ub=A, b_ub=b - 1e-9, bounds=[(None, None)] * 3, method="highs")
        assert (res.status == 0) == (not red[i]), i


def test_nested_balls_are_not_in_the_complex(orc):
    # a ball inside a larger one keeps a (non-empty) power cell but its Laguerre-
    # intersection cell is empty: it is not a vertex of C and has zero area
    xyz = np.array([[0, 0, 0], [0.3, 0.1, 0.0], [5.0, 0, 0], [5.05, 0.0, 0.02]])
    r = np.array([1.8, 1.2, 1.5, 1.2])
    o = orc.Oracle(xyz, r)
    assert list(o.simplices(0)) == [0, 2]
    a, _, g = o.areas()
    assert a[1] == 0 and a[3] == 0 and np.all(g[1] == 0) and np.all(g[3] == 0)
    gb, _ = orc.gauss_bonnet(xyz, r)
    assert np.allclose(a, gb, rtol=1e-12)


# ---------------------------------------------------------------- Euler characteristic of C
def _euler(o):
    return sum((-1) ** d * len(o.simplices(d)) for d in range(4))


def test_euler_characteristic_blob_ring_shell(orc):
    rng = np.random.default_rng(0)
    # blob: compact cluster of strongly overlapping balls -> contractible union, chi = 1
    blob = rng.normal(scale=1.2, size=(25, 3))
    assert _euler(orc.Oracle(blob, np.full(25, 1.5))) == 1
    # ring: balls on a circle, neighbours overlapping -> union is a solid torus, chi = 0
    k = 24
    th = 2 * math.pi * np.arange(k) / k
    ring = np.stack([12 * np.cos(th), 12 * np.sin(th), 0.01 * np.sin(3 * th)], 1) + 1e-6 * rng.normal(size=(k, 3))
    assert _euler(orc.Oracle(ring, np.full(k, 0.6))) == 0
    # hollow shell: balls covering a sphere -> a thick spherical shell with a cavity, chi = 2
    m = 300
    idx = np.arange(m) + 0.5
    z = 1 - 2 * idx / m
    rr = np.sqrt(1 - z * z)
    a = math.pi * (1 + 5 ** 0.5) * idx
    sh = 14 * np.stack([rr * np.cos(a), rr * np.sin(a), z], 1) + 1e-6 * rng.normal(size=(m, 3))
    assert _euler(orc.Oracle(sh, np.full(m, 1.0))) == 2


def test_paper_simplex_counts(orc, gen):
    """A 1700-atom heavy-atom molecule has >11200 tetrahedra, >22600 triangles and
    >13000 edges (paper, Sec. on simplex extraction); the synthetic heavy-atom globule
    lands within 15 % of those per-atom rates."""
    pin = PAPER["simplex_counts_1700"]
    m = gen.globule(pin["atoms"], 0)
    r = np.where(m.radii == 1.2, 1.7, m.radii)   # heavy atoms only: no hydrogen radii
    c = orc.Oracle(m.coords, r).counts()
    for key, ref in (("rt_tets", pin["tets"]), ("rt_tris", pin["triangles"]), ("rt_edges", pin["edges"])):
        assert abs(c[key] / ref - 1) < 0.15, (key, c[key], ref)
