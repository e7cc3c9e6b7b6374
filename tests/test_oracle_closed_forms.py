"""Pins of the oracle against closed forms, the paper's printed numbers and an
independent exact area (Gauss-Bonnet over exposed arcs) - no GPU needed."""
import json
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
PAPER = json.load(open(os.path.join(HERE, "golden", "paper_values.json")))
P = 1.4


def test_isolated_sphere(orc):
    # A = 4 pi (r + p)^2 exactly, gradient 0
    for r in (1.2, 1.52, 1.7, 1.9):
        a, tot, g = orc.sasa(np.array([[0.3, -2.0, 7.1]]), np.array([r]))
        assert a[0] == pytest.approx(4 * math.pi * (r + P) ** 2, rel=1e-15)
        assert np.all(g == 0)


def _cap(Ri, Rj, d):
    t = (d * d + Ri * Ri - Rj * Rj) / (2 * d)
    return 2 * math.pi * Ri * (Ri - t)


@pytest.mark.parametrize("r1,r2,d", [(1.5, 1.7, 4.0), (1.2, 1.9, 2.1), (1.7, 1.7, 0.9), (1.52, 1.2, 5.0)])
def test_two_spheres_closed_form(orc, r1, r2, d):
    R1, R2 = r1 + P, r2 + P
    u = np.array([0.6, -0.48, 0.64])
    xyz = np.array([[1.0, 2.0, 3.0], [1.0, 2.0, 3.0] + d * u])
    a, tot, g = orc.sasa(xyz, np.array([r1, r2]))
    e1 = 4 * math.pi * R1 ** 2 - _cap(R1, R2, d)
    e2 = 4 * math.pi * R2 ** 2 - _cap(R2, R1, d)
    if d <= abs(R1 - R2):
        e1, e2 = (0.0, 4 * math.pi * R2 ** 2) if R1 < R2 else (4 * math.pi * R1 ** 2, 0.0)
    assert a[0] == pytest.approx(e1, rel=1e-12, abs=1e-11)
    assert a[1] == pytest.approx(e2, rel=1e-12, abs=1e-11)
    # d(A1 + A2)/d(p2) along the axis = 2 pi (R1 t2 + R2 t1) / d when the spheres cut
    if abs(R1 - R2) < d < R1 + R2:
        t1 = (d * d + R1 * R1 - R2 * R2) / (2 * d)
        t2 = d - t1
        dAdd = 2 * math.pi * (R1 * t2 + R2 * t1) / d
        assert g[1] @ u == pytest.approx(dAdd, rel=1e-10)
        assert np.allclose(g[0], -g[1], atol=1e-12)


def test_paper_two_sphere_tangency_jump(orc):
    """Extended radii 2.9 / 3.1: total SASA is smallest at internal tangency and the
    derivative jumps at external tangency by less than 20 A^2 (paper's figure)."""
    pin = PAPER["two_sphere_tangency"]
    R1, R2 = pin["R1"], pin["R2"]
    r = np.array([R1 - P, R2 - P])
    u = np.array([0.0, 0.0, 1.0])

    def total(d):
        return orc.sasa(np.array([[0, 0, 0], d * u]), r, grad=True)

    ds = np.linspace(0.05, 7.0, 300)
    tot = np.array([total(d)[1] for d in ds])
    # minimum is reached once the smaller ball is inside (internal tangency d = R2 - R1)
    i_min = int(np.argmin(tot))
    assert ds[i_min] <= (R2 - R1) + 1e-12
    assert tot[i_min] == pytest.approx(4 * math.pi * R2 ** 2, rel=1e-13)
    inside = (ds > R2 - R1) & (ds < R1 + R2)
    assert np.all(np.diff(tot[inside]) > 0)   # grows as the atoms separate
    # derivative jump at external tangency d = R1 + R2
    dt = R1 + R2
    _, _, g_in = total(dt - 1e-9)
    _, _, g_out = total(dt + 1e-9)
    jump = abs(g_in[1] @ u - g_out[1] @ u)
    assert jump == pytest.approx(4 * math.pi * R1 * R2 / (R1 + R2), rel=1e-6)
    assert jump < pin["max_jump"]
    assert abs(g_out[1] @ u) == 0.0


def _mc_areas(xyz, R, m=400_000, seed=0):
    """Monte-Carlo exposed area per sphere (uniform points on each sphere)."""
    rng = np.random.default_rng(seed)
    out, err = [], []
    for i in range(len(R)):
        v = rng.normal(size=(m, 3))
        v /= np.linalg.norm(v, axis=1)[:, None]
        pts = xyz[i] + R[i] * v
        cov = np.zeros(m, bool)
        for j in range(len(R)):
            if j != i:
                cov |= ((pts - xyz[j]) ** 2).sum(1) < R[j] ** 2
        f = 1 - cov.mean()
        S = 4 * math.pi * R[i] ** 2
        out.append(S * f)
        err.append(S * math.sqrt(max(f * (1 - f), 1e-12) / m))
    return np.array(out), np.array(err)


def test_three_spheres_triangle_term_vs_mc_and_gauss_bonnet(orc):
    rng = np.random.default_rng(3)
    checked = 0
    for trial in range(12):
        xyz = rng.normal(scale=1.6, size=(3, 3))
        r = rng.choice([1.2, 1.52, 1.55, 1.7], size=3)
        R = r + P
        a, _, _ = orc.sasa(xyz, r)
        gb, bad = orc.gauss_bonnet(xyz, r)
        assert bad == 0
        assert np.allclose(a, gb, rtol=1e-10, atol=1e-10)
        mc, err = _mc_areas(xyz, R, seed=trial)
        assert np.all(np.abs(a - mc) <= 4.5 * err + 1e-9)
        checked += 1
    assert checked == 12


def test_triangle_term_against_mc_directly(orc):
    """S_123^(1) (Eq. trianglev) = area of sphere 1 inside balls 2 and 3."""
    p = [np.array([0.0, 0.0, 0.0]), np.array([3.1, 0.4, -0.2]), np.array([1.0, 2.7, 0.9])]
    R = [3.1, 2.9, 3.0]
    S, g = orc.tri_term(p[0], p[1], p[2], *R)
    rng = np.random.default_rng(1)
    m = 2_000_000
    v = rng.normal(size=(m, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    pts = p[0] + R[0] * v
    ins = (((pts - p[1]) ** 2).sum(1) < R[1] ** 2) & (((pts - p[2]) ** 2).sum(1) < R[2] ** 2)
    f = ins.mean()
    full = 4 * math.pi * R[0] ** 2
    assert S == pytest.approx(full * f, abs=4.5 * full * math.sqrt(f * (1 - f) / m))
    # translation invariance of its gradient
    assert np.allclose(g.sum(0), 0, atol=1e-11)


def test_gauss_bonnet_pinned_by_closed_forms(orc):
    # the Gauss-Bonnet cross-check itself: isolated and two-sphere closed forms
    a, bad = orc.gauss_bonnet(np.zeros((1, 3)), np.array([1.55]))
    assert a[0] == pytest.approx(4 * math.pi * (1.55 + P) ** 2, rel=1e-14)
    xyz = np.array([[0, 0, 0], [2.5, 1.0, 0.0]])
    a, bad = orc.gauss_bonnet(xyz, np.array([1.7, 1.2]))
    d = math.hypot(2.5, 1.0)
    assert a[0] == pytest.approx(4 * math.pi * 3.1 ** 2 - _cap(3.1, 2.6, d), rel=1e-12)
    assert a[1] == pytest.approx(4 * math.pi * 2.6 ** 2 - _cap(2.6, 3.1, d), rel=1e-12)


def test_oracle_matches_gauss_bonnet_globules(orc, gen):
    """The whole chain (triangulation, alpha = 0 complex, inclusion-exclusion) against
    the independent exact per-sphere area, per atom to 1e-9 relative."""
    for seed in range(4):
        m = gen.globule(304, seed)
        a, tot, _ = orc.sasa(m.coords, m.radii, grad=False)
        gb, bad = orc.gauss_bonnet(m.coords, m.radii)
        assert bad == 0
        assert np.all(np.abs(a - gb) <= 1e-9 * np.maximum(gb, 1.0))
        assert tot == pytest.approx(gb.sum(), rel=1e-12)


def test_oracle_matches_gauss_bonnet_rna_and_shell(orc, gen):
    for m in (gen.rna(640, 2), gen.shell(1500, 3, r_out=40.0, thickness=12.0, chain=100)):
        a, tot, _ = orc.sasa(m.coords, m.radii, grad=False)
        gb, bad = orc.gauss_bonnet(m.coords, m.radii)
        assert bad == 0
        assert np.all(np.abs(a - gb) <= 1e-9 * np.maximum(gb, 1.0))


def test_dense_points_small_cluster(orc, gen):
    """Shrake-Rupley style golden-spiral sampling (2e5 points per sphere) on N = 40."""
    m = gen.globule(40, 11)
    R = m.radii + P
    a, _, _ = orc.sasa(m.coords, m.radii, grad=False)
    k = 200_000
    idx = np.arange(k) + 0.5
    z = 1 - 2 * idx / k
    rr = np.sqrt(1 - z * z)
    th = math.pi * (1 + 5 ** 0.5) * idx
    v = np.stack([rr * np.cos(th), rr * np.sin(th), z], 1)
    for i in range(m.n):
        pts = m.coords[i] + R[i] * v
        cov = np.zeros(k, bool)
        for j in range(m.n):
            if j != i:
                cov |= ((pts - m.coords[j]) ** 2).sum(1) < R[j] ** 2
        est = 4 * math.pi * R[i] ** 2 * (1 - cov.mean())
        assert abs(est - a[i]) < 2e-3 * 4 * math.pi * R[i] ** 2
