"""Pins of the oracle's molecular volume (per-atom power-cell volumes vol(B_i cap L_i), their
sum = the volume of the union of balls, and d(volume)/dx) against closed forms, Monte Carlo
assignment of random points to power cells, finite differences and rigid-motion identities."""
import math

import numpy as np
import pytest

P = 1.4


def ball_cap(R, h):
    """Volume of the cap of height h (0 <= h <= 2R) cut from a ball of radius R."""
    return math.pi * h * h * (3 * R - h) / 3.0


def test_isolated_sphere(orc):
    v, tot, g = orc.Oracle(np.zeros((1, 3)), np.array([1.52])).volumes()
    R = 1.52 + P
    assert v[0] == pytest.approx(4.0 / 3.0 * math.pi * R ** 3, rel=1e-14)
    assert np.all(g == 0)


@pytest.mark.parametrize("d", [0.7, 2.0, 3.3, 5.0, 6.1])
def test_two_spheres_closed_form(orc, d):
    r = np.array([1.2, 1.8])
    R1, R2 = r + P
    xyz = np.array([[0.0, 0.0, 0.0], [d, 0.0, 0.0]])
    v, tot, g = orc.Oracle(xyz, r).volumes()
    if d >= R1 + R2:   # disjoint balls
        assert v == pytest.approx(4.0 / 3.0 * math.pi * np.array([R1, R2]) ** 3, rel=1e-14)
        assert np.all(g == 0)
        return
    # the radical plane at distance t1 from p1 splits the lens between the two atoms
    t1 = (d * d + R1 * R1 - R2 * R2) / (2 * d)
    t2 = d - t1
    V1 = 4.0 / 3.0 * math.pi * R1 ** 3 - ball_cap(R1, R1 - t1)
    V2 = 4.0 / 3.0 * math.pi * R2 ** 3 - ball_cap(R2, R2 - t2)
    assert v[0] == pytest.approx(V1, rel=1e-12)
    assert v[1] == pytest.approx(V2, rel=1e-12)
    # union volume of two balls (inclusion-exclusion with the lens)
    lens = ball_cap(R1, R1 - t1) + ball_cap(R2, R2 - t2)
    assert tot == pytest.approx(4.0 / 3.0 * math.pi * (R1 ** 3 + R2 ** 3) - lens, rel=1e-12)
    # moving p1 towards p2 shrinks the union at the rate of the disk area pi rho^2
    rho2 = R1 * R1 - t1 * t1
    assert g[0] == pytest.approx([-math.pi * rho2, 0, 0], abs=1e-10)
    assert g[1] == pytest.approx([math.pi * rho2, 0, 0], abs=1e-10)


def test_nested_ball_has_no_volume(orc):
    xyz = np.array([[0.0, 0.0, 0.0], [0.3, 0.0, 0.0]])
    r = np.array([1.9, 1.2])
    v, tot, g = orc.Oracle(xyz, r).volumes()
    assert v[1] == 0.0
    assert v[0] == pytest.approx(4.0 / 3.0 * math.pi * (1.9 + P) ** 3, rel=1e-12)
    assert np.all(g[1] == 0)


def _mc(xyz, radii, m, seed):
    """Monte Carlo power-cell volumes: uniform points in the bounding box, each point in the
    union assigned to the atom of least power distance |x - p|^2 - R^2."""
    R = radii + P
    lo = (xyz - R[:, None]).min(0)
    hi = (xyz + R[:, None]).max(0)
    box = float(np.prod(hi - lo))
    rng = np.random.default_rng(seed)
    counts = np.zeros(len(R))
    done = 0
    while done < m:
        k = min(200_000, m - done)
        x = lo + (hi - lo) * rng.random((k, 3))
        pw = ((x[:, None, :] - xyz[None, :, :]) ** 2).sum(-1) - R[None, :] ** 2
        j = pw.argmin(1)
        inside = pw[np.arange(k), j] <= 0
        counts += np.bincount(j[inside], minlength=len(R))
        done += k
    f = counts / m
    return f * box, np.sqrt(f * (1 - f) / m) * box


def test_monte_carlo_power_cells(orc, gen):
    m = gen.globule(30, 3)
    v, tot, _ = orc.Oracle(m.coords, m.radii).volumes(grad=False)
    mc, sig = _mc(m.coords, m.radii, 3_000_000, 1)
    assert np.all(np.abs(v - mc) <= 5 * sig + 1e-9), np.max(np.abs(v - mc) / (sig + 1e-12))
    assert abs(tot - mc.sum()) <= 5 * math.sqrt((sig ** 2).sum())
    assert tot == pytest.approx(v.sum(), rel=1e-14)
    R = m.radii + P
    assert np.all(v >= 0) and np.all(v <= 4.0 / 3.0 * math.pi * R ** 3 * (1 + 1e-12))


def test_volume_gradient_finite_differences(orc, gen):
    m = gen.globule(60, 4)
    _, tot, g = orc.Oracle(m.coords, m.radii).volumes()
    h = 1e-5
    rng = np.random.default_rng(0)
    for j in rng.choice(m.n, 8, replace=False):
        for c in range(3):
            xp, xm = m.coords.copy(), m.coords.copy()
            xp[j, c] += h
            xm[j, c] -= h
            fd = (orc.Oracle(xp, m.radii).volumes(grad=False)[1] - orc.Oracle(xm, m.radii).volumes(grad=False)[1]) / (2 * h)
            assert g[j, c] == pytest.approx(fd, rel=1e-6, abs=1e-6), (j, c)


def test_volume_rigid_motion(orc, gen):
    m = gen.globule(120, 5)
    v, tot, g = orc.Oracle(m.coords, m.radii).volumes()
    # translation and rotation invariance of the union volume
    assert np.abs(g.sum(0)).max() <= 1e-9 * np.abs(g).sum()
    torque = np.cross(m.coords, g).sum(0)
    assert np.abs(torque).max() <= 1e-8 * (np.abs(np.cross(m.coords, g)).sum())
    q, _ = np.linalg.qr(np.random.default_rng(1).normal(size=(3, 3)))
    v2, tot2, _ = orc.Oracle(m.coords @ q.T + 3.0, m.radii).volumes(grad=False)
    assert np.allclose(v2, v, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("seed", [2, 6])
def test_weighted_volume_gradient_finite_differences(orc, gen, seed):
    """d(sum_i w_i V_i)/dx for random weights against central differences of the weighted sum
    of the per-atom volumes (every component of a sample of atoms), on a small globule."""
    m = gen.globule(80, seed)
    w = np.random.default_rng(seed).uniform(-1.0, 2.0, m.n)
    v0, _, g = orc.Oracle(m.coords, m.radii).volumes(weights=w)
    h = 1e-5
    for i in np.random.default_rng(seed + 1).choice(m.n, 12, replace=False):
        for k in range(3):
            xp, xm = m.coords.copy(), m.coords.copy()
            xp[i, k] += h
            xm[i, k] -= h
            fd = (w @ orc.Oracle(xp, m.radii).volumes(grad=False)[0] - w @ orc.Oracle(xm, m.radii).volumes(grad=False)[0]) / (2 * h)
            assert abs(fd - g[i, k]) <= 1e-5 * max(1.0, abs(g[i, k])), (i, k, fd, g[i, k])


def test_weighted_volume_gradient_identities(orc, gen):
    """Unit weights give the union volume's gradient; a weight on one atom alone gives the
    gradient of that atom's volume, whose entries sum to zero (translation) and whose torque
    about the origin vanishes (rotation)."""
    m = gen.globule(150, 9)
    o = orc.Oracle(m.coords, m.radii)
    _, _, g1 = o.volumes()
    _, _, gw = o.volumes(weights=np.ones(m.n))
    assert np.allclose(gw, g1, rtol=0, atol=1e-11)
    for i in (3, 77, 140):
        e = np.zeros(m.n)
        e[i] = 1.0
        _, _, gi = o.volumes(weights=e)
        scale = np.abs(gi).sum()
        assert scale > 0
        assert np.abs(gi.sum(0)).max() <= 1e-10 * scale
        assert np.abs(np.cross(m.coords, gi).sum(0)).max() <= 1e-10 * scale * np.abs(m.coords).max()
