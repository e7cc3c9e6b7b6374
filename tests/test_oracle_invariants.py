"""Invariants and finite differences pinning the oracle's areas and gradient."""
import math

import numpy as np
import pytest

P = 1.4


def _rot(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


def test_bounds_translation_rotation_identities(orc, gen):
    m = gen.globule(304, 5)
    R = m.radii + P
    a, tot, g = orc.sasa(m.coords, m.radii)
    assert np.all(a >= 0) and np.all(a <= 4 * math.pi * R ** 2 + 1e-12)
    # sum_j dA/dx_j = 0 and sum_j x_j x dA/dx_j = 0 (rigid-motion invariance of sum A)
    scale = np.abs(g).sum()
    assert np.abs(g.sum(0)).max() < 1e-11 * scale
    c = m.coords - m.coords.mean(0)
    assert np.abs(np.cross(c, g).sum(0)).max() < 1e-10 * scale * 30
    # the same identities hold for one atom's own area (one-hot weights)
    for i in (0, 17, 200):
        w = np.zeros(m.n)
        w[i] = 1.0
        _, _, gi = orc.Oracle(m.coords, m.radii).areas(weights=w)
        assert np.abs(gi.sum(0)).max() < 1e-11 * (1 + np.abs(gi).sum())
        assert np.abs(np.cross(c, gi).sum(0)).max() < 1e-9 * (1 + np.abs(gi).sum())


def test_rigid_motion_and_permutation_invariance(orc, gen):
    m = gen.globule(304, 6)
    o = orc.Oracle(m.coords, m.radii)
    a, tot, g = o.areas()
    Q = _rot(1)
    x2 = m.coords @ Q.T + np.array([13.25, -7.5, 2.125])
    a2, tot2, g2 = orc.sasa(x2, m.radii)
    assert np.allclose(a2, a, rtol=1e-12, atol=1e-11)
    assert np.allclose(g2, g @ Q.T, rtol=1e-9, atol=1e-10)
    perm = np.random.default_rng(2).permutation(m.n)
    o3 = orc.Oracle(m.coords[perm], m.radii[perm])
    a3, _, g3 = o3.areas()
    assert np.allclose(a3, a[perm], rtol=1e-12, atol=1e-11)
    assert np.allclose(g3, g[perm], rtol=1e-10, atol=1e-11)
    for d in range(4):
        s3 = np.sort(perm[o3.simplices(d)].reshape(len(o3.simplices(d)), -1), axis=1)
        s3 = s3[np.lexsort(s3.T[::-1])]
        s = o.simplices(d).reshape(len(o.simplices(d)), -1)
        assert np.array_equal(s3, s)


def test_gradient_is_linear_in_weights(orc, gen):
    m = gen.globule(200, 8)
    o = orc.Oracle(m.coords, m.radii)
    rng = np.random.default_rng(0)
    w1, w2 = rng.uniform(0, 2, m.n), rng.uniform(-1, 1, m.n)
    _, _, g1 = o.areas(weights=w1)
    _, _, g2 = o.areas(weights=w2)
    _, _, g12 = o.areas(weights=w1 + 2 * w2)
    assert np.allclose(g12, g1 + 2 * g2, rtol=1e-10, atol=1e-10)


def _complex(o):
    return tuple(o.simplices(d).tobytes() for d in range(4))


@pytest.mark.parametrize("seed", [0, 1])
def test_central_finite_differences(orc, gen, seed):
    """Central FD (h = 1e-4 A) of the weighted local sum sum_i w_i A_i over atoms near j;
    an atom whose complex changes between x - h and x + h (an 'event') is skipped."""
    m = gen.globule(304, seed)
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 1.5, m.n)
    o = orc.Oracle(m.coords, m.radii)
    _, _, g = o.areas(weights=w)
    K0 = _complex(o)
    h = 1e-4
    checked = 0
    for j in rng.choice(m.n, 8, replace=False):
        near = np.nonzero(((m.coords - m.coords[j]) ** 2).sum(1) < (2 * (3.3 + 0.1)) ** 2)[0]
        fd = np.zeros(3)
        event = False
        for k in range(3):
            vals = []
            for s in (+1, -1):
                x = m.coords.copy()
                x[j, k] += s * h
                ox = orc.Oracle(x, m.radii)
                event |= _complex(ox) != K0
                vals.append((w[near] * ox.areas(grad=False)[0][near]).sum())
            fd[k] = (vals[0] - vals[1]) / (2 * h)
        if event:
            continue
        checked += 1
        assert np.abs(fd - g[j]).max() <= 1e-6 * max(1.0, np.abs(g[j]).max())
    assert checked >= 6
