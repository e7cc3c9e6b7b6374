"""The seeded synthetic inputs follow their stated recipe: bond length and non-bonded minimum
distances of the globule chain, the radii mixes, the RNA helix, the shell's bounds, the
jitter, determinism per seed, unit sphere points and Poisson arrivals."""
import numpy as np
import pytest
from scipy.spatial import cKDTree


def _pairs_within(x, d):
    return cKDTree(x).query_pairs(d, output_type="ndarray")


def test_globule_chain_geometry_and_radii(gen):
    m = gen.globule(5000, 7)
    x, r = m.coords, m.radii
    bonds = np.linalg.norm(np.diff(x, axis=0), axis=1)
    assert np.all(np.abs(bonds - 1.53) <= 1e-5)
    p = _pairs_within(x, 2.6 - 1e-5)
    sep = np.abs(p[:, 0] - p[:, 1])
    assert np.all(sep <= 2)                                   # only bonded neighbours and their next
    d2 = np.linalg.norm(x[p[sep == 2, 0]] - x[p[sep == 2, 1]], axis=1)
    assert np.all(d2 >= 2.2 - 1e-5)
    frac = {v: np.mean(np.isclose(r, v)) for v in (1.2, 1.7, 1.55, 1.52, 1.8)}
    assert sum(frac.values()) == pytest.approx(1.0)
    for v, want in ((1.2, 0.50), (1.7, 0.30), (1.55, 0.09), (1.52, 0.10), (1.8, 0.01)):
        assert abs(frac[v] - want) < 4 * np.sqrt(want * (1 - want) / m.n) + 1e-3, (v, frac[v])


def test_rna_helix(gen):
    m = gen.rna(3200, 2)
    x, r = m.coords, m.radii
    p = np.isclose(r, 1.9)
    assert abs(p.sum() - m.n / 32) <= 2                       # one P per 32-atom nucleotide
    # the P atoms lie on two helices of radius 20 A about a common axis: fit the axis by PCA
    xp = x[p] - x[p].mean(0)
    axis = np.linalg.svd(xp, full_matrices=False)[2][0]
    rad = np.linalg.norm(xp - np.outer(xp @ axis, axis), axis=1)
    assert np.median(np.abs(rad - 20.0)) < 0.5
    assert set(np.unique(np.round(r[~p], 3))) <= {1.2, 1.7, 1.55, 1.52}


def test_shell_bounds(gen):
    m = gen.shell(20000, 1, r_out=60.0, thickness=14.0, chain=100)
    d = np.linalg.norm(m.coords - m.coords.mean(0), axis=1)
    assert d.max() - d.min() <= m.extent * 0.3 + 16.0          # a shell, not a ball
    assert np.min(d) > 0.3 * np.max(d)


def test_jitter_and_determinism(gen):
    a, b, c = gen.globule(600, 3), gen.globule(600, 3), gen.globule(600, 4)
    assert np.array_equal(a.coords, b.coords) and np.array_equal(a.radii, b.radii)
    assert not np.array_equal(a.coords, c.coords)
    # no exactly co-planar coordinates: every coordinate carries its own jitter
    assert len(np.unique(a.coords[:, 2])) == a.n


def test_sphere_points_and_arrivals(gen):
    s = gen.sphere_points(960)
    assert s.shape == (960, 3)
    assert np.allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-6)
    assert np.linalg.norm(s.mean(0)) < 0.01                   # spread over the whole sphere
    t = gen.poisson_arrivals(4000, 500.0, seed=1)
    assert np.all(np.diff(t) >= 0)
    assert t[-1] / len(t) == pytest.approx(1 / 500.0, rel=0.1)
