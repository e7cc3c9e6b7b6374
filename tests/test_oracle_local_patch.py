"""Pins oracle.local_patch, which the largest parity checks rely on (the sampled atoms of the
1,000,000-atom shell, the finite differences of the 20,000-atom trajectory, the CPU
reference arm): the oracle run on the atoms near a centre atom i must give i exactly the
area and gradient entry that the oracle run on the whole molecule gives.

Why it holds: every simplex of the dual complex that contains i lies in B_i, where only the
balls overlapping B_i can win the power comparison (a point of B_i has non-positive power
for i and positive power for any ball that misses B_i), so the terms of every A_j that move
with p_i, and A_i itself, are decided by those balls alone.  A cutoff of R_i + R_max
therefore suffices; the default 4 R_max + 1 A and the 14 A of the reference arm have margin.
The negative control drops overlapping neighbours (a cutoff from the radii without the
probe), which must change the results."""
import numpy as np
import pytest

P = 1.4


def _groups(m, seed, n_groups=10, per=4):
    """n_groups random atoms, each with its per - 1 nearest atoms (per * n_groups atoms, so
    that one patch serves several checked atoms)."""
    rng = np.random.default_rng(seed)
    out = []
    for c in rng.choice(m.n, n_groups, replace=False):
        d = np.linalg.norm(m.coords - m.coords[c], axis=1)
        out.append(np.argsort(d)[:per])
    return out


@pytest.fixture(scope="module", params=["globule5000", "shell1500", "rna1200"])
def case(request, orc, gen):
    if request.param == "globule5000":
        m = gen.globule(5000, 0)
    elif request.param == "shell1500":
        m = gen.shell(1500, 2, r_out=40.0, thickness=12.0, chain=100)
    else:
        m = gen.rna(1200, 1)
    a, _, g = orc.sasa(m.coords, m.radii)
    return m, a, g


def _patch_outputs(orc, m, centres, cutoff):
    idx = orc.local_patch(m.coords, m.radii, centres, cutoff=cutoff)
    a, _, g = orc.sasa(m.coords[idx], m.radii[idx])
    pos = np.searchsorted(idx, centres)
    assert np.array_equal(idx[pos], centres)
    return a[pos], g[pos]


@pytest.mark.parametrize("cutoff", [None, 14.0])
def test_patch_reproduces_full_molecule(orc, case, cutoff):
    m, fa, fg = case
    checked = 0
    for grp in _groups(m, 7):
        a, g = _patch_outputs(orc, m, grp, cutoff)
        # identical up to the summation order of the oracle's terms (1e-12 relative)
        assert np.all(np.abs(a - fa[grp]) <= 1e-12 * np.maximum(fa[grp], 1.0)), (grp, a, fa[grp])
        gn = np.linalg.norm(fg[grp], axis=1)
        assert np.all(np.linalg.norm(g - fg[grp], axis=1) <= 1e-12 * np.maximum(gn, 1.0)), grp
        checked += len(grp)
    assert checked >= 40


def test_patch_of_overlapping_neighbours_suffices(orc, case):
    """The smallest cutoff the argument allows, R_i + R_max, already reproduces A_i and g_i."""
    m, fa, fg = case
    rmax = float(m.radii.max()) + P
    for grp in _groups(m, 8, n_groups=5, per=1):
        i = int(grp[0])
        a, g = _patch_outputs(orc, m, grp, m.radii[i] + P + rmax)
        assert abs(a[0] - fa[i]) <= 1e-12 * max(fa[i], 1.0)
        assert np.linalg.norm(g[0] - fg[i]) <= 1e-12 * max(np.linalg.norm(fg[i]), 1.0)


def test_negative_control_without_probe_fails(orc, case):
    """A plausible mistake, a cutoff from the van der Waals radii alone (2 r_max, the probe
    forgotten), drops overlapping neighbours; the check above must then fail for several of five exposed
    atoms (one failure is enough to fail a parity run)."""
    m, fa, fg = case
    cut = 2.0 * float(m.radii.max())
    wrong = total = 0
    exposed = np.nonzero(fa > 1.0)[0]     # a buried atom can stay buried with fewer neighbours
    for i in np.random.default_rng(9).choice(exposed, 5, replace=False):
        i = int(i)
        a, g = _patch_outputs(orc, m, np.array([i]), cut)
        bad_a = abs(a[0] - fa[i]) > 1e-12 * max(fa[i], 1.0)
        bad_g = np.linalg.norm(g[0] - fg[i]) > 1e-12 * max(np.linalg.norm(fg[i]), 1.0)
        wrong += bool(bad_a or bad_g)
        total += 1
    assert wrong >= 2, (wrong, total)
