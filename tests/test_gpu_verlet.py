"""Verlet-skin neighbour lists (contexts with skin > 0): the device reuses each atom's
candidate list while every atom stays within half the skin of its position at the last
rebuild (and n, radii, probe are unchanged), and rebuilds otherwise; the cells and
simplices are recomputed every call, so the results match a rebuild within rounding."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _run(torch, ctx, xyz, r):
    n = len(r)
    a = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    ctx.compute(torch.as_tensor(xyz, device="cuda"), torch.as_tensor(r, device="cuda"), a, g)
    reused = ctx.lists_reused()
    ctx.status_sync()
    return a.cpu().numpy(), g.cpu().numpy(), reused


def _close(a, g, ra, rg):
    assert np.all(np.abs(a - ra) <= 1e-4 * np.maximum(ra, 1.0))
    assert abs(a.sum() - ra.sum()) <= 1e-6 * ra.sum()
    err = np.linalg.norm(g - rg, axis=1)
    assert np.all(err <= 1e-3 * np.maximum(np.linalg.norm(rg, axis=1), 1e-2))


def test_reuse_and_rebuild(torch_cuda, orc, gen):
    torch = torch_cuda
    from paper_2401_10462_gb300 import api
    m = gen.globule(3000, 2)
    rng = np.random.default_rng(0)
    ctx = api.Context(skin=1.0)
    fresh = api.Context()
    x = m.coords.copy()
    a, g, reused = _run(torch, ctx, x, m.radii)
    assert not reused                                   # first call builds the lists
    for step in range(6):
        x = x + rng.normal(scale=0.03, size=x.shape)    # well within half the skin
        a, g, reused = _run(torch, ctx, x, m.radii)
        assert reused
        ra, rg, _ = _run(torch, fresh, x, m.radii)
        _close(a, g, ra, rg)
    # one atom moves by more than half the skin: the device rebuilds
    x[17] += np.array([0.6, 0.0, 0.0])
    a, g, reused = _run(torch, ctx, x, m.radii)
    assert not reused
    ra, rg, _ = _run(torch, fresh, x, m.radii)
    _close(a, g, ra, rg)
    # changed radii: rebuild; then reuse again
    r2 = m.radii.copy()
    r2[5] += 0.05
    _, _, reused = _run(torch, ctx, x, r2)
    assert not reused
    _, _, reused = _run(torch, ctx, x, r2)
    assert reused
    ctx.close()
    fresh.close()


def test_reuse_matches_the_oracle(torch_cuda, orc, gen):
    torch = torch_cuda
    from paper_2401_10462_gb300 import api
    m = gen.globule(304, 6)
    ctx = api.Context(skin=0.8)
    _run(torch, ctx, m.coords, m.radii)
    x = m.coords + np.random.default_rng(1).normal(scale=0.05, size=m.coords.shape)
    a, g, reused = _run(torch, ctx, x, m.radii)
    assert reused
    ra, _, rg = orc.sasa(x, m.radii)
    _close(a, g, ra, rg)
    ctx.close()


def test_graphed_trajectory_with_skin(torch_cuda, gen):
    torch = torch_cuda
    from paper_2401_10462_gb300 import autograd as ag, api
    m = gen.globule(2000, 9)
    x0 = torch.as_tensor(m.coords, device="cuda")
    r = torch.as_tensor(m.radii, device="cuda")
    tr = ag.GraphedTrajectory(x0, r, sigma=0.01, seed=3, skin=1.0).capture()
    tr.replay(200)      # about 0.25 A rms: the lists are reused, then rebuilt on the device
    torch.cuda.synchronize()
    tr.check()
    ctx = api.Context()
    a = torch.empty(m.n, dtype=torch.float64, device="cuda")
    g = torch.empty((m.n, 3), dtype=torch.float64, device="cuda")
    ctx.compute(tr.x, r, a, g, weights=torch.full((m.n,), 0.005, dtype=torch.float64, device="cuda"))
    ctx.status_sync()
    e = (a * 0.005).sum().item()
    assert abs(e - tr.energy.item()) <= 1e-6 * abs(e)
    gg = g.cpu().numpy()
    err = np.linalg.norm(tr.grad.cpu().numpy() - gg, axis=1)
    # carried cells evaluate the same terms from other starting vertices: the two mixed-form
    # results differ by the form's rounding, which reaches 3e-5 absolute where |g| < 0.03
    tol = np.maximum(1e-3 * np.linalg.norm(gg, axis=1), 3e-5 * 0.005)
    bad = np.nonzero(err > tol)[0]
    assert len(bad) == 0, (bad[:5], err[bad[:5]] / 0.005, np.linalg.norm(gg, axis=1)[bad[:5]] / 0.005)
