"""GPU tests of the autograd wrappers, the CUDA-graph trajectory and the serving loop."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
P = 1.4


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _grad_close(g, ref):
    err = np.linalg.norm(g - ref, axis=1)
    return np.all(err <= 1e-3 * np.maximum(np.linalg.norm(ref, axis=1), 1e-2))


def test_nonpolar_energy_autograd(torch_cuda, orc, gen):
    torch = torch_cuda
    from paper_2401_10462_gb300 import autograd as ag
    m = gen.globule(500, 2)
    x = torch.as_tensor(m.coords, device="cuda").requires_grad_(True)
    r = torch.as_tensor(m.radii, device="cuda")
    e, areas = ag.nonpolar_energy(x, r)
    e.backward()
    ra, rtot, rg = orc.sasa(m.coords, m.radii)
    assert abs(e.item() - 0.005 * rtot) <= 1e-6 * 0.005 * rtot
    assert _grad_close(x.grad.cpu().numpy(), 0.005 * rg)


def test_sasa_areas_vjp_recomputes(torch_cuda, orc, gen):
    torch = torch_cuda
    from paper_2401_10462_gb300 import autograd as ag
    m = gen.globule(400, 3)
    c = np.random.default_rng(0).uniform(-1, 1, m.n)
    x = torch.as_tensor(m.coords, device="cuda").requires_grad_(True)
    r = torch.as_tensor(m.radii, device="cuda")
    a = ag.sasa_areas(x, r)
    (a * torch.as_tensor(c, device="cuda")).sum().backward()
    _, _, rg = orc.sasa(m.coords, m.radii, weights=c)
    assert _grad_close(x.grad.cpu().numpy(), rg)


def test_graphed_trajectory_matches_eager_and_oracle(torch_cuda, orc, gen):
    torch = torch_cuda
    from paper_2401_10462_gb300 import autograd as ag, api
    m = gen.globule(2000, 5)
    x0 = torch.as_tensor(m.coords, device="cuda")
    r = torch.as_tensor(m.radii, device="cuda")
    tr = ag.GraphedTrajectory(x0, r, sigma=0.01, seed=7).capture()
    tr.replay(20)
    torch.cuda.synchronize()
    tr.check()
    x = tr.x.clone()
    # eager recomputation at the final positions gives the same energy and gradient
    ctx = api.Context()
    a = torch.empty(m.n, dtype=torch.float64, device="cuda")
    g = torch.empty((m.n, 3), dtype=torch.float64, device="cuda")
    ctx.compute(x, r, a, g, weights=torch.full((m.n,), 0.005, dtype=torch.float64, device="cuda"))
    ctx.status_sync()
    assert torch.equal(g, tr.grad)
    assert abs((a * 0.005).sum().item() - tr.energy.item()) <= 1e-12 * abs(tr.energy.item())
    # the displacement statistics are those of sigma = 0.01 A per coordinate per step
    d = (x - x0).cpu().numpy()
    assert abs(d.std() / (0.01 * np.sqrt(20)) - 1) < 0.05
    # oracle gradient at the final positions
    xn = x.cpu().numpy()
    _, _, rg = orc.sasa(xn, m.radii)
    assert _grad_close(tr.grad.cpu().numpy(), 0.005 * rg)


@pytest.mark.parametrize("resident", [0, 100_000])
def test_serving_results_same_alone_and_in_the_mix(torch_cuda, gen, resident):
    """Continuous batching (zero-copy outputs, per-molecule ready flags; with resident
    Verlet lists or without): every request's outputs equal those of the same request run
    alone through a fresh server without resident state, bit for bit without resident lists
    and within the stated tolerances with them (a context with a skin keeps only the balls
    that overlap in its cells, a plain one also near-tangent ones, which can change the
    rounding)."""
    torch = torch_cuda
    from paper_2401_10462_gb300 import serve, inputs
    reqs, mols = serve.request_pool(48, seed=3, pool=6, lo=300, hi=6000)
    rate = 400.0
    t = inputs.poisson_arrivals(len(reqs), rate, seed=1)
    for r_, ti in zip(reqs, t):
        r_.arrival = float(ti)
    srv = serve.Server(slots=3, slot_atoms=20000, resident_atoms=resident)
    stats = srv.run(reqs)
    assert stats["requests"] == 48 and stats["failed"] == 0 and stats["p99_ms"] >= stats["p50_ms"] > 0
    if resident:
        # frames of a molecule 0.01 A apart: most repeat requests reuse their lists
        assert stats["lists_reused"] >= 48 - 6 - 10, stats
    srv.close()
    for q in reqs[:12]:
        alone = serve.Request(q.rid, q.coords, q.radii)
        srv1 = serve.Server(slots=1, slot_atoms=20000)
        srv1.run([alone], realtime=False)
        srv1.close()
        if resident:
            assert np.all(np.abs(alone.areas - q.areas) <= 1e-4 * np.maximum(alone.areas, 1.0))
            assert _grad_close(q.grad, alone.grad)
        else:
            assert np.array_equal(alone.areas, q.areas) and np.array_equal(alone.grad, q.grad)


def test_resident_batch_flags_and_reuse(torch_cuda, gen):
    """dsasa_compute_batch_resident through the C ABI: zero-copy outputs in pinned host
    memory match dsasa_compute_batch's within the stated tolerances; every molecule's ready
    flag is set; the second call
    with coordinates moved by 0.01 A reuses every molecule's lists, a molecule moved by more
    than half the skin rebuilds its own, and a molecule without a slot (-1) has none."""
    torch = torch_cuda
    from paper_2401_10462_gb300 import api
    mols = [gen.globule(300, 1), gen.rna(640, 2), gen.globule(1000, 3)]
    xyz = np.concatenate([m.coords for m in mols])
    r = np.concatenate([m.radii for m in mols])
    off = np.cumsum([0] + [m.n for m in mols])
    n = len(r)
    ctx = api.Context(skin=1.0)
    arena = api.Arena(10_000)
    base = np.array([0, 2000, -1])
    ha = torch.empty(n, dtype=torch.float64, pin_memory=True)
    hg = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
    ready = torch.zeros(3, dtype=torch.int32, pin_memory=True)
    ref = api.Context()
    a = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(0)
    for step, shift in enumerate((0.0, 0.01, 0.01)):
        xyz = xyz + shift * rng.normal(size=xyz.shape)
        if step == 2:
            xyz[off[1]:off[2]] += 0.6                     # molecule 1 moves rigidly by more than skin / 2
        x = torch.as_tensor(xyz, device="cuda")
        rr = torch.as_tensor(r, device="cuda")
        ready.zero_()
        ctx.compute_batch_resident(off, x, rr, ha, hg, arena=arena, arena_base=base, mol_ready=ready)
        ctx.status_sync()
        assert ready.tolist() == [1, 1, 1]
        reused = ctx.batch_reused(3).tolist()
        assert reused == ([False] * 3 if step == 0 else ([True, True, False] if step == 1 else [True, False, False]))
        ref.compute_batch(off, x, rr, a, g)
        ref.status_sync()
        ra, rg = a.cpu().numpy(), g.cpu().numpy()
        assert np.all(np.abs(ha.numpy() - ra) <= 1e-4 * np.maximum(ra, 1.0))
        assert _grad_close(hg.numpy(), rg)
    ctx.close()
    ref.close()
    arena.close()


def test_serving_reports_the_failing_request(torch_cuda, gen):
    """A request with a non-finite coordinate in a batch of six: it alone gets the input
    error status (its outputs are meaningless), the others their normal results."""
    from paper_2401_10462_gb300 import serve
    reqs, _ = serve.request_pool(6, seed=4, pool=3, lo=300, hi=2000)
    bad = reqs[2]
    bad.coords = bad.coords.copy()
    bad.coords[5, 1] = np.nan
    srv = serve.Server(slots=1, slot_atoms=20000)
    st = srv.run(reqs, realtime=False)
    assert st["failed"] == 1 and bad.status == 8
    for r_ in reqs:
        if r_ is not bad:
            assert r_.status == 0 and np.all(np.isfinite(r_.areas)) and np.all(np.isfinite(r_.grad))
            alone = serve.Request(r_.rid, r_.coords, r_.radii)
            srv.run([alone], realtime=False)
            assert np.array_equal(alone.areas, r_.areas)
    srv.close()
