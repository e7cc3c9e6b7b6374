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


def test_serving_results_same_alone_and_in_the_mix(torch_cuda, gen):
    torch = torch_cuda
    from paper_2401_10462_gb300 import serve, inputs
    reqs, mols = serve.request_pool(48, seed=3, pool=6, lo=300, hi=6000)
    rate = 400.0
    t = inputs.poisson_arrivals(len(reqs), rate, seed=1)
    for r_, ti in zip(reqs, t):
        r_.arrival = float(ti)
    srv = serve.Server(slots=3, slot_atoms=20000)
    stats = srv.run(reqs)
    assert stats["requests"] == 48 and stats["p99_ms"] >= stats["p50_ms"] > 0
    # every request alone through a fresh server gives bit-identical outputs
    for q in reqs[:12]:
        alone = serve.Request(q.rid, q.coords, q.radii)
        srv1 = serve.Server(slots=1, slot_atoms=20000)
        srv1.run([alone], realtime=False)
        srv1.close()
        assert np.array_equal(alone.areas, q.areas) and np.array_equal(alone.grad, q.grad)
    srv.close()


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
