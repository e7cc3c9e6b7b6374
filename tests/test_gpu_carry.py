"""Carried cells, the incremental update of the complex across MD steps: on calls that reuse
the neighbour lists, each atom's cell starts from the one the previous call built (its faces'
planes at the current positions), is kept when exact predicates certify it, and is then cut by
the new neighbours; a cell that fails the certification is built from the cube.  The
simplices of C must be exactly the oracle's at every step, the areas and gradient those of a
fresh build up to the rounding of the terms, and most cells must carry over small steps."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def api():
    from paper_2401_10462_gb300 import api
    return api


def _sets(rec):
    out = {d: set() for d in range(4)}
    owners = {}
    for r in rec:
        simp = tuple(int(x) for x in r[1:] if x >= 0)
        out[len(simp) - 1].add(simp)
        owners.setdefault(simp, set()).add(int(r[0]))
    return out, owners


def _check_against_oracle(orc, rec, x, r):
    got, owners = _sets(rec)
    o = orc.Oracle(x, r)
    for d in range(4):
        ref = {tuple(int(v) for v in np.atleast_1d(s)) for s in o.simplices(d)}
        assert got[d] == ref, (d, len(got[d]), len(ref), list(got[d] ^ ref)[:5])
    for simp, who in owners.items():
        assert who == set(simp), (simp, who)


def _grad_close(g, ref):
    """The mixed form's gradient bound: 1e-3 relative, and its measured rounding floor of
    3e-5 absolute where |g| < 0.03."""
    err = np.linalg.norm(g - ref, axis=1)
    tol = np.maximum(1e-3 * np.linalg.norm(ref, axis=1), 3e-5)
    bad = np.nonzero(err > tol)[0]
    assert len(bad) == 0, (bad[:5], err[bad[:5]], np.linalg.norm(ref, axis=1)[bad[:5]])


def _run(torch, ctx, x, r, weights=None):
    n = len(r)
    a = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    ctx.compute(torch.as_tensor(x, device="cuda"), torch.as_tensor(r, device="cuda"), a, g)
    carried = ctx.cells_carried()
    reused = ctx.lists_reused()
    ctx.status_sync()
    return a.cpu().numpy(), g.cpu().numpy(), carried, reused


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_carried_complex_is_the_oracles(api, torch_cuda, orc, gen, precision):
    """Three steps of 0.02 A rms per coordinate on a 3,000-atom globule: the complex that the
    carried cells give is exactly the oracle's at each step (about 45 % of the cells carry over
    steps this large)."""
    torch = torch_cuda
    m = gen.globule(3000, 4)
    rng = np.random.default_rng(7)
    ctx = api.Context(precision=precision, skin=1.0, carry=2)
    r = torch.as_tensor(m.radii, device="cuda")
    x = m.coords.copy()
    ctx.export_complex(torch.as_tensor(x, device="cuda"), r)   # builds the lists and the cells
    assert ctx.cells_carried() == 0
    for _ in range(3):
        x = x + rng.normal(scale=0.02, size=x.shape)
        rec = ctx.export_complex(torch.as_tensor(x, device="cuda"), r).cpu().numpy()
        carried = ctx.cells_carried()
        assert ctx.lists_reused()
        ctx.status_sync()
        _check_against_oracle(orc, rec, x, m.radii)
        assert carried >= 0.3 * m.n, carried
    ctx.close()


def test_carry_matches_fresh_cells(api, torch_cuda, orc, gen):
    """Ten steps of 0.01 A on a 2,000-atom globule: carried cells, lists without carrying and
    a context without lists agree up to the rounding of the terms; the last step also against
    the oracle."""
    torch = torch_cuda
    m = gen.globule(2000, 9)
    rng = np.random.default_rng(5)
    carry = api.Context(skin=1.0, carry=2)
    plain = api.Context(skin=1.0, carry=0)
    fresh = api.Context()
    x = m.coords.copy()
    for step in range(11):
        if step:
            x = x + rng.normal(scale=0.01, size=x.shape)
        a, g, nc, reused = _run(torch, carry, x, m.radii)
        ap, gp, ncp, _ = _run(torch, plain, x, m.radii)
        af, gf, _, _ = _run(torch, fresh, x, m.radii)
        assert reused == (step > 0)
        assert ncp == 0
        assert (nc == 0) if step == 0 else (nc >= 0.6 * m.n), (step, nc)
        for aa, gg in ((a, g), (ap, gp)):
            assert np.all(np.abs(aa - af) <= 1e-5 * np.maximum(af, 1.0))
            assert abs(aa.sum() - af.sum()) <= 1e-8 * af.sum()
            _grad_close(gg, gf)
    ra, _, rg = orc.sasa(x, m.radii)
    assert np.all(np.abs(a - ra) <= 1e-4 * np.maximum(ra, 1.0))
    assert abs(a.sum() - ra.sum()) <= 1e-6 * ra.sum()
    _grad_close(g, rg)
    for c in (carry, plain, fresh):
        c.close()


def test_same_positions_carry_every_cell(api, torch_cuda, orc, gen):
    """Unchanged coordinates: every cell of the previous call certifies (all vertices lie
    strictly inside their other face planes, or on them with the same tie-break), so every
    atom with a cell carries it; areas equal the first call's up to summation order."""
    torch = torch_cuda
    m = gen.globule(1500, 3)
    ctx = api.Context(skin=0.8, carry=2)
    a0, g0, nc0, _ = _run(torch, ctx, m.coords, m.radii)
    a1, g1, nc1, reused = _run(torch, ctx, m.coords, m.radii)
    assert nc0 == 0 and reused
    assert nc1 >= np.count_nonzero(a0 > 0), (nc1, np.count_nonzero(a0 > 0))
    assert np.all(np.abs(a1 - a0) <= 1e-9 * np.maximum(a0, 1.0))
    assert np.all(np.linalg.norm(g1 - g0, axis=1) <= 1e-6 * np.maximum(np.linalg.norm(g0, axis=1), 1e-2))
    ctx.close()


@pytest.mark.parametrize("case", ["lattice", "cospherical"])
def test_degenerate_inputs_carry_consistently(api, torch_cuda, orc, case):
    """Exactly degenerate inputs (every vertex on more than three bisectors) called twice:
    the certification meets exact ties, which the same Simulation of Simplicity decides, and
    the complex stays the oracle's."""
    torch = torch_cuda
    if case == "lattice":
        g = np.stack(np.meshgrid(np.arange(4), np.arange(4), np.arange(3), indexing="ij"), -1).reshape(-1, 3)
        x, r = g * 2.5, np.full(len(g), 1.5)
    else:
        c = np.array([[a, b, d] for a in (-1.5, 1.5) for b in (-1.5, 1.5) for d in (-1.5, 1.5)])
        f = np.array([[3.5, 0, 0], [-3.5, 0, 0], [0, 3.5, 0], [0, -3.5, 0], [0, 0, 3.5], [0, 0, -3.5]])
        x = np.concatenate([[[0.0, 0.0, 0.0]], c, f]) + np.array([4.0, -2.0, 1.5])
        r = np.concatenate([[1.2], np.full(8, 1.5), np.full(6, 1.7)])
    ctx = api.Context(skin=0.5, carry=2)
    xt, rt = torch.as_tensor(x, device="cuda"), torch.as_tensor(r, device="cuda")
    for call in range(2):
        rec = ctx.export_complex(xt, rt).cpu().numpy()
        assert ctx.lists_reused() == (call == 1)
        ctx.status_sync()
        _check_against_oracle(orc, rec, x, r)
    ctx.close()


def test_rebuild_carries_nothing(api, torch_cuda, gen):
    """A step that rebuilds the lists (one atom moved by more than half the skin) builds every
    cell afresh; so does a context with carrying off."""
    torch = torch_cuda
    m = gen.globule(1000, 2)
    ctx = api.Context(skin=1.0, carry=2)
    x = m.coords.copy()
    _run(torch, ctx, x, m.radii)
    x[10] += np.array([0.0, 0.7, 0.0])
    _, _, nc, reused = _run(torch, ctx, x, m.radii)
    assert not reused and nc == 0
    _, _, nc, reused = _run(torch, ctx, x, m.radii)
    assert reused and nc > 0
    ctx.close()


def test_default_policy_carries_beyond_one_wave(api, torch_cuda, gen):
    """carry = 1 (the default): a molecule that fits one wave of the fused cell kernel keeps
    the fused kernel (no carried cells); a larger one carries, with results as a fresh build's."""
    torch = torch_cuda
    rng = np.random.default_rng(9)
    small = gen.globule(2000, 1)
    ctx = api.Context(skin=1.0)
    _run(torch, ctx, small.coords, small.radii)
    _, _, nc, reused = _run(torch, ctx, small.coords + rng.normal(scale=0.01, size=small.coords.shape), small.radii)
    assert reused and nc == 0
    ctx.close()
    big = gen.make("globule", 12000, 3)
    ctx, fresh = api.Context(skin=1.0), api.Context()
    _run(torch, ctx, big.coords, big.radii)
    x = big.coords + rng.normal(scale=0.01, size=big.coords.shape)
    a, g, nc, reused = _run(torch, ctx, x, big.radii)
    af, gf, _, _ = _run(torch, fresh, x, big.radii)
    assert reused and nc >= 0.5 * big.n, nc
    assert np.all(np.abs(a - af) <= 1e-5 * np.maximum(af, 1.0))
    _grad_close(g, gf)
    ctx.close()
    fresh.close()


def _large_ball_in_shell(m=40, zcut=-2.0):
    """A large ball inside a partly open shell of small ones (its cell needs the 128 / 128
    pass), in a field of small balls around it."""
    import math
    rng = np.random.default_rng(3)
    idx = np.arange(m) + 0.5
    z = 1 - 2 * idx / m
    rr = np.sqrt(1 - z * z)
    ang = math.pi * (1 + 5 ** 0.5) * idx
    shell = 5.2 * np.stack([rr * np.cos(ang), rr * np.sin(ang), z], 1) + 1e-5 * rng.normal(size=(m, 3))
    shell = shell[z > zcut]
    return np.concatenate([np.zeros((1, 3)) + 1e-6, shell]), np.concatenate([[3.6], np.full(len(shell), 1.2)])


def test_deferred_cell_through_carried_steps(api, torch_cuda, orc):
    """An atom whose cell needs the large-capacity pass, over list-reusing steps with carrying
    on: it is never carried (the redo list sends it to the cell kernel, which defers it), the
    other cells carry, and the complex stays the oracle's."""
    torch = torch_cuda
    x0, r = _large_ball_in_shell()
    ctx = api.Context(skin=0.6, carry=2)
    rng = np.random.default_rng(11)
    x = x0.copy()
    for step in range(3):
        if step:
            x = x + rng.normal(scale=0.005, size=x.shape)
        rec = ctx.export_complex(torch.as_tensor(x, device="cuda"), torch.as_tensor(r, device="cuda")).cpu().numpy()
        carried = ctx.cells_carried()
        assert ctx.deferred_count() >= 1
        ctx.status_sync()
        _check_against_oracle(orc, rec, x, r)
        if step:
            assert 0 < carried < len(r)
    ctx.close()


def test_volumes_through_carried_cells(api, torch_cuda, gen):
    """The volume kernel reads the carried cells' records: volumes and their gradient over
    carried steps equal those of a context without lists."""
    torch = torch_cuda
    m = gen.globule(2500, 6)
    ctx, fresh = api.Context(skin=1.0, carry=2), api.Context()
    rng = np.random.default_rng(12)
    x = m.coords.copy()
    rt = torch.as_tensor(m.radii, device="cuda")
    for step in range(3):
        if step:
            x = x + rng.normal(scale=0.01, size=x.shape)
        xt = torch.as_tensor(x, device="cuda")
        out = []
        for c in (ctx, fresh):
            a = torch.empty(m.n, dtype=torch.float64, device="cuda")
            v = torch.empty(m.n, dtype=torch.float64, device="cuda")
            vg = torch.empty((m.n, 3), dtype=torch.float64, device="cuda")
            c.compute_volume(xt, rt, a, v, vol_grad_out=vg)
            c.status_sync()
            out.append((a.cpu().numpy(), v.cpu().numpy(), vg.cpu().numpy()))
        if step:
            assert ctx.cells_carried() > 0.5 * m.n
        (a1, v1, g1), (a0, v0, g0) = out
        assert np.all(np.abs(a1 - a0) <= 1e-5 * np.maximum(a0, 1.0))
        assert np.all(np.abs(v1 - v0) <= 1e-5 * np.maximum(v0, 1.0))
        assert abs(v1.sum() - v0.sum()) <= 1e-9 * v0.sum()
        _grad_close(g1, g0)
    ctx.close()
    fresh.close()
