"""GPU parity of the CUDA path (through the C ABI) against the oracle.

Tolerances (per atom, total, gradient) are the ones the workload statement fixes:
|dA_i| <= 1e-4 max(A_i, 1 A^2), total within 1e-6 relative, ||dg_j|| <= 1e-3 max(||g_j||, 1e-2);
the dual complex C (the simplices that exist) must match exactly."""
import math

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


@pytest.fixture(scope="module")
def api(torch_cuda):
    from paper_2401_10462_gb300 import api
    return api


def _dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def gpu_sasa(api, torch, coords, radii, precision="mixed", weights=None, grad=True):
    ctx = api.Context(precision=precision)
    n = len(radii)
    a = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.empty((n, 3), dtype=torch.float64, device="cuda") if grad else None
    w = None if weights is None else _dev(torch, weights)
    ctx.compute(_dev(torch, coords), _dev(torch, radii), a, g, w)
    ctx.status_sync()
    out = a.cpu().numpy(), (g.cpu().numpy() if grad else None)
    ctx.close()
    return out


def check_areas(a, ref):
    err = np.abs(a - ref)
    assert np.all(np.isfinite(a))
    bad = err > 1e-4 * np.maximum(ref, 1.0)
    assert not bad.any(), (np.nonzero(bad)[0][:10], a[bad][:5], ref[bad][:5])
    assert abs(a.sum() - ref.sum()) <= 1e-6 * ref.sum()


def check_grad(g, ref):
    assert np.all(np.isfinite(g))
    err = np.linalg.norm(g - ref, axis=1)
    lim = 1e-3 * np.maximum(np.linalg.norm(ref, axis=1), 1e-2)
    bad = err > lim
    assert not bad.any(), (np.nonzero(bad)[0][:10], g[bad][:3], ref[bad][:3])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_isolated_two_and_three_spheres(api, torch_cuda, orc, precision):
    cases = [
        (np.array([[1.0, 2.0, 3.0]]), np.array([1.7])),
        (np.array([[0.0, 0.0, 0.0], [2.4, 1.1, -0.3]]), np.array([1.5, 1.7])),
        (np.array([[0.0, 0.0, 0.0], [3.1, 0.4, -0.2], [1.0, 2.7, 0.9]]), np.array([1.7, 1.5, 1.6])),
        (np.array([[0.0, 0.0, 0.0], [0.2, 0.1, 0.0]]), np.array([1.8, 1.2])),   # nested ball
    ]
    for xyz, r in cases:
        a, g = gpu_sasa(api, torch_cuda, xyz, r, precision)
        ra, _, rg = orc.sasa(xyz, r)
        check_areas(a, ra)
        check_grad(g, rg)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("seed", list(range(10)))
def test_globule_304(api, torch_cuda, orc, gen, precision, seed):
    m = gen.globule(304, seed)
    a, g = gpu_sasa(api, torch_cuda, m.coords, m.radii, precision)
    ra, _, rg = orc.sasa(m.coords, m.radii)
    check_areas(a, ra)
    check_grad(g, rg)


def _complex_sets(rec):
    out = {d: set() for d in range(4)}
    owners = {}
    for r in rec:
        simp = tuple(int(x) for x in r[1:] if x >= 0)
        out[len(simp) - 1].add(simp)
        owners.setdefault(simp, set()).add(int(r[0]))
    return out, owners


def _large_ball_in_shell(m=40, zcut=-2.0):
    """A large ball inside a partly open shell of small ones: its cell has more vertices than
    the fast pass holds, so it goes through the large-capacity (128 / 128) pass."""
    rng = np.random.default_rng(3)
    idx = np.arange(m) + 0.5
    z = 1 - 2 * idx / m
    rr = np.sqrt(1 - z * z)
    ang = math.pi * (1 + 5 ** 0.5) * idx
    shell = 5.2 * np.stack([rr * np.cos(ang), rr * np.sin(ang), z], 1) + 1e-5 * rng.normal(size=(m, 3))
    shell = shell[z > zcut]
    xyz = np.concatenate([np.zeros((1, 3)) + 1e-6, shell])
    r = np.concatenate([[3.6], np.full(len(shell), 1.2)])
    return xyz, r


def _check_complex(api, torch, orc, coords, radii, precision):
    ctx = api.Context(precision=precision)
    rec = ctx.export_complex(_dev(torch, coords), _dev(torch, radii)).cpu().numpy()
    ctx.status_sync()
    ctx.close()
    got, owners = _complex_sets(rec)
    o = orc.Oracle(coords, radii)
    for d in range(4):
        ref = {tuple(int(v) for v in np.atleast_1d(s)) for s in o.simplices(d)}
        assert got[d] == ref, (d, len(got[d]), len(ref), list(got[d] ^ ref)[:5])
    # every atom of a simplex sees it in its own cell (consistency of the local cells)
    for simp, who in owners.items():
        assert who == set(simp), (simp, who)


COMPLEX_CASES = ["globule304-0", "globule304-5", "globule5000-0", "globule5000-1", "globule5000-2",
                 "globule7000-12", "rna1000-1", "shell3000-2", "large-ball"]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("case", COMPLEX_CASES)
def test_dual_complex_bit_exact(api, torch_cuda, orc, gen, case, precision):
    """The simplices of C that the GPU cells find are exactly the oracle's, on the 304- and
    5,000-atom globules, a 7,000-atom globule (more atoms than one wave of the cell kernel:
    separate cell and classification kernels), an RNA, a shell, and a cell that needs the
    large-capacity pass."""
    kind, _, seed = case.partition("-")
    if kind == "large":
        xyz, r = _large_ball_in_shell()
    elif kind.startswith("globule"):
        m = gen.globule(int(kind[7:]), int(seed))
        xyz, r = m.coords, m.radii
    elif kind.startswith("rna"):
        m = gen.rna(int(kind[3:]), int(seed))
        xyz, r = m.coords, m.radii
    else:
        m = gen.shell(int(kind[5:]), int(seed), r_out=45.0, thickness=14.0, chain=100)
        xyz, r = m.coords, m.radii
    _check_complex(api, torch_cuda, orc, xyz, r, precision)


def _degenerate(case):
    if case == "lattice":
        # 4 x 4 x 3 cubic lattice of equal balls: every cell vertex is met by several
        # bisectors (co-spherical and co-planar atoms everywhere)
        g = np.stack(np.meshgrid(np.arange(4), np.arange(4), np.arange(3), indexing="ij"), -1).reshape(-1, 3)
        return g * 2.5, np.full(len(g), 1.5)
    # eight equal balls on the corners of a cube (co-spherical) around a smaller central ball,
    # and the six face centres one layer out
    c = np.array([[x, y, z] for x in (-1.5, 1.5) for y in (-1.5, 1.5) for z in (-1.5, 1.5)])
    f = np.array([[3.5, 0, 0], [-3.5, 0, 0], [0, 3.5, 0], [0, -3.5, 0], [0, 0, 3.5], [0, 0, -3.5]])
    xyz = np.concatenate([[[0.0, 0.0, 0.0]], c, f]) + np.array([4.0, -2.0, 1.5])
    return xyz, np.concatenate([[1.2], np.full(8, 1.5), np.full(6, 1.7)])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("case", ["lattice", "cospherical"])
def test_degenerate_inputs_resolved_as_the_oracle(api, torch_cuda, orc, case, precision):
    """Exactly degenerate inputs (no jitter): the device breaks the ties of its clip test by
    the same Simulation of Simplicity as the oracle's triangulation, so the complex is the
    oracle's, the status is OK and the areas and gradient match."""
    xyz, r = _degenerate(case)
    _check_complex(api, torch_cuda, orc, xyz, r, precision)
    a, g = gpu_sasa(api, torch_cuda, xyz, r, precision)     # raises on a non-OK status
    ra, _, rg = orc.sasa(xyz, r)
    check_areas(a, ra)
    check_grad(g, rg)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sliver_atoms(api, torch_cuda, orc, gen, seed, precision):
    """A globule with one atom whose exposed area is about 1e-5 A^2 (its terms cancel about a
    million-fold), against the oracle.  The FP64 form meets the stated tolerances on every
    atom.  The mixed form meets them on every area and on every gradient above the noise
    floor of its float inputs (|g| >= 0.02); below it, within 3e-5 absolute (the limit the
    header states)."""
    import slivers
    torch = torch_cuda
    xyz, r, i = slivers.sliver(gen.globule(304, seed), orc, seed=seed)
    a, g = gpu_sasa(api, torch, xyz, r, precision)
    ra, _, rg = orc.sasa(xyz, r)
    assert 0 < ra[i] < 1e-4
    check_areas(a, ra)
    if precision == "fp64":
        check_grad(g, rg)
        return
    gn = np.linalg.norm(rg, axis=1)
    err = np.linalg.norm(g - rg, axis=1)
    big = gn >= 0.02
    assert np.all(err[big] <= 1e-3 * gn[big]), np.nonzero(big & (err > 1e-3 * gn))[0]
    assert np.all(err[~big] <= 3e-5), (np.nonzero(~big & (err > 3e-5))[0], err[~big].max())


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_globule_5000(api, torch_cuda, orc, gen, precision):
    m = gen.globule(5000, 0)
    a, g = gpu_sasa(api, torch_cuda, m.coords, m.radii, precision)
    ra, _, rg = orc.sasa(m.coords, m.radii)
    check_areas(a, ra)
    check_grad(g, rg)


def test_weights_vjp(api, torch_cuda, orc, gen):
    m = gen.globule(304, 7)
    w = np.random.default_rng(0).uniform(-1, 2, m.n)
    a, g = gpu_sasa(api, torch_cuda, m.coords, m.radii, "mixed", weights=w)
    ra, _, rg = orc.sasa(m.coords, m.radii, weights=w)
    check_areas(a, ra)
    check_grad(g, rg)


def test_rna_and_shell(api, torch_cuda, orc, gen):
    for m in (gen.rna(1000, 1), gen.shell(3000, 2, r_out=45.0, thickness=14.0, chain=100)):
        a, g = gpu_sasa(api, torch_cuda, m.coords, m.radii, "mixed")
        ra, _, rg = orc.sasa(m.coords, m.radii)
        check_areas(a, ra)
        check_grad(g, rg)


def test_edge_cases(api, torch_cuda):
    torch = torch_cuda
    ctx = api.Context()
    # n = 0: nothing enqueued, OK
    z = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    ctx.compute(z, torch.empty(0, dtype=torch.float64, device="cuda"), torch.empty(0, dtype=torch.float64, device="cuda"))
    ctx.status_sync()
    # non-finite input is reported, not computed
    xyz = _dev(torch, np.array([[0.0, 0.0, 0.0], [np.nan, 1.0, 2.0]]))
    a = torch.empty(2, dtype=torch.float64, device="cuda")
    ctx.compute(xyz, _dev(torch, np.array([1.5, 1.5])), a)
    assert ctx.status_code() == 8
    # argument errors return synchronously
    assert api._lib.dsasa_compute(ctx._h, None, None, 1.4, 5, None, None) == 1
    assert api._lib.dsasa_compute(ctx._h, None, None, 1.4, -1, None, None) == 1
    assert api._lib.dsasa_compute(ctx._h, None, None, float("nan"), 0, None, None) == 1
    ctx.close()


def test_host_entry_point_matches_device(api, torch_cuda, gen):
    m = gen.globule(500, 3)
    ctx = api.Context()
    a_h, g_h = ctx.compute_host(m.coords, m.radii)
    a_d, g_d = gpu_sasa(api, torch_cuda, m.coords, m.radii)
    assert np.array_equal(a_h, a_d) and np.array_equal(g_h, g_d)


@pytest.mark.parametrize("case", ["pinned", "pinned-weights", "pinned-skin", "pinned-in-pageable-out"])
def test_host_entry_point_in_place_on_pinned_buffers(api, torch_cuda, gen, case):
    """Pinned host buffers are read and written in place by the kernels (no staging copy);
    the results equal the device entry point's bit for bit, also with weights, with Verlet
    lists (the list check reads the host coordinates) and with pageable outputs (copy path)."""
    torch = torch_cuda
    m = gen.globule(2000, 5)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    hx, hr = pin(m.coords), pin(m.radii)
    w = pin(np.linspace(0.5, 1.5, m.n)) if case == "pinned-weights" else None
    if case == "pinned-in-pageable-out":
        ha, hg = np.empty(m.n), np.empty((m.n, 3))
    else:
        ha, hg = pin(np.zeros(m.n)), pin(np.zeros((m.n, 3)))
    ctx = api.Context(skin=1.0 if case == "pinned-skin" else 0.0)
    ref = api.Context()
    steps = [m.coords, m.coords + np.random.default_rng(2).normal(scale=0.01, size=m.coords.shape)]
    for xs in steps if case == "pinned-skin" else steps[:1]:
        hx[:] = xs
        ctx.compute_host(hx, hr, weights=w, out=(ha, hg))
        a = torch.empty(m.n, dtype=torch.float64, device="cuda")
        g = torch.empty((m.n, 3), dtype=torch.float64, device="cuda")
        ref.compute(_dev(torch, xs), _dev(torch, m.radii), a, g, weights=None if w is None else _dev(torch, w))
        ref.status_sync()
        assert np.array_equal(ha, a.cpu().numpy()) and np.array_equal(hg, g.cpu().numpy())
    if case == "pinned-skin":
        assert ctx.lists_reused()
    ctx.close()
    ref.close()


def test_batch_equals_separate(api, torch_cuda, gen):
    torch = torch_cuda
    mols = [gen.globule(300, 1), gen.rna(640, 2), gen.globule(1000, 3)]
    xyz = np.concatenate([m.coords for m in mols])
    r = np.concatenate([m.radii for m in mols])
    off = np.cumsum([0] + [m.n for m in mols])
    ctx = api.Context()
    a = torch.empty(len(r), dtype=torch.float64, device="cuda")
    g = torch.empty((len(r), 3), dtype=torch.float64, device="cuda")
    ctx.compute_batch(off, _dev(torch, xyz), _dev(torch, r), a, g)
    ctx.status_sync()
    for k, m in enumerate(mols):
        a1, g1 = gpu_sasa(api, torch, m.coords, m.radii)
        assert np.array_equal(a.cpu().numpy()[off[k]:off[k + 1]], a1)
        assert np.array_equal(g.cpu().numpy()[off[k]:off[k + 1]], g1)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_one_wave_and_split_kernels_agree(api, torch_cuda, orc, gen, precision):
    """A molecule alone (few atoms: the cell and classification steps run as one kernel) and
    the same molecule inside a batch of more atoms than one wave of the cell kernel holds
    (separate cell and classification kernels) give bit-identical results."""
    torch = torch_cuda
    small, big = gen.globule(304, 11), gen.globule(7000, 12)
    xyz = np.concatenate([small.coords, big.coords])
    r = np.concatenate([small.radii, big.radii])
    off = np.array([0, small.n, small.n + big.n])
    ctx = api.Context(precision=precision)
    a = torch.empty(len(r), dtype=torch.float64, device="cuda")
    g = torch.empty((len(r), 3), dtype=torch.float64, device="cuda")
    k0 = api.kernel_launches()
    ctx.compute_batch(off, _dev(torch, xyz), _dev(torch, r), a, g)
    ctx.status_sync()
    # multi-molecule cell-list build (9), cell, classification, terms, large-capacity pass
    assert api.kernel_launches() - k0 == 9 + 4
    a1, g1 = gpu_sasa(api, torch, small.coords, small.radii, precision)
    assert np.array_equal(a.cpu().numpy()[:small.n], a1)
    assert np.array_equal(g.cpu().numpy()[:small.n], g1)
    ra, _, rg = orc.sasa(small.coords, small.radii)
    check_areas(a1, ra)
    check_grad(g1, rg)


def test_single_molecule_build_sizes(api, torch_cuda, gen):
    """The single-molecule cell-list build runs ceil(n / 1024) blocks whose last block finishes
    the sort (and resets its ticket); sizes at the block and kernel-choice boundaries, computed
    one after another on one context, equal the multi-molecule build's results (a batch with a
    2-atom molecule far away takes the multi-kernel build)."""
    torch = torch_cuda
    ctx = api.Context()
    for n in (1, 1023, 1024, 1025, 4097, 16384, 16385, 3000):
        m = gen.globule(n, 20 + n % 7)
        x, r = _dev(torch, m.coords), _dev(torch, m.radii)
        a = torch.empty(n, dtype=torch.float64, device="cuda")
        g = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        ctx.compute(x, r, a, g)
        ctx.status_sync()
        far = np.array([[1e4, 0.0, 0.0], [1e4 + 3.0, 0.0, 0.0]])
        xb = np.concatenate([m.coords, far])
        rb = np.concatenate([m.radii, [1.5, 1.5]])
        ab = torch.empty(n + 2, dtype=torch.float64, device="cuda")
        gb = torch.empty((n + 2, 3), dtype=torch.float64, device="cuda")
        ctx.compute_batch(np.array([0, n, n + 2]), _dev(torch, xb), _dev(torch, rb), ab, gb)
        ctx.status_sync()
        assert np.array_equal(a.cpu().numpy(), ab.cpu().numpy()[:n]), n
        assert np.array_equal(g.cpu().numpy(), gb.cpu().numpy()[:n]), n
    ctx.close()


def test_kernel_launch_count(api, torch_cuda, gen):
    """The library's launch counter: one small molecule takes the one-block cell-list build,
    the fused cell + classification kernel, the terms kernel and the (empty) large pass."""
    torch = torch_cuda
    m = gen.globule(304, 2)
    ctx = api.Context()
    x, r = _dev(torch, m.coords), _dev(torch, m.radii)
    a = torch.empty(m.n, dtype=torch.float64, device="cuda")
    g = torch.empty((m.n, 3), dtype=torch.float64, device="cuda")
    ctx.compute(x, r, a, g)
    ctx.status_sync()
    k0 = api.kernel_launches()
    for _ in range(3):
        ctx.compute(x, r, a, g)
    ctx.status_sync()
    assert api.kernel_launches() - k0 == 3 * 4
    ctx.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_deterministic(api, torch_cuda, gen, precision):
    m = gen.globule(2000, 4)
    r1 = gpu_sasa(api, torch_cuda, m.coords, m.radii, precision)
    r2 = gpu_sasa(api, torch_cuda, m.coords, m.radii, precision)
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("m,zcut", [(40, -2.0), (56, -0.5)])
def test_large_cells_take_the_deferred_pass(api, torch_cuda, orc, precision, m, zcut):
    """A cell with more vertices than the fast pass holds (a large ball inside a shell of
    small ones: ~2 x 40 - 4 cell vertices > 64 slots) is deferred to the large-capacity
    pass; the partly open shell leaves the centre exposed."""
    rng = np.random.default_rng(3)
    idx = np.arange(m) + 0.5
    z = 1 - 2 * idx / m
    rr = np.sqrt(1 - z * z)
    ang = math.pi * (1 + 5 ** 0.5) * idx
    shell = 5.2 * np.stack([rr * np.cos(ang), rr * np.sin(ang), z], 1) + 1e-5 * rng.normal(size=(m, 3))
    shell = shell[z > zcut]
    xyz = np.concatenate([np.zeros((1, 3)) + 1e-6, shell])
    r = np.concatenate([[3.6], np.full(len(shell), 1.2)])
    torch = torch_cuda
    ctx = api.Context(precision=precision)
    a = torch.empty(len(r), dtype=torch.float64, device="cuda")
    g = torch.empty((len(r), 3), dtype=torch.float64, device="cuda")
    ctx.compute(_dev(torch, xyz), _dev(torch, r), a, g)
    assert ctx.deferred_count() >= 1   # the large ball went through the large-capacity pass
    ctx.status_sync()
    ctx.close()
    ra, _, rg = orc.sasa(xyz, r)
    check_areas(a.cpu().numpy(), ra)
    check_grad(g.cpu().numpy(), rg)


def test_capsid_million_sampled_parity(api, torch_cuda, orc, gen):
    """The 1,000,000-atom capsid-like shell at full size, in the launch configuration the
    capsid benchmark times: sampled atoms against the oracle on local patches (an atom's
    area and gradient entry depend only on balls overlapping its own), and properties that
    hold at any size on every atom."""
    torch = torch_cuda
    m = gen.make("shell", 1_000_000, 0)
    a, g = gpu_sasa(api, torch, m.coords, m.radii, "mixed")
    R = m.radii + P
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(g))
    # FP32 terms may leave a buried atom a few 1e-6 A^2 below zero: within the per-atom
    # tolerance 1e-4 max(A, 1), so the bound is that tolerance
    assert a.min() >= -1e-4, a.min()
    assert np.all(a <= 4 * math.pi * R ** 2 * (1 + 1e-6))
    assert np.abs(g.sum(0)).max() <= 1e-6 * np.abs(g).sum()          # translation invariance
    rng = np.random.default_rng(0)
    for i in rng.choice(m.n, 24, replace=False):
        idx = orc.local_patch(m.coords, m.radii, [i])
        k = int(np.nonzero(idx == i)[0][0])
        ra, _, rg = orc.sasa(m.coords[idx], m.radii[idx])
        assert abs(a[i] - ra[k]) <= 1e-4 * max(ra[k], 1.0), (i, a[i], ra[k])
        assert np.linalg.norm(g[i] - rg[k]) <= 1e-3 * max(np.linalg.norm(rg[k]), 1e-2), (i, g[i], rg[k])
