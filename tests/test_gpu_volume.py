"""GPU parity of the molecular volume (per-atom power-cell volumes, their sum = the union
volume, and d(union volume)/dx) against the oracle, through the C ABI.

Tolerances as for the areas: per atom |dV_i| <= 1e-4 max(V_i, 1 A^3), total 1e-6 relative,
gradient ||dg_j|| <= 1e-3 max(||g_j||, 1e-2)."""
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


def _dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def gpu_volume(torch, coords, radii, precision="mixed"):
    from paper_2401_10462_gb300 import api
    ctx = api.Context(precision=precision)
    n = len(radii)
    a = torch.empty(n, dtype=torch.float64, device="cuda")
    v = torch.empty(n, dtype=torch.float64, device="cuda")
    gv = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    ctx.compute_volume(_dev(torch, coords), _dev(torch, radii), a, v, vol_grad_out=gv)
    ctx.status_sync()
    out = a.cpu().numpy(), v.cpu().numpy(), gv.cpu().numpy()
    ctx.close()
    return out


def check(v, gv, ref_v, ref_g):
    assert np.all(np.isfinite(v)) and np.all(np.isfinite(gv))
    bad = np.abs(v - ref_v) > 1e-4 * np.maximum(ref_v, 1.0)
    assert not bad.any(), (np.nonzero(bad)[0][:10], v[bad][:5], ref_v[bad][:5])
    assert abs(v.sum() - ref_v.sum()) <= 1e-6 * ref_v.sum()
    err = np.linalg.norm(gv - ref_g, axis=1)
    badg = err > 1e-3 * np.maximum(np.linalg.norm(ref_g, axis=1), 1e-2)
    assert not badg.any(), (np.nonzero(badg)[0][:10], gv[badg][:3], ref_g[badg][:3])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_one_and_two_spheres(torch_cuda, orc, precision):
    for xyz, r in ((np.zeros((1, 3)), np.array([1.7])),
                   (np.array([[0.0, 0.0, 0.0], [2.9, 0.3, -0.2]]), np.array([1.2, 1.8])),
                   (np.array([[0.0, 0.0, 0.0], [0.3, 0.0, 0.0]]), np.array([1.9, 1.2]))):
        _, v, gv = gpu_volume(torch_cuda, xyz, r, precision)
        rv, _, rg = orc.Oracle(xyz, r).volumes()
        check(v, gv, rv, rg)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("seed", list(range(10)))
def test_globule_304(torch_cuda, orc, gen, precision, seed):
    m = gen.globule(304, seed)
    a, v, gv = gpu_volume(torch_cuda, m.coords, m.radii, precision)
    rv, _, rg = orc.Oracle(m.coords, m.radii).volumes()
    check(v, gv, rv, rg)
    ra, _, _ = orc.sasa(m.coords, m.radii, grad=False)
    assert np.all(np.abs(a - ra) <= 1e-4 * np.maximum(ra, 1.0))


def test_areas_unchanged_by_the_volume_pass(torch_cuda, gen):
    torch = torch_cuda
    from paper_2401_10462_gb300 import api
    m = gen.globule(2000, 7)
    a_vol, _, _ = gpu_volume(torch, m.coords, m.radii)
    ctx = api.Context()
    a = torch.empty(m.n, dtype=torch.float64, device="cuda")
    ctx.compute(_dev(torch, m.coords), _dev(torch, m.radii), a)
    ctx.status_sync()
    assert np.array_equal(a.cpu().numpy(), a_vol)


def test_globule_5000_rna_shell(torch_cuda, orc, gen):
    for m in (gen.globule(5000, 0), gen.rna(3000, 1), gen.shell(6000, 2, r_out=40.0)):
        _, v, gv = gpu_volume(torch_cuda, m.coords, m.radii)
        rv, _, rg = orc.Oracle(m.coords, m.radii).volumes()
        check(v, gv, rv, rg)
        # translation invariance of the union volume
        assert np.abs(gv.sum(0)).max() <= 1e-6 * np.abs(gv).sum()


def test_large_cell_takes_the_fused_pass(torch_cuda, orc):
    """A ball inside a shell of 56 small ones has more cell vertices than the fast kernels
    hold: its volume comes from the large-capacity fused pass."""
    rng = np.random.default_rng(3)
    m = 56
    idx = np.arange(m) + 0.5
    z = 1 - 2 * idx / m
    rr = np.sqrt(1 - z * z)
    ang = math.pi * (1 + 5 ** 0.5) * idx
    shell = 5.2 * np.stack([rr * np.cos(ang), rr * np.sin(ang), z], 1) + 1e-5 * rng.normal(size=(m, 3))
    shell = shell[z > -0.5]
    xyz = np.concatenate([np.zeros((1, 3)) + 1e-6, shell])
    r = np.concatenate([[3.6], np.full(len(shell), 1.2)])
    _, v, gv = gpu_volume(torch_cuda, xyz, r)
    rv, _, rg = orc.Oracle(xyz, r).volumes()
    check(v, gv, rv, rg)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("case", ["globule304", "globule3000", "rna", "large-ball"])
def test_weighted_volume_gradient(torch_cuda, orc, gen, case, precision):
    """d(sum_i w_i V_i)/dx for random weights (dsasa_compute_volume_vjp) against the oracle,
    including the large-capacity pass (a cell too large for the fast pass)."""
    from paper_2401_10462_gb300 import api
    torch = torch_cuda
    if case == "globule304":
        m = gen.globule(304, 4)
        xyz, r = m.coords, m.radii
    elif case == "globule3000":
        m = gen.globule(3000, 5)
        xyz, r = m.coords, m.radii
    elif case == "rna":
        m = gen.rna(900, 6)
        xyz, r = m.coords, m.radii
    else:
        k = 40
        idx = np.arange(k) + 0.5
        z = 1 - 2 * idx / k
        rr = np.sqrt(1 - z * z)
        ang = math.pi * (1 + 5 ** 0.5) * idx
        shell = 5.2 * np.stack([rr * np.cos(ang), rr * np.sin(ang), z], 1)
        shell = shell[z > -2.0] + 1e-5 * np.random.default_rng(3).normal(size=(int((z > -2.0).sum()), 3))
        xyz = np.concatenate([np.zeros((1, 3)) + 1e-6, shell])
        r = np.concatenate([[3.6], np.full(len(shell), 1.2)])
    n = len(r)
    w = np.random.default_rng(11).uniform(-1.0, 2.0, n)
    ctx = api.Context(precision=precision)
    a = torch.empty(n, dtype=torch.float64, device="cuda")
    v = torch.empty(n, dtype=torch.float64, device="cuda")
    gv = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    ctx.compute_volume_vjp(_dev(torch, xyz), _dev(torch, r), _dev(torch, w), a, v, gv)
    ctx.status_sync()
    ctx.close()
    rv, _, rg = orc.Oracle(xyz, r).volumes(weights=w)
    check(v.cpu().numpy(), gv.cpu().numpy(), rv, rg)


def test_volume_autograd(torch_cuda, orc, gen):
    """molecular_volumes through torch.autograd: the backward of sum_i c_i V_i is the oracle's
    weighted volume gradient."""
    from paper_2401_10462_gb300 import autograd as ag
    torch = torch_cuda
    m = gen.globule(500, 8)
    c = np.random.default_rng(2).uniform(0.0, 1.0, m.n)
    x = torch.as_tensor(m.coords, device="cuda").requires_grad_(True)
    vol = ag.molecular_volumes(x, torch.as_tensor(m.radii, device="cuda"))
    (vol * torch.as_tensor(c, device="cuda")).sum().backward()
    rv, _, rg = orc.Oracle(m.coords, m.radii).volumes(weights=c)
    check(vol.detach().cpu().numpy(), x.grad.cpu().numpy(), rv, rg)
