"""Error paths of the library, made on the host or with bounded inputs (no GPU fault is made
or expected): a fixed capacity exceeded, a cell with more overlapping neighbours than the
large-capacity pass holds, a Verlet list longer than its capacity, an allocation failure
(injected on the host), and an exact expansion longer than its capacity (a host build of the
device arithmetic with a tiny capacity)."""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
P = 1.4


# ------------------------------------------------------------------ host: expansion capacity
@pytest.fixture(scope="module")
def mc_pair():
    """The device arithmetic built for the host twice: with the shipped expansion capacity
    and with a capacity of 4 components."""
    src = os.path.join(HERE, "mathcheck.cpp")
    hdr = os.path.join(ROOT, "paper_2401_10462_gb300", "csrc", "dsasa_math.cuh")
    out = []
    for tag, flags in (("", []), ("_xp4", ["-DDS_XP_N=4"])):
        so = os.path.join(ROOT, "paper_2401_10462_gb300", "_build", f"libmathcheck{tag}.so")
        os.makedirs(os.path.dirname(so), exist_ok=True)
        if not os.path.exists(so) or os.path.getmtime(so) < max(os.path.getmtime(src), os.path.getmtime(hdr)):
            tmp = so + f".tmp{os.getpid()}"
            subprocess.check_call(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", *flags,
                                   "-o", tmp, src])
            os.replace(tmp, so)
        lib = ctypes.CDLL(so)
        lib.mc_pred.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        lib.mc_xp_len.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        out.append(lib)
    return out


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def test_expansion_overflow_is_flagged_not_guessed(mc_pair):
    """An exact predicate whose expansion outgrows its capacity reports the overflow (the
    kernels turn it into DSASA_ERR_UNRESOLVED and a NaN output); it never returns a sign
    that differs from the exact one."""
    full, tiny = mc_pair
    rng = np.random.default_rng(5)
    flagged = 0
    for _ in range(200):
        pts = np.zeros((5, 4))
        pts[:, :3] = rng.normal(scale=2.0, size=(5, 3)) + np.array([31.7, -8.2, 4.9])
        pts[:, 3] = rng.choice([1.2, 1.52, 1.55, 1.7, 1.8], size=5) + P
        exact = full.mc_pred(0, 2, _d(pts))
        assert exact != 2
        got = tiny.mc_pred(0, 2, _d(pts))
        if got == 2:
            flagged += 1
        else:
            assert got == exact
    assert flagged > 0


# ------------------------------------------------------------------ GPU (bounded inputs)
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


def _spiral(k, radius, seed):
    idx = np.arange(k) + 0.5
    z = 1 - 2 * idx / k
    r = np.sqrt(1 - z * z)
    ang = math.pi * (1 + 5 ** 0.5) * idx
    jit = 1e-4 * np.random.default_rng(seed).normal(size=(k, 3))
    return radius * np.stack([r * np.cos(ang), r * np.sin(ang), z], 1) + jit


def _dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.gpu
def test_fixed_capacity_rejects_more_atoms(api, torch_cuda, gen):
    torch = torch_cuda
    m = gen.globule(500, 1)
    ctx = api.Context(max_atoms=m.n - 1)
    a = torch.full((m.n,), 7.0, dtype=torch.float64, device="cuda")
    k0 = api.kernel_launches()
    with pytest.raises(api.DSASAError) as ei:
        ctx.compute(_dev(torch, m.coords), _dev(torch, m.radii), a)
    assert ei.value.code == 3
    assert api.kernel_launches() == k0                     # nothing was enqueued
    assert bool((a == 7.0).all())
    ctx.status_sync()                                      # and no device error is pending
    ctx.close()


@pytest.mark.gpu
def test_too_many_neighbours_gives_capacity_and_one_nan(api, torch_cuda, orc):
    """A large ball inside a shell of 150 overlapping small balls: its cell needs more planes
    than the large-capacity pass holds (122).  The status is DSASA_ERR_CAPACITY, that atom's
    outputs are NaN, and every other atom's outputs are the oracle's."""
    torch = torch_cuda
    xyz = np.concatenate([np.full((1, 3), 1e-5), _spiral(150, 8.0, 1)])
    r = np.concatenate([[6.0], np.full(150, 1.2)])
    ctx = api.Context()
    a = torch.empty(len(r), dtype=torch.float64, device="cuda")
    g = torch.empty((len(r), 3), dtype=torch.float64, device="cuda")
    ctx.compute(_dev(torch, xyz), _dev(torch, r), a, g)
    assert ctx.status_code() == 3
    ctx.close()
    a, g = a.cpu().numpy(), g.cpu().numpy()
    assert np.isnan(a[0]) and np.all(np.isnan(g[0]))
    assert np.all(np.isfinite(a[1:])) and np.all(np.isfinite(g[1:]))
    ra, _, rg = orc.sasa(xyz, r)
    assert np.all(np.abs(a[1:] - ra[1:]) <= 1e-4 * np.maximum(ra[1:], 1.0))
    err = np.linalg.norm(g[1:] - rg[1:], axis=1)
    assert np.all(err <= 1e-3 * np.maximum(np.linalg.norm(rg[1:], axis=1), 1e-2))


@pytest.mark.gpu
def test_verlet_list_overflow_forces_rebuild(api, torch_cuda, orc):
    """A ball with 55 overlapping neighbours and 70 more in the skin band (125 > 122 list
    entries): its list cannot be kept, so every call rebuilds the cell list; the results are
    still exact (the plane table holds only the 55 overlapping balls) and no error is
    reported."""
    torch = torch_cuda
    xyz = np.concatenate([np.full((1, 3), 1e-5), _spiral(55, 8.0, 2), _spiral(70, 10.5, 3)])
    r = np.concatenate([[6.0], np.full(125, 1.2)])
    x, rr = _dev(torch, xyz), _dev(torch, r)
    ctx = api.Context(skin=1.0)
    a = torch.empty(len(r), dtype=torch.float64, device="cuda")
    g = torch.empty((len(r), 3), dtype=torch.float64, device="cuda")
    for _ in range(3):
        ctx.compute(x, rr, a, g)
        ctx.status_sync()
        assert not ctx.lists_reused()
    ctx.close()
    ra, _, rg = orc.sasa(xyz, r)
    a, g = a.cpu().numpy(), g.cpu().numpy()
    assert np.all(np.abs(a - ra) <= 1e-4 * np.maximum(ra, 1.0))
    err = np.linalg.norm(g - rg, axis=1)
    assert np.all(err <= 1e-3 * np.maximum(np.linalg.norm(rg, axis=1), 1e-2))


@pytest.mark.gpu
def test_allocation_failure_is_oom_and_the_context_survives(api, torch_cuda, gen):
    torch = torch_cuda
    lib = api._lib
    # creating a context needs device memory
    lib.dsasa_debug_fail_allocations(1)
    h = ctypes.c_void_p()
    assert lib.dsasa_create(ctypes.byref(h), 0, None, None) == 2 and not h.value
    lib.dsasa_debug_fail_allocations(0)
    # a compute call that has to grow the scratch
    m = gen.globule(600, 2)
    x, r = _dev(torch, m.coords), _dev(torch, m.radii)
    ctx = api.Context()
    a = torch.empty(m.n, dtype=torch.float64, device="cuda")
    lib.dsasa_debug_fail_allocations(3)
    with pytest.raises(api.DSASAError) as ei:
        ctx.compute(x, r, a)
    assert ei.value.code == 2
    lib.dsasa_debug_fail_allocations(0)
    ctx.status_sync()
    ctx.compute(x, r, a)                                   # the context is still usable
    ctx.status_sync()
    ref = api.Context()
    b = torch.empty(m.n, dtype=torch.float64, device="cuda")
    ref.compute(x, r, b)
    ref.status_sync()
    assert torch.equal(a, b)
    ctx.close()
    ref.close()
