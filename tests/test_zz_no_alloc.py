"""dsasa_compute_noalloc, the entry point for callers that must not have the library
allocate device memory (their memory is budgeted or owned elsewhere): through the C ABI it
must give what dsasa_compute gives, on two calls in a row (the static scratch keeps the
previous call's contents), at sizes that take the one-kernel and the multi-kernel cell-list
build (up to exactly DSASA_NOALLOC_MAX_ATOMS), match the oracle, leave the device's free
memory unchanged, and refuse sizes beyond its fixed capacity.

This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
MAX_ATOMS = 32768   # DSASA_NOALLOC_MAX_ATOMS


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_10462_gb300 import api
    lib = api._lib
    vp = ctypes.c_void_p
    lib.dsasa_compute_noalloc.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int64, vp, vp, vp]
    lib.dsasa_compute_noalloc.restype = ctypes.c_int
    return torch, api, lib


def _noalloc(env, xyz, rad, n):
    torch, _, lib = env
    vp = ctypes.c_void_p
    a = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    g = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    rc = lib.dsasa_compute_noalloc(vp(xyz.data_ptr()), vp(rad.data_ptr()), 1.4, n, vp(a.data_ptr()),
                                   vp(g.data_ptr()), vp(torch.cuda.current_stream().cuda_stream))
    return rc, a, g


def _check(a, g, ra, rg):
    a, g = a.cpu().numpy(), g.cpu().numpy()
    assert np.all(np.abs(a - ra) <= 1e-4 * np.maximum(ra, 1.0))
    assert abs(a.sum() - ra.sum()) <= 1e-6 * ra.sum()
    err = np.linalg.norm(g - rg, axis=1)
    assert np.all(err <= 1e-3 * np.maximum(np.linalg.norm(rg, axis=1), 1e-2))


def test_noalloc_matches_compute_on_two_calls_in_a_row(env, gen):
    torch, api, lib = env
    for mol in (gen.globule(3000, 21), gen.rna(1600, 22), gen.globule(20000, 24), gen.globule(MAX_ATOMS, 23)):
        xyz = torch.as_tensor(mol.coords, dtype=torch.float64, device="cuda")
        rad = torch.as_tensor(mol.radii, dtype=torch.float64, device="cuda")
        n = mol.n
        ref_a = torch.empty(n, dtype=torch.float64, device="cuda")
        ref_g = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        ctx = api.Context()
        ctx.compute(xyz, rad, ref_a, ref_g)
        ctx.status_sync()
        ctx.close()
        ra, rg = ref_a.cpu().numpy(), ref_g.cpu().numpy()
        for _ in range(2):
            rc, a, g = _noalloc(env, xyz, rad, n)
            assert rc == 0, rc
            _check(a, g, ra, rg)


def test_noalloc_against_the_oracle_and_allocates_nothing(env, gen, orc):
    torch, _, _ = env
    m = gen.globule(3000, 21)
    xyz = torch.as_tensor(m.coords, dtype=torch.float64, device="cuda")
    rad = torch.as_tensor(m.radii, dtype=torch.float64, device="cuda")
    a = torch.empty(m.n, dtype=torch.float64, device="cuda")
    g = torch.empty((m.n, 3), dtype=torch.float64, device="cuda")
    assert _noalloc(env, xyz, rad, m.n)[0] == 0         # the first call in this context
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    reserved0 = torch.cuda.memory_reserved()
    vp = ctypes.c_void_p
    rc = env[2].dsasa_compute_noalloc(vp(xyz.data_ptr()), vp(rad.data_ptr()), 1.4, m.n, vp(a.data_ptr()),
                                      vp(g.data_ptr()), vp(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    ra, _, rg = orc.sasa(m.coords, m.radii)
    _check(a, g, ra, rg)


def test_noalloc_refuses_sizes_beyond_its_capacity(env, gen):
    torch, _, lib = env
    m = gen.globule(300, 2)
    xyz = torch.as_tensor(m.coords, dtype=torch.float64, device="cuda")
    rad = torch.as_tensor(m.radii, dtype=torch.float64, device="cuda")
    a = torch.full((m.n,), 5.0, dtype=torch.float64, device="cuda")
    vp = ctypes.c_void_p
    # beyond the fixed capacity: a clear error, nothing enqueued (nothing is read or written)
    rc = lib.dsasa_compute_noalloc(vp(xyz.data_ptr()), vp(rad.data_ptr()), 1.4, MAX_ATOMS + 1, vp(a.data_ptr()),
                                   None, vp(torch.cuda.current_stream().cuda_stream))
    assert rc == 3
    torch.cuda.synchronize()
    assert bool((a == 5.0).all())
