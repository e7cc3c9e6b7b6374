"""dsasa_compute_noalloc, the entry point for callers that must not have the library
allocate device memory (their memory is budgeted or owned elsewhere): through the C ABI it
must give what dsasa_compute gives, on two calls in a row (the static scratch keeps the
previous call's contents), and refuse sizes beyond its fixed capacity.

This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_compute_on_two_calls_in_a_row(gen):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_10462_gb300 import api
    lib = api._lib
    vp = ctypes.c_void_p
    lib.dsasa_compute_noalloc.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int64, vp, vp, vp]
    lib.dsasa_compute_noalloc.restype = ctypes.c_int
    stream = torch.cuda.current_stream()
    for mol in (gen.globule(3000, 21), gen.rna(1600, 22)):
        xyz = torch.as_tensor(mol.coords, dtype=torch.float64, device="cuda")
        rad = torch.as_tensor(mol.radii, dtype=torch.float64, device="cuda")
        n = mol.n
        ref_a = torch.empty(n, dtype=torch.float64, device="cuda")
        ref_g = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        ctx = api.Context()
        ctx.compute(xyz, rad, ref_a, ref_g)
        ctx.status_sync()
        ctx.close()
        a = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        g = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.dsasa_compute_noalloc(vp(xyz.data_ptr()), vp(rad.data_ptr()), 1.4, n, vp(a.data_ptr()),
                                       vp(g.data_ptr()), vp(stream.cuda_stream))
        assert rc == 0, rc
        a, g = a.cpu().numpy(), g.cpu().numpy()
        ra, rg = ref_a.cpu().numpy(), ref_g.cpu().numpy()
        assert np.all(np.abs(a - ra) <= 1e-4 * np.maximum(ra, 1.0))
        assert abs(a.sum() - ra.sum()) <= 1e-6 * ra.sum()
        err = np.linalg.norm(g - rg, axis=1)
        assert np.all(err <= 1e-3 * np.maximum(np.linalg.norm(rg, axis=1), 1e-2))
    # beyond the fixed capacity: a clear error, nothing enqueued
    big = 32768 + 1
    rc = lib.dsasa_compute_noalloc(vp(xyz.data_ptr()), vp(rad.data_ptr()), 1.4, big, vp(a.ctypes.data),
                                   None, vp(stream.cuda_stream))
    assert rc == 3
