"""GPU Shrake-Rupley numerical SASA: exposed-point counts bit-exact against the oracle's
float32 evaluation of the same decisions, and agreement with the exact areas within the
sampling error."""
import numpy as np
import pytest

from oracle import shrake_rupley as sr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def gpu_sr(torch, coords, radii, m):
    from paper_2401_10462_gb300 import api
    ctx = api.Context()
    n = len(radii)
    pts = torch.as_tensor(sr.sphere_points(m), device="cuda")
    a = torch.empty(n, dtype=torch.float64, device="cuda")
    c = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.compute_sr(torch.as_tensor(coords, device="cuda"), torch.as_tensor(radii, device="cuda"), pts, a, c)
    ctx.status_sync()
    tests = ctx.sr_tests()
    ctx.close()
    return a.cpu().numpy(), c.cpu().numpy(), tests


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_counts_bit_exact(torch_cuda, gen, seed):
    m = gen.globule(304, seed)
    a, c, tests = gpu_sr(torch_cuda, m.coords, m.radii, 960)
    ref = sr.exposed_counts(m.coords, m.radii, sr.sphere_points(960))
    assert np.array_equal(c, ref)
    R = m.radii + 1.4
    assert np.allclose(a, 4 * np.pi * R * R * ref / 960, rtol=1e-15)
    assert tests > 0


def test_rna_and_edge_cases(torch_cuda, gen):
    m = gen.rna(640, 3)
    _, c, _ = gpu_sr(torch_cuda, m.coords, m.radii, 500)
    assert np.array_equal(c, sr.exposed_counts(m.coords, m.radii, sr.sphere_points(500)))
    _, c1, _ = gpu_sr(torch_cuda, np.zeros((1, 3)), np.array([1.5]), 333)
    assert c1[0] == 333


def test_agrees_with_the_exact_areas(torch_cuda, orc, gen):
    from paper_2401_10462_gb300 import api
    torch = torch_cuda
    m = gen.globule(5000, 0)
    a_sr, _, _ = gpu_sr(torch, m.coords, m.radii, 3840)
    ctx = api.Context()
    a = torch.empty(m.n, dtype=torch.float64, device="cuda")
    ctx.compute(torch.as_tensor(m.coords, device="cuda"), torch.as_tensor(m.radii, device="cuda"), a)
    ctx.status_sync()
    ex = a.cpu().numpy()
    assert abs(a_sr.sum() - ex.sum()) < 1e-3 * ex.sum()
    R = m.radii + 1.4
    assert np.abs(a_sr - ex).max() < 0.05 * (4 * np.pi * R * R).max()
