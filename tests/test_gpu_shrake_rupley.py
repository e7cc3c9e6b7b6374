"""GPU Shrake-Rupley numerical SASA against the oracle's decisions by the definition
(exposed: strictly outside every other ball, decided on the real numbers), and agreement
with the exact areas within the sampling error.

The kernel decides each point in float32 (its arithmetic is stated in include/dsasa.h); a
float32 decision can differ from the real one only where the margin |x - p_j|^2 - R_j^2 is
within the float32 error bound of that arithmetic.  Those points are counted ("uncertain")
and must stay rare; every other point must be decided as the definition decides it."""
import numpy as np
import pytest

from oracle import shrake_rupley as sr

pytestmark = pytest.mark.gpu
U = 2.0 ** -24   # float32 unit roundoff
P = 1.4


def f32_classes(coords, radii, pts, i):
    """(certainly exposed, uncertain) point counts of atom i under the float32 error bound:
    x_c = fl(fl(R_i) s_c), q_c = fl(p_j - p_i) and d_c = fl(x_c - q_c) each err by at most
    3.1 u (R_i |s_c| + |q_c|) (e_c); the rounded sum of squares and fl(R_j)^2 add 3.1 u of
    their sizes; the bound is doubled for safety."""
    nb, D, margin = sr.point_margins(coords, radii, pts, i)
    if len(nb) == 0:
        return len(pts), 0
    R = np.asarray(radii) + P
    s = np.abs(pts.astype(np.float64))
    Q = np.abs(coords[nb] - coords[i])
    e = 3.1 * U * (R[i] * s[:, None, :] + Q[None, :, :])
    B = 2.0 * (3.1 * U * (D * D).sum(-1) + (e * (2.0 * np.abs(D) + e)).sum(-1) + 3.1 * U * R[nb][None, :] ** 2)
    cert_cov = (margin < -B).any(1)
    cert_exp = (margin > B).all(1)
    return int(cert_exp.sum()), int((~cert_cov & ~cert_exp).sum())


def check_counts(coords, radii, pts, c):
    exact = sr.exposed_counts(coords, radii, pts)
    unc_total = 0
    for i in range(len(radii)):
        lo, unc = f32_classes(coords, radii, pts, i)
        assert lo <= c[i] <= lo + unc, (i, c[i], lo, unc, exact[i])
        assert lo <= exact[i] <= lo + unc
        unc_total += unc
    # the uncertain points are rare (the bound is a few 1e-6 A^2 of margin)
    assert unc_total <= 1e-4 * len(radii) * len(pts), unc_total
    # and the counts differ from the definition's by no more than those points
    assert np.abs(c - exact).sum() <= unc_total
    return exact, unc_total


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
def test_counts_match_the_definition(torch_cuda, gen, seed):
    m = gen.globule(304, seed)
    pts = sr.sphere_points(960)
    a, c, tests = gpu_sr(torch_cuda, m.coords, m.radii, 960)
    check_counts(m.coords, m.radii, pts, c)
    R = m.radii + 1.4
    assert np.allclose(a, 4 * np.pi * R * R * c / 960, rtol=1e-15)
    assert tests > 0


def test_rna_and_edge_cases(torch_cuda, gen):
    m = gen.rna(640, 3)
    _, c, _ = gpu_sr(torch_cuda, m.coords, m.radii, 500)
    check_counts(m.coords, m.radii, sr.sphere_points(500), c)
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
