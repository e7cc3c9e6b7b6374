"""The differentiation workload: a 20,000-atom globule, E_np = sum 0.005 A_i through the
autograd Function, 1,000 Gaussian steps (sigma = 0.01 A per coordinate) replayed from one
captured CUDA graph; at steps 0, 100, ..., 1000 the gradient of 64 seeded atoms is checked
against central finite differences (h = 1e-4 A) of the FP64 oracle's total area.  Run twice:
cells built afresh every step, and with a 1 A Verlet skin, where steps that reuse the lists
carry each atom's cell from the previous step (the incremental update of the complex).

The oracle runs on local patches: the outputs that depend on p_j are the areas of the
atoms whose balls overlap B_j, and those depend only on the balls overlapping them, so the
atoms within 4 R_max + 1 A of j reproduce d(sum_i A_i)/dp_j exactly.  An atom whose dual
complex changes between p_j - h and p_j + h (a combinatorial event, where the gradient is
not defined) is reported and left out, and must stay rare."""
import multiprocessing as mp

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
GAMMA = 0.005
H = 1e-4


def _complex(o):
    return tuple(o.simplices(d).tobytes() for d in range(4))


def _fd_one(args):
    """(d sum A / d p_j by central differences, oracle analytic gradient, event flag)."""
    coords, radii, k = args
    from oracle import oracle
    o = oracle.Oracle(coords, radii)
    _, _, g = o.areas(grad=True)
    fd = np.zeros(3)
    event = False
    for c in range(3):
        xp = coords.copy()
        xm = coords.copy()
        xp[k, c] += H
        xm[k, c] -= H
        op, om = oracle.Oracle(xp, radii), oracle.Oracle(xm, radii)
        if _complex(op) != _complex(om):
            event = True
        fd[c] = (op.areas(grad=False)[1] - om.areas(grad=False)[1]) / (2 * H)
    return fd, g[k], event


@pytest.fixture(scope="module")
def pool():
    # spawn: worker processes must not inherit a CUDA context
    p = mp.get_context("spawn").Pool(min(16, mp.cpu_count()))
    yield p
    p.close()
    p.join()


@pytest.mark.parametrize("skin", [0.0, 1.0])
def test_graphed_trajectory_fd(pool, orc, gen, skin):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_10462_gb300 import autograd as ag
    m = gen.make("globule", 20000, 0)
    x0 = torch.as_tensor(m.coords, device="cuda")
    r = torch.as_tensor(m.radii, device="cuda")
    rng = np.random.default_rng(2024)
    # step 0: the eager autograd path at the initial coordinates
    xr = x0.clone().requires_grad_(True)
    e, _ = ag.nonpolar_energy(xr, r)
    e.backward()
    checkpoints = [(0, x0.cpu().numpy(), xr.grad.cpu().numpy())]
    tr = ag.GraphedTrajectory(x0, r, sigma=0.01, seed=11, skin=skin).capture()
    for step in range(100, 1001, 100):
        tr.replay(100)
        torch.cuda.synchronize()
        checkpoints.append((step, tr.x.cpu().numpy(), tr.grad.cpu().numpy()))
    tr.check()
    jobs, meta = [], []
    for step, x, g in checkpoints:
        for j in rng.choice(m.n, 64, replace=False):
            idx = orc.local_patch(x, m.radii, [j])
            k = int(np.nonzero(idx == j)[0][0])
            jobs.append((x[idx].copy(), m.radii[idx].copy(), k))
            meta.append((step, int(j), g[j] / GAMMA))
    res = pool.map(_fd_one, jobs, chunksize=4)
    events, bad = 0, []
    for (step, j, gj), (fd, ga, event) in zip(meta, res):
        # the oracle's own analytic gradient agrees with its finite differences
        if event:
            events += 1
            continue
        tol = 1e-3 * max(np.linalg.norm(fd), 1e-2)
        assert np.linalg.norm(ga - fd) <= tol, (step, j, ga, fd)
        if np.linalg.norm(gj - fd) > tol:
            bad.append((step, j, gj, fd))
    assert not bad, bad[:5]
    assert events <= 0.02 * len(jobs), events
