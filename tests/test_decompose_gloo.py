"""Spatial domain decomposition of one molecule over ranks (slabs, halo 2 R_max), with gloo
ranks on the CPU: each rank owns one slab's atoms, the boundary layers are exchanged once,
and every rank's outputs for its own atoms equal the whole-molecule oracle's.  The oracle
stands in for the GPU compute step here (no GPU in these ranks)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _molecule():
    from paper_2401_10462_gb300 import inputs
    return inputs.globule(1500, 3)


def _oracle_compute(coords, radii):
    from oracle import oracle
    a, _, g = oracle.sasa(coords, radii)
    return a, g


def _rank(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from paper_2401_10462_gb300 import decompose
    m = _molecule()
    slabs = decompose.make_slabs(m.coords, m.radii, ws)
    mine = np.nonzero(slabs.owner(m.coords[:, slabs.axis]) == rank)[0]
    ids, a, g = decompose.distributed_sasa(slabs, mine, m.coords[mine], m.radii[mine], compute=_oracle_compute)
    out[rank] = (ids, a, g, len(mine))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_slabs_reproduce_the_whole_molecule(orc, ws):
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
    m = _molecule()
    ra, _, rg = orc.sasa(m.coords, m.radii)
    seen = np.zeros(m.n, dtype=int)
    for r in range(ws):
        ids, a, g, k = out[r]
        assert len(ids) == k > 0
        seen[ids] += 1
        # identical up to the summation order of the oracle's terms
        assert np.all(np.abs(a - ra[ids]) <= 1e-12 * np.maximum(ra[ids], 1.0))
        gn = np.linalg.norm(rg[ids], axis=1)
        assert np.all(np.linalg.norm(g - rg[ids], axis=1) <= 1e-12 * np.maximum(gn, 1.0))
    assert np.all(seen == 1)      # every atom owned by exactly one rank


def test_partition_and_halo_bookkeeping(gen):
    from paper_2401_10462_gb300 import decompose
    m = gen.globule(3000, 4)
    s = decompose.make_slabs(m.coords, m.radii, 4)
    x = m.coords[:, s.axis]
    own = s.owner(x)
    counts = np.bincount(own, minlength=4)
    assert counts.sum() == m.n and counts.min() >= m.n // 4 - 1      # equal shares
    assert s.halo == pytest.approx(2 * (m.radii.max() + 1.4))
    R = m.radii + 1.4
    for p in range(4):
        ext = s.extended(p, x)
        # every ball overlapping an owned atom's ball is in the extended slab
        for i in np.nonzero(own == p)[0][::25]:
            d = np.linalg.norm(m.coords - m.coords[i], axis=1)
            assert np.all(ext[d < R + R[i]])
        # every atom of the extended slab that another rank owns is in that rank's boundary layer
        for q in range(4):
            if q != p:
                need = ext & (own == q)
                assert np.all(s.boundary_layer(q, x)[need])
