"""Spatial domain decomposition of one large molecule over ranks (slabs with a halo).

Each rank owns the atoms of one slab along the longest axis of the molecule and computes
their areas and gradient entries.  The area A_i and the gradient entry g_i of an atom depend
only on the atoms whose balls overlap B_i: every simplex of the dual complex that contains i
lies in B_i, where a ball that misses B_i never has the smaller power.  Those atoms lie
within R_i + R_max <= 2 R_max of p_i, so a rank that also holds every atom within 2 R_max
(+ skin, for Verlet lists) of its slab computes its own atoms' outputs exactly, with no
exchange afterwards.  The one exchange is before the compute: every rank sends the atoms of
its boundary layers (within the halo width of a slab face) to the others, which keep those
inside their extended slab.

The slab bounds are fixed from the whole molecule once (equal atom counts per slab); in a
simulation the ranks then keep ownership by position.  The compute step is pluggable: the
default runs the library on the rank's GPU (dsasa_compute through paper_2401_10462_gb300.api);
any function (coords, radii) -> (areas, grad) on host arrays can stand in for it.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

PROBE = 1.4


@dataclass
class Slabs:
    axis: int
    bounds: np.ndarray     # nparts + 1 increasing values; slab p is [bounds[p], bounds[p+1])
    halo: float            # width of the halo (2 R_max + skin)

    @property
    def nparts(self) -> int:
        return len(self.bounds) - 1

    def owner(self, x: np.ndarray) -> np.ndarray:
        """Slab index of each coordinate along the axis (the outermost slabs are open)."""
        return np.clip(np.searchsorted(self.bounds, x, side="right") - 1, 0, self.nparts - 1)

    def extended(self, p: int, x: np.ndarray) -> np.ndarray:
        """Mask of coordinates inside slab p widened by the halo on both sides."""
        lo = -np.inf if p == 0 else self.bounds[p] - self.halo
        hi = np.inf if p == self.nparts - 1 else self.bounds[p + 1] + self.halo
        return (x >= lo) & (x < hi)

    def boundary_layer(self, p: int, x: np.ndarray) -> np.ndarray:
        """Mask of slab p's own atoms within the halo width of one of its inner faces (the
        atoms another slab's extended region can contain)."""
        own = self.owner(x) == p
        m = np.zeros(len(x), dtype=bool)
        if p > 0:
            m |= x < self.bounds[p] + self.halo
        if p < self.nparts - 1:
            m |= x >= self.bounds[p + 1] - self.halo
        return own & m


def make_slabs(coords, radii, nparts: int, probe: float = PROBE, skin: float = 0.0) -> Slabs:
    """Slabs of equal atom counts along the molecule's longest axis, halo 2 R_max + skin."""
    xyz = np.asarray(coords, dtype=np.float64)
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    ext = xyz.max(0) - xyz.min(0)
    axis = int(np.argmax(ext))
    x = np.sort(xyz[:, axis])
    n = len(x)
    cuts = [x[min(n - 1, (p * n) // nparts)] for p in range(1, nparts)]
    bounds = np.array([-np.inf] + cuts + [np.inf])
    halo = 2.0 * (float(np.max(radii)) + probe) + skin
    return Slabs(axis, bounds, halo)


def local_problem(slabs: Slabs, p: int, ids, coords, radii):
    """From atoms (global ids, coords, radii) that include every atom of slab p's extended
    region: the atoms of that region, sorted by global id, and a mask of the owned ones."""
    ids = np.asarray(ids)
    xyz = np.asarray(coords, dtype=np.float64)
    keep = slabs.extended(p, xyz[:, slabs.axis])
    order = np.argsort(ids[keep], kind="stable")
    gid = ids[keep][order]
    sub_xyz = xyz[keep][order]
    sub_r = np.asarray(radii)[keep][order]
    owned = slabs.owner(sub_xyz[:, slabs.axis]) == p
    return gid, sub_xyz, sub_r, owned


def gpu_compute(device: int = 0, probe: float = PROBE, precision: str = "mixed"):
    """The default compute step: dsasa_compute on this rank's GPU (host arrays in and out)."""
    from . import api
    ctx = api.Context(device=device, precision=precision)

    def run(coords, radii):
        a, g = ctx.compute_host(coords, radii, probe=probe)
        ctx.status_sync()
        return a, g
    return run


def _all_gather_varlen(t, group=None):
    """all_gather of tensors whose first dimension differs between ranks."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size(group)
    n = torch.tensor([t.shape[0]], dtype=torch.int64, device=t.device)
    sizes = [torch.zeros_like(n) for _ in range(ws)]
    dist.all_gather(sizes, n, group=group)
    mx = int(max(int(s.item()) for s in sizes))
    pad = torch.zeros((mx,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
    pad[: t.shape[0]] = t
    out = [torch.zeros_like(pad) for _ in range(ws)]
    dist.all_gather(out, pad, group=group)
    return [o[: int(s.item())] for o, s in zip(out, sizes)]


def distributed_sasa(slabs: Slabs, ids, coords, radii, compute=None, group=None):
    """One rank's part of the decomposed computation.

    ids, coords, radii: the atoms this rank owns (global ids, (k, 3), (k,)), host arrays.
    Exchanges the boundary layers (one all_gather of coordinates, radii and ids), computes the
    rank's extended slab and returns (ids, areas, grad) of its owned atoms, sorted by id."""
    import torch
    import torch.distributed as dist
    rank = dist.get_rank(group)
    if slabs.nparts != dist.get_world_size(group):
        raise ValueError("one slab per rank")
    compute = compute or gpu_compute()
    ids = np.asarray(ids, dtype=np.int64)
    xyz = np.asarray(coords, dtype=np.float64).reshape(-1, 3)
    r = np.asarray(radii, dtype=np.float64)
    if np.any(slabs.owner(xyz[:, slabs.axis]) != rank):
        raise ValueError("every atom passed to a rank must lie in its slab")
    layer = slabs.boundary_layer(rank, xyz[:, slabs.axis])
    pack = torch.as_tensor(np.concatenate([xyz[layer], r[layer, None], ids[layer, None].astype(np.float64)], 1))
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    got = _all_gather_varlen(pack.to(dev), group)
    recv = [g.cpu().numpy() for k, g in enumerate(got) if k != rank]
    hx = np.concatenate([xyz] + [g[:, :3] for g in recv]) if recv else xyz
    hr = np.concatenate([r] + [g[:, 3] for g in recv]) if recv else r
    hid = np.concatenate([ids] + [g[:, 4].astype(np.int64) for g in recv]) if recv else ids
    gid, sx, sr, owned = local_problem(slabs, rank, hid, hx, hr)
    a, g = compute(sx, sr)
    return gid[owned], np.asarray(a)[owned], np.asarray(g)[owned]
