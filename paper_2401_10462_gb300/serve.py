"""Continuous-batching SASA + gradient server on one GPU.

Requests (a molecule: coordinates and radii on the host) arrive over time.  The server
keeps a fixed set of in-flight slots, each with its own CUDA stream, library context and
preallocated device and pinned host buffers (device memory is reserved once; admission is
by that budget: a batch takes queued requests first-come first-served while their atoms
fit the slot).  Whenever a slot is free and requests are waiting, it packs them into one
batch and issues, on its stream, the host-to-device copies, one batched launch
(dsasa_compute_batch: per-molecule cell grids, no interaction across molecules) and the
device-to-host copies of areas and gradients.  Requests that arrive while other batches
are on the GPU go into the next free slot, so their work overlaps on the device with the
batches already running.  Latency is measured per request from its arrival to its result
being on the host.  Results do not depend on the batch composition: every atom's outputs
are computed from its own molecule only, in a fixed order.  Each finished batch's device
status is read at once and attached to its requests (a failed batch is re-run one request
at a time, so that the status names the request that caused it).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import api


@dataclass
class Request:
    rid: int
    coords: np.ndarray     # (n, 3) float64
    radii: np.ndarray      # (n,) float64
    arrival: float = 0.0   # seconds from the start of the stream
    done: float = None
    areas: np.ndarray = None
    grad: np.ndarray = None
    status: int = None     # the library's status code for this request (0 = OK)

    @property
    def n(self):
        return self.coords.shape[0]


@dataclass
class _Slot:
    stream: torch.cuda.Stream
    ctx: api.Context
    d_xyz: torch.Tensor
    d_rad: torch.Tensor
    d_area: torch.Tensor
    d_grad: torch.Tensor
    h_xyz: torch.Tensor
    h_rad: torch.Tensor
    h_area: torch.Tensor
    h_grad: torch.Tensor
    event: torch.cuda.Event = None
    batch: list = field(default_factory=list)
    offsets: np.ndarray = None


class Server:
    def __init__(self, device: int = 0, slots: int = 3, slot_atoms: int = 200_000, precision: str = "mixed",
                 with_grad: bool = True):
        self.device = torch.device("cuda", device)
        self.slot_atoms = slot_atoms
        self.with_grad = with_grad
        self.slots = []
        for _ in range(slots):
            st = torch.cuda.Stream(device=self.device)
            ctx = api.Context(device=device, stream=st, precision=precision, max_atoms=slot_atoms)
            f64 = dict(dtype=torch.float64)
            self.slots.append(_Slot(
                stream=st, ctx=ctx,
                d_xyz=torch.empty((slot_atoms, 3), device=self.device, **f64),
                d_rad=torch.empty(slot_atoms, device=self.device, **f64),
                d_area=torch.empty(slot_atoms, device=self.device, **f64),
                d_grad=torch.empty((slot_atoms, 3), device=self.device, **f64),
                h_xyz=torch.empty((slot_atoms, 3), pin_memory=True, **f64),
                h_rad=torch.empty(slot_atoms, pin_memory=True, **f64),
                h_area=torch.empty(slot_atoms, pin_memory=True, **f64),
                h_grad=torch.empty((slot_atoms, 3), pin_memory=True, **f64)))

    def _launch(self, slot: _Slot, batch):
        off = np.zeros(len(batch) + 1, dtype=np.int64)
        for k, r in enumerate(batch):
            off[k + 1] = off[k] + r.n
        n = int(off[-1])
        hx, hr = slot.h_xyz.numpy(), slot.h_rad.numpy()
        for k, r in enumerate(batch):
            hx[off[k]:off[k + 1]] = r.coords
            hr[off[k]:off[k + 1]] = r.radii
        with torch.cuda.stream(slot.stream):
            slot.d_xyz[:n].copy_(slot.h_xyz[:n], non_blocking=True)
            slot.d_rad[:n].copy_(slot.h_rad[:n], non_blocking=True)
            slot.ctx.compute_batch(off, slot.d_xyz[:n], slot.d_rad[:n], slot.d_area[:n],
                                   slot.d_grad[:n] if self.with_grad else None)
            slot.h_area[:n].copy_(slot.d_area[:n], non_blocking=True)
            if self.with_grad:
                slot.h_grad[:n].copy_(slot.d_grad[:n], non_blocking=True)
            slot.event = torch.cuda.Event()
            slot.event.record(slot.stream)
        slot.batch = batch
        slot.offsets = off

    def _finish(self, slot: _Slot, t0: float):
        # the slot's stream is idle: reading its device status word costs no wait
        code = slot.ctx.status_code()
        off = slot.offsets
        ha = slot.h_area.numpy()
        hg = slot.h_grad.numpy()
        batch = slot.batch
        for k, r in enumerate(batch):
            r.areas = ha[off[k]:off[k + 1]].copy()
            if self.with_grad:
                r.grad = hg[off[k]:off[k + 1]].copy()
            r.status = code
        if code != api.DSASA_OK and len(batch) > 1:
            # the status word covers the whole batch: run its requests one by one to find
            # which of them failed (each one's outputs do not depend on the batch)
            for r in batch:
                self._launch(slot, [r])
                slot.event.synchronize()
                r.status = slot.ctx.status_code()
                r.areas = slot.h_area.numpy()[: r.n].copy()
                if self.with_grad:
                    r.grad = slot.h_grad.numpy()[: r.n].copy()
        t_now = time.perf_counter() - t0
        for r in batch:
            r.done = t_now
        slot.batch = []
        slot.event = None

    def run(self, requests, realtime: bool = True):
        """Serve the requests (sorted by arrival).  With realtime=False every request is
        available at t = 0 (saturated throughput)."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        for r in reqs:
            if r.n > self.slot_atoms:
                raise ValueError(f"request {r.rid} has {r.n} atoms > slot capacity {self.slot_atoms}")
        queue, nxt, done = [], 0, 0
        t0 = time.perf_counter()
        while done < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and (not realtime or reqs[nxt].arrival <= now):
                queue.append(reqs[nxt])
                nxt += 1
            progressed = False
            for slot in self.slots:
                if slot.event is not None and slot.event.query():
                    self._finish(slot, t0)
                    progressed = True
            done = sum(1 for r in reqs if r.done is not None)
            for slot in self.slots:
                if slot.event is None and queue:
                    batch, atoms = [], 0
                    while queue and atoms + queue[0].n <= self.slot_atoms:
                        r = queue.pop(0)
                        batch.append(r)
                        atoms += r.n
                    if batch:
                        self._launch(slot, batch)
                        progressed = True
            if not progressed:
                time.sleep(50e-6)
        wall = time.perf_counter() - t0
        lat = np.array([r.done - (r.arrival if realtime else 0.0) for r in reqs])
        atoms = sum(r.n for r in reqs)
        failed = sum(1 for r in reqs if r.status != api.DSASA_OK)
        return {"requests": len(reqs), "failed": failed, "atoms": atoms, "wall_s": wall, "atoms_per_s": atoms / wall,
                "requests_per_s": len(reqs) / wall, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)), "mean_ms": 1e3 * float(lat.mean())}

    def close(self):
        for s in self.slots:
            s.ctx.close()


def request_pool(count: int, seed: int = 0, pool: int = 32, lo: int = 300, hi: int = 50000):
    """The serving mix (log-uniform 300-50,000 atoms, 70 % globules / 30 % RNA mimics) drawn
    from a pool of distinct generated molecules, each request a rigidly moved copy."""
    from . import inputs
    mix = inputs.serving_requests(pool, seed=seed, lo=lo, hi=hi)
    mols = [inputs.make(kind, n, s) for kind, n, s in mix]
    rng = np.random.default_rng(seed + 1)
    out = []
    for k in range(count):
        m = mols[int(rng.integers(len(mols)))]
        shift = rng.uniform(-50, 50, size=3)
        out.append(Request(k, m.coords + shift, m.radii.copy()))
    return out, mols
