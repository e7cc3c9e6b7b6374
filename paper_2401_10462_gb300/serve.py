"""Continuous-batching SASA + gradient server on one GPU.

Requests (a molecule: coordinates and radii on the host, and the key of the molecule they
are a frame of) arrive over time.  The server keeps a fixed set of in-flight slots, each with
its own CUDA stream, library context and preallocated device input buffers; admission is by
that device-memory budget (a batch takes queued requests first-come first-served while their
atoms fit the slot).  Whenever a slot is free and requests are waiting, it packs them into
one batch and issues, on its stream, the host-to-device copy of the coordinates and radii and
one batched pass of the kernels over all molecules of the batch
(dsasa_compute_batch_resident: per-molecule cell grids and offsets, no interaction across
molecules).  Requests that arrive while other batches are on the GPU go into the next free
slot, so their work overlaps on the device with the batches already running.

GB300-specific: the outputs are written by the kernels straight into pinned host memory over
the coherent CPU-GPU link (zero-copy, no device-to-host copy), and every molecule raises a
ready flag in pinned memory as soon as its last atom is final; the host polls those flags
and returns each request on its own, before the rest of its batch has finished.

State stays on the device: every molecule key gets a slot range in a resident arena of
Verlet lists (dsasa_arena), least recently used slots are given away when the arena is full;
a frame of a molecule whose atoms all moved less than half the skin since its lists were
built reuses them (decided on the device, per molecule; the cells and simplices are always
rebuilt, so the results do not depend on reuse).  Two batches in flight never hold the same
molecule key, so a molecule's lists are never written by two batches at once.

Latency is measured per request from its arrival to its result being ready on the host.
Results do not depend on the batch composition: every atom's outputs are computed from its
own molecule only, in a fixed order.  A batch whose device status is not OK is run again one
request at a time, so that the status names the request that caused it.
"""
from __future__ import annotations

import gc
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
    key: object = None     # the molecule this request is a frame of (None: no resident state)
    done: float = None
    areas: np.ndarray = None
    grad: np.ndarray = None
    status: int = None     # the library's status code for this request (0 = OK)
    reused: bool = None    # whether its resident lists were reused

    @property
    def n(self):
        return self.coords.shape[0]


@dataclass
class _Slot:
    stream: torch.cuda.Stream
    ctx: api.Context
    d_xyz: torch.Tensor
    d_rad: torch.Tensor
    h_xyz: torch.Tensor      # pinned staging of the inputs
    h_rad: torch.Tensor
    h_area: torch.Tensor     # pinned outputs, written by the kernels (zero-copy)
    h_grad: torch.Tensor
    h_ready: torch.Tensor    # pinned int32 ready flags, one per molecule of the batch
    event: torch.cuda.Event = None
    batch: list = field(default_factory=list)
    offsets: np.ndarray = None
    pending: set = field(default_factory=set)


class _ArenaSlots:
    """First-fit slot ranges of the resident arena with least-recently-used eviction."""

    def __init__(self, capacity: int):
        self.capacity = capacity
        self.used = {}          # key -> (base, n, last use)
        self.clock = 0

    def lookup(self, key, n, busy):
        """(base, fresh) for key's slot of n atoms, allocating (and evicting keys not in
        `busy`) if needed; (-1, False) if it cannot be placed."""
        self.clock += 1
        if key in self.used and self.used[key][1] == n:
            b, _, _ = self.used[key]
            self.used[key] = (b, n, self.clock)
            return b, False
        self.used.pop(key, None)
        while True:
            b = self._fit(n)
            if b >= 0:
                self.used[key] = (b, n, self.clock)
                return b, True
            victims = [k for k in self.used if k not in busy]
            if not victims:
                return -1, False
            del self.used[min(victims, key=lambda k: self.used[k][2])]

    def _fit(self, n):
        spans = sorted((b, b + m) for b, m, _ in self.used.values())
        pos = 0
        for lo, hi in spans:
            if lo - pos >= n:
                return pos
            pos = max(pos, hi)
        return pos if self.capacity - pos >= n else -1


class Server:
    def __init__(self, device: int = 0, slots: int = 3, slot_atoms: int = 200_000, precision: str = "mixed",
                 with_grad: bool = True, resident_atoms: int = 0, skin: float = 1.0, max_molecules: int = 4096):
        self.device = torch.device("cuda", device)
        self.slot_atoms = slot_atoms
        self.with_grad = with_grad
        self.arena = api.Arena(resident_atoms, device) if resident_atoms > 0 else None
        self.arena_slots = _ArenaSlots(resident_atoms) if resident_atoms > 0 else None
        self.slots = []
        for _ in range(slots):
            st = torch.cuda.Stream(device=self.device)
            ctx = api.Context(device=device, stream=st, precision=precision, max_atoms=slot_atoms,
                              skin=skin if self.arena is not None else 0.0)
            f64 = dict(dtype=torch.float64)
            self.slots.append(_Slot(
                stream=st, ctx=ctx,
                d_xyz=torch.empty((slot_atoms, 3), device=self.device, **f64),
                d_rad=torch.empty(slot_atoms, device=self.device, **f64),
                h_xyz=torch.empty((slot_atoms, 3), pin_memory=True, **f64),
                h_rad=torch.empty(slot_atoms, pin_memory=True, **f64),
                h_area=torch.empty(slot_atoms, pin_memory=True, **f64),
                h_grad=torch.empty((slot_atoms, 3), pin_memory=True, **f64),
                h_ready=torch.zeros(max_molecules, dtype=torch.int32, pin_memory=True)))
        self.max_molecules = max_molecules

    def _busy_keys(self):
        return {r.key for s in self.slots for r in s.batch if r.key is not None}

    def _launch(self, slot: _Slot, batch):
        off = np.zeros(len(batch) + 1, dtype=np.int64)
        for k, r in enumerate(batch):
            off[k + 1] = off[k] + r.n
        n = int(off[-1])
        hx, hr = slot.h_xyz.numpy(), slot.h_rad.numpy()
        for k, r in enumerate(batch):
            hx[off[k]:off[k + 1]] = r.coords
            hr[off[k]:off[k + 1]] = r.radii
        ready = slot.h_ready.numpy()
        ready[: len(batch)] = 0
        bases = None
        if self.arena is not None:
            busy = self._busy_keys() | {r.key for r in batch}
            bases = np.full(len(batch), -1, dtype=np.int64)
            for k, r in enumerate(batch):
                if r.key is None:
                    continue
                b, fresh = self.arena_slots.lookup(r.key, r.n, busy)
                if b >= 0 and fresh:
                    self.arena.invalidate(b, r.n, slot.stream)
                bases[k] = b
        with torch.cuda.stream(slot.stream):
            slot.d_xyz[:n].copy_(slot.h_xyz[:n], non_blocking=True)
            slot.d_rad[:n].copy_(slot.h_rad[:n], non_blocking=True)
            slot.ctx.compute_batch_resident(off, slot.d_xyz[:n], slot.d_rad[:n], slot.h_area[:n],
                                            slot.h_grad[:n] if self.with_grad else None,
                                            arena=self.arena if bases is not None else None, arena_base=bases,
                                            mol_ready=slot.h_ready)
            slot.event = torch.cuda.Event()
            slot.event.record(slot.stream)
        slot.batch = batch
        slot.offsets = off
        slot.pending = set(range(len(batch)))

    def _collect(self, slot: _Slot, t0: float):
        """Return every request of the slot whose ready flag is up; True when the slot is free."""
        ready = slot.h_ready.numpy()
        off = slot.offsets
        t_now = None
        for k in list(slot.pending):
            if ready[k]:
                r = slot.batch[k]
                r.areas = slot.h_area.numpy()[off[k]:off[k + 1]].copy()
                if self.with_grad:
                    r.grad = slot.h_grad.numpy()[off[k]:off[k + 1]].copy()
                t_now = t_now if t_now is not None else time.perf_counter() - t0
                if r.done is None:
                    self._n_done += 1
                r.done = t_now
                slot.pending.discard(k)
        if slot.pending or not slot.event.query():
            return False
        self._finish(slot)
        return True

    def _finish(self, slot: _Slot):
        # the slot's stream is idle: its device status word and reuse flags cost no wait
        code = slot.ctx.status_code()
        batch = slot.batch
        reused = slot.ctx.batch_reused(len(batch)) if self.arena is not None else np.zeros(len(batch), bool)
        for k, r in enumerate(batch):
            r.status = code
            r.reused = bool(reused[k])
        if code != api.DSASA_OK and len(batch) > 1:
            # the status word covers the whole batch: run its requests one by one to find which
            # of them failed (each one's outputs do not depend on the batch)
            for r in batch:
                done = r.done
                self._launch(slot, [r])
                slot.event.synchronize()
                r.status = slot.ctx.status_code()
                r.areas = slot.h_area.numpy()[: r.n].copy()
                if self.with_grad:
                    r.grad = slot.h_grad.numpy()[: r.n].copy()
                r.done = done
        slot.batch = []
        slot.event = None
        slot.pending = set()

    def run(self, requests, realtime: bool = True):
        """Serve the requests (sorted by arrival).  With realtime=False every request is
        available at t = 0 (saturated throughput).  Python's cyclic garbage collector is paused
        while the requests are served (a collection would stall the polling loop)."""
        gc_was_enabled = gc.isenabled()
        gc.disable()
        try:
            return self._run(requests, realtime)
        finally:
            if gc_was_enabled:
                gc.enable()

    def _run(self, requests, realtime: bool):
        reqs = sorted(requests, key=lambda r: r.arrival)
        for r in reqs:
            if r.n > self.slot_atoms:
                raise ValueError(f"request {r.rid} has {r.n} atoms > slot capacity {self.slot_atoms}")
            if r.n == 0:
                raise ValueError(f"request {r.rid} has no atoms")
        queue, nxt, done = [], 0, 0
        self._n_done = sum(1 for r in reqs if r.done is not None)   # completions, counted as they come
        t0 = time.perf_counter()
        while done < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and (not realtime or reqs[nxt].arrival <= now):
                queue.append(reqs[nxt])
                nxt += 1
            progressed = False
            for slot in self.slots:
                if slot.event is not None and self._collect(slot, t0):
                    progressed = True
            done = self._n_done
            for slot in self.slots:
                if slot.event is None and queue:
                    # first come, first served while the atoms fit; a request whose molecule is
                    # in flight (in another slot or earlier in this batch) waits for it
                    busy = self._busy_keys()
                    batch, atoms, keys, rest, full = [], 0, set(), [], False
                    for r in queue:
                        if full or (r.key is not None and (r.key in busy or r.key in keys)):
                            rest.append(r)
                        elif atoms + r.n > self.slot_atoms or len(batch) >= self.max_molecules:
                            full = True
                            rest.append(r)
                        else:
                            batch.append(r)
                            atoms += r.n
                            keys.add(r.key)
                    queue = rest
                    if batch:
                        self._launch(slot, batch)
                        progressed = True
            if not progressed:
                time.sleep(20e-6)
        for slot in self.slots:   # the last batches' status and reuse flags
            if slot.event is not None:
                slot.event.synchronize()
                self._finish(slot)
        wall = time.perf_counter() - t0
        lat = np.array([r.done - (r.arrival if realtime else 0.0) for r in reqs])
        atoms = sum(r.n for r in reqs)
        failed = sum(1 for r in reqs if r.status != api.DSASA_OK)
        reused = sum(1 for r in reqs if r.reused)
        return {"requests": len(reqs), "failed": failed, "lists_reused": reused, "atoms": atoms, "wall_s": wall,
                "atoms_per_s": atoms / wall, "requests_per_s": len(reqs) / wall,
                "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                "mean_ms": 1e3 * float(lat.mean())}

    def close(self):
        for s in self.slots:
            s.ctx.close()
        if self.arena is not None:
            self.arena.close()


def request_pool(count: int, seed: int = 0, pool: int = 32, lo: int = 300, hi: int = 50000, sigma: float = 0.01):
    """The serving mix (log-uniform 300-50,000 atoms, 70 % globules / 30 % RNA mimics): a pool
    of distinct generated molecules, each request the next frame of one of them (every atom
    displaced by N(0, sigma) A per coordinate from that molecule's previous frame, as
    successive steps of a simulation)."""
    from . import inputs
    mix = inputs.serving_requests(pool, seed=seed, lo=lo, hi=hi)
    mols = [inputs.make(kind, n, s) for kind, n, s in mix]
    rng = np.random.default_rng(seed + 1)
    frames = [m.coords.copy() for m in mols]
    out = []
    for k in range(count):
        p = int(rng.integers(len(mols)))
        frames[p] = frames[p] + rng.normal(0.0, sigma, size=frames[p].shape)
        out.append(Request(k, frames[p].copy(), mols[p].radii.copy(), key=p))
    return out, mols
