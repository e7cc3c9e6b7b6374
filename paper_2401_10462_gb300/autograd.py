"""torch.autograd.Function wrappers over the CUDA library and a CUDA-graph trajectory step.

* ``nonpolar_energy(coords, radii, gamma)`` returns E_np = sum_i gamma_i A_i (the nonpolar
  solvation term, gamma = 0.005 kcal/mol/A^2 by default, i.e. the paper's 5 cal/(mol A^2)).
  Its forward runs one fused pass that returns the areas and d(sum gamma_i A_i)/dx
  (dsasa_compute_vjp with weights gamma); backward only scales that saved gradient.
* ``sasa_areas(coords, radii)`` returns the per-atom areas A_i; its backward receives
  dL/dA and recomputes the cells with those weights (a vector-Jacobian product) instead of
  storing per-simplex intermediates.
* ``molecular_volumes(coords, radii)`` returns the per-atom volumes V_i (sum = the solvent-
  accessible volume); its backward recomputes the cells with dL/dV as volume weights
  (dsasa_compute_volume_vjp).
* ``GraphedTrajectory`` captures one trajectory step (a Gaussian displacement of every
  atom, E_np and its gradient through autograd) in a CUDA graph with fixed capacities; the
  device status word is checked after replays.
"""
from __future__ import annotations

import torch

from . import api

GAMMA = 0.005   # kcal / (mol A^2)


class _Ctxs:
    """One library context per (device, precision, capacity), reused across calls."""
    cache = {}

    @classmethod
    def get(cls, device, precision="mixed", max_atoms=0):
        key = (device, precision, max_atoms)
        if key not in cls.cache:
            cls.cache[key] = api.Context(device=device, precision=precision, max_atoms=max_atoms)
        return cls.cache[key]


class NonpolarEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coords, radii, gamma, probe, lib_ctx):
        n = coords.shape[0]
        areas = torch.empty(n, dtype=torch.float64, device=coords.device)
        grad = torch.empty((n, 3), dtype=torch.float64, device=coords.device)
        w = gamma.expand(n).contiguous() if gamma.dim() == 0 or gamma.numel() == 1 else gamma.contiguous()
        lib_ctx.compute(coords.detach().contiguous(), radii.contiguous(), areas, grad, weights=w, probe=probe)
        ctx.save_for_backward(grad)
        ctx.mark_non_differentiable(areas)
        return (areas * w).sum(), areas

    @staticmethod
    def backward(ctx, g_energy, g_areas):
        (grad,) = ctx.saved_tensors
        return g_energy * grad, None, None, None, None


class SASAAreas(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coords, radii, probe, lib_ctx):
        n = coords.shape[0]
        areas = torch.empty(n, dtype=torch.float64, device=coords.device)
        lib_ctx.compute(coords.detach().contiguous(), radii.contiguous(), areas, None, probe=probe)
        ctx.save_for_backward(coords.detach(), radii)
        ctx.probe = probe
        ctx.lib_ctx = lib_ctx
        return areas

    @staticmethod
    def backward(ctx, g_areas):
        coords, radii = ctx.saved_tensors
        n = coords.shape[0]
        areas = torch.empty(n, dtype=torch.float64, device=coords.device)
        grad = torch.empty((n, 3), dtype=torch.float64, device=coords.device)
        # recompute the cells with the incoming weights: grad = d(sum_i g_i A_i)/dx
        ctx.lib_ctx.compute(coords, radii.contiguous(), areas, grad, weights=g_areas.contiguous(), probe=ctx.probe)
        return grad, None, None, None


class MolecularVolumes(torch.autograd.Function):
    """Per-atom volumes V_i = vol(B_i cap L_i) (their sum is the solvent-accessible volume);
    backward recomputes the cells with the incoming weights (dsasa_compute_volume_vjp)."""

    @staticmethod
    def forward(ctx, coords, radii, probe, lib_ctx):
        n = coords.shape[0]
        areas = torch.empty(n, dtype=torch.float64, device=coords.device)
        vols = torch.empty(n, dtype=torch.float64, device=coords.device)
        lib_ctx.compute_volume(coords.detach().contiguous(), radii.contiguous(), areas, vols, probe=probe)
        ctx.save_for_backward(coords.detach(), radii)
        ctx.probe = probe
        ctx.lib_ctx = lib_ctx
        return vols

    @staticmethod
    def backward(ctx, g_vols):
        coords, radii = ctx.saved_tensors
        n = coords.shape[0]
        areas = torch.empty(n, dtype=torch.float64, device=coords.device)
        vols = torch.empty(n, dtype=torch.float64, device=coords.device)
        grad = torch.empty((n, 3), dtype=torch.float64, device=coords.device)
        ctx.lib_ctx.compute_volume_vjp(coords, radii.contiguous(), g_vols.contiguous(), areas, vols, grad,
                                       probe=ctx.probe)
        return grad, None, None, None


def molecular_volumes(coords, radii, probe: float = api.PROBE, precision: str = "mixed", lib_ctx=None):
    """Per-atom volumes of the union of probe-inflated balls, differentiable in coords."""
    if lib_ctx is None:
        lib_ctx = _Ctxs.get(coords.device.index or 0, precision)
    return MolecularVolumes.apply(coords, radii, probe, lib_ctx)


def nonpolar_energy(coords, radii, gamma=GAMMA, probe: float = api.PROBE, precision: str = "mixed", lib_ctx=None):
    """E_np = sum_i gamma_i A_i (differentiable in coords); also returns the areas."""
    if lib_ctx is None:
        lib_ctx = _Ctxs.get(coords.device.index or 0, precision)
    g = gamma if torch.is_tensor(gamma) else torch.tensor(float(gamma), dtype=torch.float64, device=coords.device)
    return NonpolarEnergy.apply(coords, radii, g, probe, lib_ctx)


def sasa_areas(coords, radii, probe: float = api.PROBE, precision: str = "mixed", lib_ctx=None):
    """Per-atom SASA, differentiable in coords (backward recomputes with the VJP weights)."""
    if lib_ctx is None:
        lib_ctx = _Ctxs.get(coords.device.index or 0, precision)
    return SASAAreas.apply(coords, radii, probe, lib_ctx)


class GraphedTrajectory:
    """A trajectory of Gaussian displacements with E_np and its gradient, replayed from one
    captured CUDA graph.  Capacities are fixed at construction (no allocation in the graph)."""

    def __init__(self, coords, radii, sigma: float = 0.01, gamma: float = GAMMA, seed: int = 0,
                 precision: str = "mixed", headroom: float = 1.25, skin: float = 0.0, carry: int = 1):
        dev = coords.device
        n = coords.shape[0]
        self.n = n
        self.stream = torch.cuda.Stream(device=dev)
        # skin > 0: the neighbour lists stay on the device between steps and are rebuilt by
        # the device itself once an atom has moved by half the skin (no host decision in the
        # graph); with carry (see api.Context), steps that reuse the lists keep the previous
        # step's cells where exact predicates certify them
        self.lib_ctx = api.Context(device=dev.index or 0, stream=self.stream, precision=precision,
                                   max_atoms=int(n * headroom) + 64, skin=skin, carry=carry)
        self.x = coords.detach().clone().contiguous()
        self.radii = radii.contiguous()
        self.sigma = sigma
        self.gamma = torch.tensor(float(gamma), dtype=torch.float64, device=dev)
        self.noise = torch.zeros_like(self.x)
        self.energy = torch.zeros((), dtype=torch.float64, device=dev)
        self.grad = torch.zeros_like(self.x)
        self.seed = seed
        self.graph = None

    def _step(self):
        self.noise.normal_(0.0, self.sigma)
        self.x.add_(self.noise)
        xr = self.x.detach().requires_grad_(True)
        e, _ = NonpolarEnergy.apply(xr, self.radii, self.gamma, api.PROBE, self.lib_ctx)
        (g,) = torch.autograd.grad(e, xr)
        self.energy.copy_(e.detach())
        self.grad.copy_(g)

    def capture(self, warmup: int = 3):
        torch.cuda.manual_seed(self.seed)
        x0 = self.x.clone()
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            for _ in range(warmup):
                self._step()
        torch.cuda.current_stream().wait_stream(self.stream)
        self.lib_ctx.status_sync()
        self.x.copy_(x0)
        torch.cuda.manual_seed(self.seed)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self._step()
        self.x.copy_(x0)
        return self

    def replay(self, steps: int = 1):
        """Replay the captured step on the trajectory's stream (asynchronous)."""
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            for _ in range(steps):
                self.graph.replay()
        torch.cuda.current_stream().wait_stream(self.stream)

    def check(self):
        """Raise if any replay recorded a device-side error."""
        self.lib_ctx.status_sync()
