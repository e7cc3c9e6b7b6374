"""Benchmark: exact SASA + gradient throughput (atoms/s) on GB300.

Default workload (N = 1): the 5,000-atom synthetic globule (seed 0, probe 1.4 A), per-atom
SASA and the gradient of sum_i A_i, FP32 area arithmetic with FP32/FP64/exact predicates
(the mixed form), next to the all-FP64 GPU form of the same kernels.  One step = one full
pass of the hot path (cell list, per-atom cells, classification, areas, gradient).

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on the
library's stream; L2 is flushed (a 256 MiB write) before every timed step because the
inputs are smaller than L2.  Multi-GPU runs are independent replicas (the method has no
exchange step for independent molecules): every rank processes its own copy, barrier and
max over ranks, value = atoms of all ranks / slowest rank's time.

--impl reference times the CPU oracle (single-threaded, exact predicates) on the same
workload: the baseline the GPU path is compared against.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "SASA+grad atoms/s on 1 GB300 vs all-FP64 GPU form; serving p50/p99 latency"
UNIT = "atoms/s"
WORKLOAD = {"workload": "globule-5000: 5,000-atom synthetic globule, seed 0, probe 1.4 A, "
                        "SASA + gradient, FP32 terms / FP64+exact predicates"}
N_ATOMS, SEED = 5000, 0
# per-atom algorithmic FP32 work model (flop) of the hot path:
# 82 per tetrahedron of the atom's star (certification), 145 per boundary tetrahedron term
# (solid angle + 3 dihedrals), 15 per boundary edge (cap), 180 per boundary triangle; the
# gradient adds 3x the forward term work.
FLOP_STAR_TET, FLOP_TET, FLOP_EDGE, FLOP_TRI, GRAD_FACTOR = 82.0, 145.0, 15.0, 180.0, 4.0
STAR_TETS_PER_ATOM = 26.0


def peaks():
    p = {"hbm_gbs": 6800.0, "source": "fallback"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        p.update(d)
        p["source"] = "measured"
    # FP32 vector peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x max SM clock
    p["fp32_tflops"] = 152 * 128 * 2 * float(p.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    return p


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def kernel_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("dsasa_atoms.cuh", "dsasa_math.cuh", "dsasa_kernels.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2401_10462_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_counters():
    """Counters of one launch of the dominant kernel from the last ncu capture
    (profiles/traffic.json), only if the kernel sources are the ones that capture measured
    (else an empty dict)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return {}
    try:
        d = json.load(open(path))
    except Exception:
        return {}
    return d if d.get("kernel_sha") == kernel_sha() else {}


def measured_traffic():
    """DRAM bytes per launch of the dominant kernel from the last ncu capture (or None)."""
    return measured_counters().get("bytes_per_launch")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def algorithmic_flops_per_atom(rec, n):
    """Work model applied to the complex the GPU path itself exported (records of C)."""
    simp = rec[:, 1:]
    dim = (simp >= 0).sum(1) - 1
    tets = (dim == 3).sum() / n      # incidences (atom, tetrahedron of C) per atom
    edges = (dim == 1).sum() / n
    tris = (dim == 2).sum() / n
    fwd = FLOP_TET * tets + FLOP_EDGE * edges + FLOP_TRI * tris
    return FLOP_STAR_TET * STAR_TETS_PER_ATOM + GRAD_FACTOR * fwd, {"tets": tets, "edges": edges, "tris": tris}


def replica_throughput(total_s: float, ws: int, n: int, steps: int, device=None) -> float:
    """Whole-job atoms/s of N independent replicas: every rank timed `steps` steps of `n`
    atoms in `total_s` seconds; the job takes as long as the slowest rank (max over ranks)."""
    if ws > 1:
        import torch
        t = torch.tensor([total_s], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_s = float(t.item())
    return ws * n * steps / total_s


def run_gpu(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2401_10462_gb300 import api, inputs
    m = inputs.globule(N_ATOMS, SEED)
    n = m.n
    xyz = torch.as_tensor(m.coords, dtype=torch.float64, device=dev)
    rad = torch.as_tensor(m.radii, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(precision, steps, warmup, grad=True):
        ctx = api.Context(device=local, stream=stream, precision=precision)
        a = torch.empty(n, dtype=torch.float64, device=dev)
        g = torch.empty((n, 3), dtype=torch.float64, device=dev) if grad else None
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                ctx.compute(xyz, rad, a, g)
            ctx.status_sync()
            evs = []
            k0 = api.kernel_launches()
            for _ in range(steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.compute(xyz, rad, a, g)
                e1.record(stream)
                evs.append((e0, e1))
            ctx.status_sync()
        torch.cuda.synchronize(dev)
        launches = api.kernel_launches() - k0
        ms = [e0.elapsed_time(e1) for e0, e1 in evs]
        ctx.close()
        timed.launches = launches
        return ms, a, g

    def phases(precision, steps, grad=True):
        """Mean device time per kernel phase: the same steps with CUDA events recorded between
        the library's kernels (the events hold back the early launch of each next kernel, so
        these steps are not the timed ones)."""
        ctx = api.Context(device=local, stream=stream, precision=precision)
        a = torch.empty(n, dtype=torch.float64, device=dev)
        g = torch.empty((n, 3), dtype=torch.float64, device=dev) if grad else None
        with torch.cuda.stream(stream):
            ctx.compute(xyz, rad, a, g)
            ctx.status_sync()
            ctx.set_timing(True)
            for _ in range(steps):
                flush.zero_()
                ctx.compute(xyz, rad, a, g)
            ctx.status_sync()
        torch.cuda.synchronize(dev)
        ph, calls = ctx.kernel_times()
        ctx.close()
        return {k: v / max(calls, 1) for k, v in ph.items()}

    # timed region: barrier, then K steps with CUDA events on the library's stream around each
    # step; the per-kernel times (dominant kernel) come from the same number of steps right
    # after, with events between the kernels
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        ms_mixed, a_mix, g_mix = timed("mixed", args.steps, args.warmup)
        launches_mixed = timed.launches
        t_wall1 = time.perf_counter()
    ms_fp64, a_64, g_64 = timed("fp64", max(3, args.steps // 2), args.warmup)
    ph_mixed = phases("mixed", args.steps)
    ph_fp64 = phases("fp64", max(3, args.steps // 2))
    step_ms = sum(ms_mixed) / len(ms_mixed)
    value = replica_throughput(sum(ms_mixed) / 1e3, ws, n, args.steps, dev)
    fp64_value = n / (sum(ms_fp64) / len(ms_fp64) / 1e3)

    # molecular volume (per-atom power-cell volumes and d(union volume)/dx) on top of the
    # areas: same workload, same timing discipline
    ctx = api.Context(device=local, stream=stream)
    av = torch.empty(n, dtype=torch.float64, device=dev)
    vv = torch.empty(n, dtype=torch.float64, device=dev)
    gvv = torch.empty((n, 3), dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            ctx.compute_volume(xyz, rad, av, vv, vol_grad_out=gvv)
        ctx.status_sync()
        vev = []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.compute_volume(xyz, rad, av, vv, vol_grad_out=gvv)
            e1.record(stream)
            vev.append((e0, e1))
        ctx.status_sync()
    torch.cuda.synchronize(dev)
    vol_ms = sum(e0.elapsed_time(e1) for e0, e1 in vev) / len(vev)
    volume = {"ms_per_step": vol_ms, "atoms_per_s": n / vol_ms * 1e3, "total_volume_A3": float(vv.sum().item()),
              "note": "areas + per-atom power-cell volumes + d(union volume)/dx (no area gradient)"}
    ctx.close()

    # Shrake-Rupley numerical SASA (cross-check kernel): 960 points per sphere; every point
    # is tested against every overlapping neighbour, 9 FP32 operations per test
    ctx = api.Context(device=local, stream=stream)
    pts = torch.as_tensor(inputs.sphere_points(960), device=dev)
    asr = torch.empty(n, dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            ctx.compute_sr(xyz, rad, pts, asr)
        ctx.status_sync()
        sev = []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.compute_sr(xyz, rad, pts, asr)
            e1.record(stream)
            sev.append((e0, e1))
        ctx.status_sync()
    torch.cuda.synchronize(dev)
    sr_ms = sum(e0.elapsed_time(e1) for e0, e1 in sev) / len(sev)
    sr_tf = ctx.sr_tests() * 9.0 / (sr_ms / 1e3) / 1e12
    shrake_rupley = {"points_per_sphere": 960, "ms_per_call": sr_ms, "atoms_per_s": n / sr_ms * 1e3,
                     "achieved_tflops": sr_tf, "frac_of_fp32_peak": sr_tf / peaks()["fp32_tflops"],
                     "total_sasa": float(asr.sum().item()),
                     "note": "call time includes the cell-list build; 9 FP32 flop per point-neighbour test"}
    ctx.close()

    # e2e through the C ABI with pinned host buffers (copies inside the timed region)
    ctx = api.Context(device=local, stream=stream)
    hx = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    hr = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    ha = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    hg = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    hx[:] = m.coords
    hr[:] = m.radii
    for _ in range(args.warmup):
        ctx.compute_host(hx, hr, out=(ha, hg))
    e2e = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx.compute_host(hx, hr, out=(ha, hg))
        e2e.append(time.perf_counter() - t0)
    ctx.status_sync()
    e2e_value = n / (sum(e2e) / len(e2e))

    # work model from the complex the GPU path exports (outside the timed region)
    ctx = api.Context(device=local, stream=stream)
    with torch.cuda.stream(stream):
        rec = ctx.export_complex(xyz, rad).cpu().numpy()
    ctx.close()
    fl_atom, inc = algorithmic_flops_per_atom(rec, n)
    pk = peaks()
    achieved_path = fl_atom * n / (step_ms / 1e3) / 1e12
    traffic = measured_traffic()
    # the dominant kernel (largest device time per step) and its algorithmic work: the cell
    # kernel certifies the atom's star (FLOP_STAR_TET per star tetrahedron); the terms
    # kernel evaluates the area terms and their gradient; the other phases do integer and
    # topology work only (no term of the flop model)
    fwd = fl_atom - FLOP_STAR_TET * STAR_TETS_PER_ATOM
    phase_flop = {"cell": FLOP_STAR_TET * STAR_TETS_PER_ATOM * n, "terms": fwd * n}
    dom = max(ph_mixed, key=lambda k: ph_mixed[k])
    dom_ms = ph_mixed[dom]
    # the kernel is bound by instruction issue: its warp instructions per launch (ncu) over its
    # live duration, against 152 SMs x 4 schedulers x 1 instruction per cycle at the max clock
    inst = measured_counters().get("warp_instructions_per_launch")
    issue_peak = 152 * 4 * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e9
    issue = None
    if inst and dom_ms > 0:
        ach = inst / (dom_ms / 1e3) / 1e9
        issue = {"warp_inst_per_launch": inst, "achieved_ginst_s": ach, "peak_ginst_s": issue_peak,
                 "frac": ach / issue_peak,
                 "source": "smsp__inst_executed.sum of one launch (profiles/traffic.json) / live duration"}
    achieved = phase_flop.get(dom, 0.0) / (dom_ms / 1e3) / 1e12 if dom_ms > 0 else 0.0
    terms_tf = phase_flop["terms"] / (ph_mixed["terms"] / 1e3) / 1e12 if ph_mixed["terms"] > 0 else 0.0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": dict(WORKLOAD, n_atoms=n, replicas=ws, l2="flushed before every timed step (256 MiB write)",
                       fp64_form_atoms_per_s=fp64_value, mixed_over_fp64=value / ws / fp64_value,
                       total_sasa=float(a_mix.sum().item()),
                       fp64_minus_mixed_total_rel=float((a_64.sum() - a_mix.sum()).item() / a_64.sum().item()),
                       volume=volume, shrake_rupley=shrake_rupley),
        "roofline": {"bound": "alu", "kernel": f"k_atoms phase '{dom}'", "achieved": achieved,
                     "peak": pk["fp32_tflops"], "unit": "TFLOP/s", "frac": achieved / pk["fp32_tflops"],
                     "traffic": traffic, "kernel_ms": dom_ms,
                     "peak_source": "FP32 vector peak derived: 152 SMs x 128 lanes x 2 x max SM clock",
                     "work_model_flop_per_launch": phase_flop.get(dom, 0.0), "issue": issue,
                     "note": "achieved = algorithmic flop of the dominant kernel per launch / its mean "
                             "CUDA-event duration (events between the library's kernels, over K steps of "
                             "the same workload run right after the timed steps)"},
        "roofline_terms": {"achieved": terms_tf, "frac": terms_tf / pk["fp32_tflops"], "kernel_ms": ph_mixed["terms"],
                           "work_model_flop_per_launch": phase_flop["terms"]},
        "roofline_path": {"achieved": achieved_path, "frac": achieved_path / pk["fp32_tflops"],
                          "work_model_flop_per_atom": fl_atom, "complex_incidences_per_atom": inc,
                          "note": "whole step (every kernel of the hot path)"},
        "phase_ms": {"mixed": ph_mixed, "fp64": ph_fp64},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 32 * n, "d2h_bytes_per_step": 32 * n},
        "gpu_launches": launches_mixed,
        "clocks": clk.summary(),
    }
    if rank == 0 and ws == 1 and not args.no_serving:
        line["serving"] = serving_measure(512, 12, loads=(0.8,))
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(m)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def cpu_baseline(m):
    """The oracle as it stands (single-threaded C++, exact predicates) on the same molecule."""
    from oracle import oracle
    oracle.build()
    t0 = time.perf_counter()
    o = oracle.Oracle(m.coords, m.radii)
    o.areas(grad=True)
    dt = time.perf_counter() - t0
    return {"value": m.n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"the full workload ({m.n} atoms, one step: triangulation + complex + areas + gradient), {dt:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle
    from paper_2401_10462_gb300 import inputs
    oracle.build()
    m = inputs.globule(N_ATOMS, SEED)
    # each step is the oracle on a bounded sample of the workload: the atoms within a
    # patch around a seeded set of centres (about 5 s of CPU work per step)
    rng = np.random.default_rng(0)
    times, atoms = [], 0
    for s in range(args.warmup + args.steps):
        centres = rng.choice(m.n, 8, replace=False)
        idx = oracle.local_patch(m.coords, m.radii, centres, cutoff=14.0)
        t0 = time.perf_counter()
        o = oracle.Oracle(m.coords[idx], m.radii[idx])
        o.areas(grad=True)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            atoms += len(idx)
    value = atoms / sum(times)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+exact", "data": "synthetic",
            "config": dict(WORKLOAD), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "per step: the oracle on the atoms within 14 A of 8 seeded atoms of the workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serving_measure(count: int, pool: int, loads=(0.8,), seed: int = 0, slots: int = 3):
    """Serving stream: log-uniform 300-50,000-atom requests (70 % globules, 30 % RNA), Poisson
    arrivals.  The saturated throughput mu is measured first (all requests queued at t = 0);
    then the stream is replayed at lambda = load x mu and p50 / p99 latency (arrival to
    result on the host) are reported."""
    from paper_2401_10462_gb300 import serve, inputs
    reqs, mols = serve.request_pool(count, seed=seed, pool=pool)
    srv = serve.Server(slots=slots, slot_atoms=200_000)
    srv.run(reqs[: min(len(reqs), 32)], realtime=False)          # warm-up
    for r in reqs:
        r.done = None
    sat = srv.run(reqs, realtime=False)
    mu = sat["requests_per_s"]
    out = {"requests": count, "pool_molecules": pool, "slots": slots, "saturated_requests_per_s": mu,
           "saturated_atoms_per_s": sat["atoms_per_s"], "loads": []}
    for ld in loads:
        t = inputs.poisson_arrivals(count, ld * mu, seed=seed + 11)
        for r, ti in zip(reqs, t):
            r.arrival = float(ti)
            r.done = None
        st = srv.run(reqs, realtime=True)
        out["loads"].append({"lambda_over_mu": ld, "lambda_requests_per_s": ld * mu, "p50_ms": st["p50_ms"],
                             "p99_ms": st["p99_ms"], "atoms_per_s": st["atoms_per_s"]})
    srv.close()
    return out


def run_capsid(args):
    """The 1,000,000-atom capsid-like shell, mixed vs FP64, SASA + gradient."""
    import torch
    from paper_2401_10462_gb300 import api, inputs
    m = inputs.make("shell", 1_000_000, 0)
    dev = torch.device("cuda", 0)
    xyz = torch.as_tensor(m.coords, device=dev)
    rad = torch.as_tensor(m.radii, device=dev)
    stream = torch.cuda.Stream(device=dev)
    res = {}
    for prec, steps in (("mixed", args.steps), ("fp64", max(1, args.steps // 2))):
        ctx = api.Context(stream=stream, precision=prec)
        a = torch.empty(m.n, dtype=torch.float64, device=dev)
        g = torch.empty((m.n, 3), dtype=torch.float64, device=dev)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                ctx.compute(xyz, rad, a, g)
            ctx.status_sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                ctx.compute(xyz, rad, a, g)
            e1.record(stream)
            ctx.status_sync()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[prec] = {"ms_per_step": ms, "atoms_per_s": m.n / ms * 1e3, "total_sasa": float(a.sum().item())}
        ctx.close()
    print(json.dumps({"workload": "capsid shell 1,000,000 atoms", "outer_radius_A": m.extent,
                      "density_per_A3": m.density(), "inputs_larger_than_L2": True, **res,
                      "mixed_over_fp64": res["mixed"]["atoms_per_s"] / res["fp64"]["atoms_per_s"]}), flush=True)


def run_trajectory(args):
    """Trajectory: 20,000-atom globule, E_np through the autograd Function, Gaussian steps
    (sigma 0.01 A) replayed from one captured CUDA graph; reports ms per graphed step without
    and with Verlet-skin lists (skin 1 A: rebuilt on the device once an atom moved 0.5 A)."""
    import torch
    from paper_2401_10462_gb300 import autograd as ag, inputs
    m = inputs.make("globule", 20000, 0)
    dev = torch.device("cuda", 0)
    out = {"workload": "graphed trajectory, 20,000-atom globule"}
    for skin in (0.0, 1.0):
        tr = ag.GraphedTrajectory(torch.as_tensor(m.coords, device=dev), torch.as_tensor(m.radii, device=dev),
                                  sigma=0.01, seed=0, skin=skin).capture()
        tr.replay(args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = max(args.steps, 100)
        e0.record()
        tr.replay(steps)      # replays on the trajectory stream, joined back to the current one
        e1.record()
        torch.cuda.synchronize()
        tr.check()
        ms = e0.elapsed_time(e1) / steps
        out[f"skin_{skin:g}"] = {"steps": steps, "ms_per_step": ms, "atoms_per_s": m.n / ms * 1e3,
                                 "energy_kcal_mol": tr.energy.item()}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="globule5k", choices=["globule5k", "capsid", "trajectory", "serving"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "capsid":
        run_capsid(args)
    elif args.workload == "trajectory":
        run_trajectory(args)
    elif args.workload == "serving":
        print(json.dumps({"workload": "serving stream, 4,096 requests of 300-50,000 atoms",
                          **serving_measure(4096, 32, loads=(0.5, 0.8, 0.95))}), flush=True)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
