"""Benchmark: exact SASA + gradient throughput (atoms/s) on GB300.

Headline workload (N = 1): the 5,000-atom synthetic globule (seed 0, probe 1.4 A), per-atom
SASA and the gradient of sum_i A_i, FP32 area arithmetic with FP32/FP64/exact predicates
(the mixed form), next to the all-FP64 GPU form of the same kernels.  One step = one full
pass of the hot path (cell list, per-atom cells, classification, areas, gradient).

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on the
library's stream; L2 is flushed (a 256 MiB write) before every timed step because the
inputs are smaller than L2.  Multi-GPU runs are independent replicas (the method has no
exchange step for independent molecules): every rank processes its own copy, barrier and
max over ranks, value = atoms of all ranks / slowest rank's time.

The same JSON line also carries (rank 0, one GPU): the arithmetic roofs measured in this run
(libdsasa_peaks.so), the roofline of the dominant kernel from the oracle-counted work model
(profiles/work_model_globule5000.json), the accuracy against the FP64 oracle, the
1,000,000-atom capsid shell, the graphed 20,000-atom trajectory, the 4,096-request serving
stream at three loads, each with its own clock record, and the oracle timed on the host.

--impl reference times the CPU oracle (exact predicates, FP64) on the same workload: every
step is one full pass over the 5,000-atom globule.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import platform
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
WORK_MODEL = os.path.join(ROOT, "profiles", "work_model_globule5000.json")


def driver_peaks():
    p = {"hbm_gbs": 6800.0, "source": "fallback"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        p.update(d)
        p["source"] = "measured"
    return p


def measure_peaks(device: int):
    """FP32 FMA, FP64 FMA, rsqrt and atan2f throughput and the warp-instruction issue rate,
    measured now on this GPU by libdsasa_peaks.so (CUDA events; no setting is changed)."""
    from paper_2401_10462_gb300 import build
    lib = ctypes.CDLL(build.PEAKS_LIB)
    lib.dsasa_peaks_measure.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    out = (ctypes.c_double * 6)()
    rc = lib.dsasa_peaks_measure(device, out)
    if rc != 0:
        raise RuntimeError(f"peak microbenchmarks failed (CUDA error {rc})")
    return {"fp32_tflops": out[0], "fp64_tflops": out[1], "rsqrt_gops": out[2], "atan2f_gops": out[3],
            "issue_ginst_s": out[4], "sms": int(out[5]),
            "source": "microbenchmarks in this run (libdsasa_peaks.so: FMA / rsqrt / atan2f streams, "
                      "8 blocks of 256 threads per SM, best of 5, CUDA events)"}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while a measured region runs."""

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
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            time.sleep(0.15)   # the first sample lands inside the region
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.06)
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


def measured_counters(name="traffic.json"):
    """Counters of one launch of the dominant kernel from the last ncu capture
    (profiles/<name>), only if the kernel sources are the ones that capture measured."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return {}
    try:
        d = json.load(open(path))
    except Exception:
        return {}
    return d if d.get("kernel_sha") == kernel_sha() else {}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_throughput(total_s: float, ws: int, n: int, steps: int, device=None) -> float:
    """Whole-job atoms/s of N independent replicas: every rank timed `steps` steps of `n`
    atoms in `total_s` seconds; the job takes as long as the slowest rank (max over ranks)."""
    if ws > 1:
        import torch
        t = torch.tensor([total_s], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_s = float(t.item())
    return ws * n * steps / total_s


class Timer:
    """K steps of ctx.compute on one molecule, each bracketed by CUDA events, L2 flushed
    before every timed step; per-kernel phases on K further steps."""

    def __init__(self, api, torch, dev, local, stream, flush):
        self.api, self.torch, self.dev, self.local, self.stream, self.flush = api, torch, dev, local, stream, flush

    def steps(self, xyz, rad, precision, steps, warmup, grad=True):
        api, torch = self.api, self.torch
        n = xyz.shape[0]
        ctx = api.Context(device=self.local, stream=self.stream, precision=precision)
        a = torch.empty(n, dtype=torch.float64, device=self.dev)
        g = torch.empty((n, 3), dtype=torch.float64, device=self.dev) if grad else None
        with torch.cuda.stream(self.stream):
            for _ in range(warmup):
                ctx.compute(xyz, rad, a, g)
            ctx.status_sync()
            evs = []
            k0 = api.kernel_launches()
            for _ in range(steps):
                self.flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(self.stream)
                ctx.compute(xyz, rad, a, g)
                e1.record(self.stream)
                evs.append((e0, e1))
            ctx.status_sync()
        torch.cuda.synchronize(self.dev)
        launches = api.kernel_launches() - k0
        ms = [e0.elapsed_time(e1) for e0, e1 in evs]
        ctx.close()
        return ms, a, g, launches

    def phases(self, xyz, rad, precision, steps, grad=True):
        """Mean device time per kernel phase: the same steps with CUDA events recorded between
        the library's kernels (the events hold back the early launch of each next kernel, so
        these steps are not the timed ones)."""
        api, torch = self.api, self.torch
        n = xyz.shape[0]
        ctx = api.Context(device=self.local, stream=self.stream, precision=precision)
        a = torch.empty(n, dtype=torch.float64, device=self.dev)
        g = torch.empty((n, 3), dtype=torch.float64, device=self.dev) if grad else None
        with torch.cuda.stream(self.stream):
            ctx.compute(xyz, rad, a, g)
            ctx.status_sync()
            ctx.set_timing(True)
            for _ in range(steps):
                self.flush.zero_()
                ctx.compute(xyz, rad, a, g)
            ctx.status_sync()
        torch.cuda.synchronize(self.dev)
        ph, calls = ctx.kernel_times()
        ctx.close()
        return {k: v / max(calls, 1) for k, v in ph.items()}


def roofline_block(wm, n, ph, pk, dpk, counters):
    """The dominant kernel's roofline from the oracle-counted work model (per-atom flop x the
    atoms one launch processes / its mean CUDA-event duration) against the roofs measured in
    this run, plus the terms kernel and the instruction-issue roof."""
    dom = max(ph, key=lambda k: ph[k])
    flop = {"cell": wm["cell_flop_per_atom"] * n, "terms": wm["terms_flop_per_atom"] * n}
    dom_ms = ph[dom]
    achieved = flop.get(dom, 0.0) / (dom_ms / 1e3) / 1e12 if dom_ms > 0 else 0.0
    issue = None
    inst = counters.get("warp_instructions_per_launch")
    if inst and dom_ms > 0:
        ach = inst / (dom_ms / 1e3) / 1e9
        issue = {"warp_inst_per_launch": inst, "achieved_ginst_s": ach, "peak_ginst_s": pk["issue_ginst_s"],
                 "frac": ach / pk["issue_ginst_s"],
                 "source": "smsp__inst_executed.sum of one ncu launch (profiles/traffic.json) / live duration; "
                           "peak = warp instructions/s of the FP32 FMA microbenchmark"}
    names = {"cell": "k_atoms<float,0,64,64,PH_CC or PH_CELL> (restricted power cell; with all atoms in one wave "
                     "also the classification)", "terms": "k_atoms<float,1,64,64,PH_TERMS>"}
    out = {"bound": "alu", "kernel": names.get(dom, dom), "achieved": achieved, "peak": pk["fp32_tflops"],
           "unit": "TFLOP/s", "frac": achieved / pk["fp32_tflops"], "traffic": counters.get("bytes_per_launch"),
           "kernel_ms": dom_ms, "peak_source": "FP32 FMA roof measured in this run (of measured)",
           "frac_of_fp64_roof": achieved / pk["fp64_tflops"],
           "work_model": f"{wm['flop_table']['certification']:.0f} flop per star tetrahedron x "
                         f"{wm['star_tets_per_atom']:.2f} per atom (oracle counts, profiles/work_model_globule5000.json)",
           "work_model_flop_per_launch": flop.get(dom, 0.0), "issue": issue,
           "hbm_peak_gbs": dpk.get("hbm_gbs"), "hbm_peak_source": dpk.get("source"),
           "note": "achieved = algorithmic flop per launch / mean CUDA-event duration of the kernel (events "
                   "between the library's kernels, K steps of the same workload after the timed steps)"}
    t_ms = ph.get("terms", 0.0)
    terms = None
    if t_ms > 0:
        tf = flop["terms"] / (t_ms / 1e3) / 1e12
        sfu = wm["terms_sfu_per_atom"] * n / (t_ms / 1e3) / 1e9
        terms = {"kernel_ms": t_ms, "achieved_tflops": tf, "frac_of_fp32_roof": tf / pk["fp32_tflops"],
                 "achieved_sfu_gops": sfu, "frac_of_rsqrt_roof": sfu / pk["rsqrt_gops"],
                 "work_model_flop_per_launch": flop["terms"]}
    return out, terms


def accuracy(ra, rg, a, g):
    """Errors of one GPU result against the FP64 oracle: plain relative and with the floors
    of the stated tolerances (areas max(A, 1 A^2), gradients max(|g|, 1e-2))."""
    a, g = np.asarray(a), np.asarray(g)
    da = np.abs(a - ra)
    dg = np.linalg.norm(g - rg, axis=1)
    gn = np.linalg.norm(rg, axis=1)
    pos, gpos = ra > 0, gn > 0
    return {"max_area_rel": float((da[pos] / ra[pos]).max()) if pos.any() else 0.0,
            "max_area_rel_floor1": float((da / np.maximum(ra, 1.0)).max()),
            "total_rel": float(abs(a.sum() - ra.sum()) / ra.sum()),
            "max_grad_rel": float((dg[gpos] / gn[gpos]).max()) if gpos.any() else 0.0,
            "max_grad_rel_floor": float((dg / np.maximum(gn, 1e-2)).max()),
            "n_area_over_1e-4_rel": int((da[pos] / ra[pos] > 1e-4).sum()),
            "n_grad_over_1e-3_rel": int((dg[gpos] / gn[gpos] > 1e-3).sum()),
            "n_over_stated_tolerances": int((da > 1e-4 * np.maximum(ra, 1.0)).sum()
                                            + (dg > 1e-3 * np.maximum(gn, 1e-2)).sum())}


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
    tm = Timer(api, torch, dev, local, stream, flush)
    pk = measure_peaks(local)
    dpk = driver_peaks()

    # timed region: barrier, then K steps with CUDA events on the library's stream around each
    # step; the clock sampler runs over the timed steps and the per-kernel steps after them
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        ms_mixed, a_mix, g_mix, launches_mixed = tm.steps(xyz, rad, "mixed", args.steps, args.warmup)
        ph_mixed = tm.phases(xyz, rad, "mixed", args.steps)
    ms_fp64, a_64, g_64, _ = tm.steps(xyz, rad, "fp64", max(3, args.steps // 2), args.warmup)
    ph_fp64 = tm.phases(xyz, rad, "fp64", max(3, args.steps // 2))
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
                     "achieved_tflops": sr_tf, "frac_of_fp32_roof": sr_tf / pk["fp32_tflops"],
                     "total_sasa": float(asr.sum().item()),
                     "note": "call time includes the cell-list build; 9 FP32 flop per point-neighbour test"}
    ctx.close()

    # e2e through the C ABI with pinned host buffers: the kernels read the inputs and write the
    # outputs in host memory over the CPU-GPU link (inside the timed region, with the sync)
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
    ctx.close()
    e2e_value = n / (sum(e2e) / len(e2e))

    wm = json.load(open(WORK_MODEL))
    roofline, roofline_terms = roofline_block(wm, n, ph_mixed, pk, dpk, measured_counters())
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": dict(WORKLOAD, n_atoms=n, replicas=ws, l2="flushed before every timed step (256 MiB write)",
                       fp64_form_atoms_per_s=fp64_value, mixed_over_fp64=value / ws / fp64_value,
                       total_sasa=float(a_mix.sum().item()),
                       fp64_minus_mixed_total_rel=float((a_64.sum() - a_mix.sum()).item() / a_64.sum().item()),
                       volume=volume, shrake_rupley=shrake_rupley),
        "roofline": roofline,
        "roofline_terms": roofline_terms,
        "peaks_measured": pk,
        "phase_ms": {"mixed": ph_mixed, "fp64": ph_fp64},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 32 * n, "d2h_bytes_per_step": 32 * n,
                "transfer": "pinned host buffers read and written in place by the kernels over the CPU-GPU "
                            "link (dsasa_compute_host); wall clock per call including the synchronisation"},
        "gpu_launches": launches_mixed,
        "clocks": clk.summary(),
    }
    # the further workloads and the CPU legs: a failure of one of them is reported in its own
    # key, and the headline line is still printed
    def leg(name, fn):
        try:
            line[name] = fn()
        except Exception as ex:   # noqa: BLE001 - reported, not swallowed
            line[name] = {"error": f"{type(ex).__name__}: {ex}"}

    if rank == 0 and ws == 1 and not args.quick:
        leg("capsid", lambda: capsid_measure(args, tm, wm, pk))
        leg("trajectory", lambda: trajectory_measure(args, local))

        def serving():
            with ClockSampler(local) as sclk:
                out = serving_measure(4096, 32, loads=(0.5, 0.8, 0.95))
            out["clocks"] = sclk.summary()
            return out
        leg("serving", serving)
    if rank == 0 and not args.no_cpu_baseline:
        def cpu_legs():
            base, ref = cpu_baseline(m)
            line["accuracy_vs_oracle"] = {
                "mixed": accuracy(ref[0], ref[1], a_mix.cpu().numpy(), g_mix.cpu().numpy()),
                "fp64": accuracy(ref[0], ref[1], a_64.cpu().numpy(), g_64.cpu().numpy()),
                "tolerances": "per atom |dA| <= 1e-4 max(A, 1 A^2); total 1e-6; |dg| <= 1e-3 max(|g|, 1e-2)"}
            return base
        leg("cpu_baseline", cpu_legs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def capsid_measure(args, tm, wm, pk):
    """The 1,000,000-atom capsid-like shell (inputs larger than L2), mixed vs FP64, SASA +
    gradient; the dominant (split) cell kernel's roofline with the globule's per-atom work
    model, and its DRAM traffic per atom when an ncu record of that kernel exists."""
    import torch
    from paper_2401_10462_gb300 import inputs
    m = inputs.make("shell", 1_000_000, 0)
    xyz = torch.as_tensor(m.coords, device=tm.dev)
    rad = torch.as_tensor(m.radii, device=tm.dev)
    res = {"workload": "capsid shell 1,000,000 atoms, seed 0", "outer_radius_A": m.extent,
           "density_per_A3": m.density(), "inputs_larger_than_L2": True}
    with ClockSampler(tm.local) as clk:
        ms, a, _, _ = tm.steps(xyz, rad, "mixed", max(3, args.steps // 2), 2)
        ph = tm.phases(xyz, rad, "mixed", 3)
    res["clocks"] = clk.summary()
    ms64, a64, _, _ = tm.steps(xyz, rad, "fp64", 3, 1)
    t = sum(ms) / len(ms)
    t64 = sum(ms64) / len(ms64)
    res.update({"mixed": {"ms_per_step": t, "atoms_per_s": m.n / t * 1e3, "total_sasa": float(a.sum().item())},
                "fp64": {"ms_per_step": t64, "atoms_per_s": m.n / t64 * 1e3, "total_sasa": float(a64.sum().item())},
                "mixed_over_fp64": t64 / t, "phase_ms": ph,
                "fp64_minus_mixed_total_rel": float((a64.sum() - a.sum()).item() / a64.sum().item())})
    cnt = measured_counters("traffic_capsid.json")
    rl, _ = roofline_block(wm, m.n, ph, pk, driver_peaks(), cnt)
    rl["work_model"] += " (per-atom counts of the 5,000-atom globule, same placement rules)"
    rl["traffic_bytes_per_atom"] = (cnt["bytes_per_launch"] / m.n) if cnt.get("bytes_per_launch") else None
    res["roofline"] = rl
    return res


def trajectory_measure(args, local):
    """20,000-atom globule, E_np through the autograd Function, Gaussian steps (sigma 0.01 A)
    replayed from one captured CUDA graph: cells built afresh every step (no lists), with
    Verlet-skin lists, and with the lists and carried cells (the incremental update)."""
    import torch
    from paper_2401_10462_gb300 import autograd as ag, inputs
    m = inputs.make("globule", 20000, 0)
    dev = torch.device("cuda", local)
    out = {"workload": "graphed trajectory, 20,000-atom globule, sigma 0.01 A"}
    for name, skin, carry in (("skin_0", 0.0, 0), ("skin_1", 1.0, 0), ("skin_1_carry", 1.0, 1)):
        tr = ag.GraphedTrajectory(torch.as_tensor(m.coords, device=dev), torch.as_tensor(m.radii, device=dev),
                                  sigma=0.01, seed=0, skin=skin, carry=carry).capture()
        tr.replay(args.warmup)
        torch.cuda.synchronize()
        steps = max(args.steps, 200)
        with ClockSampler(local) as clk:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            tr.replay(steps)      # replays on the trajectory stream, joined back to the current one
            e1.record()
            torch.cuda.synchronize()
        tr.check()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"steps": steps, "ms_per_step": ms, "atoms_per_s": m.n / ms * 1e3,
                     "energy_kcal_mol": tr.energy.item(), "clocks": clk.summary()}
        if skin > 0:
            # after the timed region: 100 more steps one at a time, reading the list reuse and
            # the carried cells of each
            reused, carried = 0, 0
            for _ in range(100):
                tr.replay(1)
                reused += tr.lib_ctx.lists_reused()
                carried += tr.lib_ctx.cells_carried()
            out[name]["steps_reusing_lists"] = reused / 100
            out[name]["cells_carried_per_step"] = carried / (100 * m.n)
    return out


def host_info():
    model = platform.processor() or platform.machine()
    try:
        txt = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in txt.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


def cpu_baseline(m):
    """The oracle as it stands on the host cores of the machine that runs the GPU: single-threaded end to end (triangulation
    + complex + areas + gradient) on the 304- and 5,000-atom globules and a 20,000-atom one,
    and its area and gradient stage on all cores (OpenMP; the triangulation stays serial);
    1,000,000 atoms extrapolated as n log n from the 20,000-atom time.  Returns the record and
    the oracle's areas and gradient of the 5,000-atom workload."""
    from oracle import oracle
    from paper_2401_10462_gb300 import inputs
    oracle.build()
    info = host_info()
    sizes = {}
    ref = None
    for name, mol in (("globule304", inputs.globule(304, 0)), ("globule5000", m), ("globule20000", inputs.make("globule", 20000, 0))):
        t0 = time.perf_counter()
        o = oracle.Oracle(mol.coords, mol.radii)
        t1 = time.perf_counter()
        a, _, g = o.areas(grad=True)
        t2 = time.perf_counter()
        _, _, _, used = o.areas_parallel(info["nproc"] or 1)
        t3 = time.perf_counter()
        sizes[name] = {"n_atoms": mol.n, "single_thread_s": t2 - t0, "single_thread_atoms_per_s": mol.n / (t2 - t0),
                       "triangulation_and_complex_s": t1 - t0, "area_gradient_stage_1_thread_s": t2 - t1,
                       "area_gradient_stage_all_cores_s": t3 - t2, "threads": used}
        if mol is m:
            ref = (a, g)
    t20 = sizes["globule20000"]["single_thread_s"]
    ext = t20 * (1e6 * math.log(1e6)) / (2e4 * math.log(2e4))
    sizes["capsid1000000_extrapolated"] = {"n_atoms": 1_000_000, "single_thread_s": ext,
                                           "single_thread_atoms_per_s": 1e6 / ext,
                                           "note": "extrapolated as n log n from the 20,000-atom time, not measured"}
    head = sizes["globule5000"]
    rec = {"value": head["single_thread_atoms_per_s"], "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"the full 5,000-atom workload, one pass (triangulation + complex + areas + gradient), "
                     f"{head['single_thread_s']:.1f} s on one core; sizes and the all-core area stage below",
           "host": info, "sizes": sizes}
    return rec, ref


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle
    from paper_2401_10462_gb300 import inputs
    oracle.build()
    m = inputs.globule(N_ATOMS, SEED)
    # every step is one full oracle pass over the same 5,000-atom workload (about 3-4 s)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        o = oracle.Oracle(m.coords, m.radii)
        o.areas(grad=True)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    value = m.n * len(times) / sum(times)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+exact", "data": "synthetic",
            "config": dict(WORKLOAD), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "per step: one full oracle pass over the 5,000-atom workload",
                             "host": host_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serving_measure(count: int, pool: int, loads=(0.8,), seed: int = 0, slots: int = 3):
    """Serving stream: log-uniform 300-50,000-atom requests (70 % globules, 30 % RNA), Poisson
    arrivals.  The saturated throughput mu is measured first (all requests queued at t = 0);
    then the stream is replayed at lambda = load x mu and p50 / p99 latency (arrival to
    result on the host) are reported."""
    from paper_2401_10462_gb300 import serve, inputs
    reqs, mols = serve.request_pool(count, seed=seed, pool=pool)
    resident = int(1.25 * sum(m.n for m in mols)) + 1000
    srv = serve.Server(slots=slots, slot_atoms=200_000, resident_atoms=resident, skin=1.0)
    srv.run(reqs[: min(len(reqs), 32)], realtime=False)          # warm-up
    for r in reqs:
        r.done = None
    sat = srv.run(reqs, realtime=False)
    mu = sat["requests_per_s"]
    out = {"requests": count, "pool_molecules": pool, "slots": slots, "saturated_requests_per_s": mu,
           "saturated_atoms_per_s": sat["atoms_per_s"], "failed": sat["failed"],
           "lists_reused_saturated": sat["lists_reused"], "resident_arena_atoms": resident,
           "design": "zero-copy outputs in pinned host memory, per-molecule ready flags polled by the host, "
                     "resident Verlet lists (skin 1 A) per pool molecule; requests are frames of the pool "
                     "molecules (N(0, 0.01 A) per coordinate per frame)", "loads": []}
    for ld in loads:
        t = inputs.poisson_arrivals(count, ld * mu, seed=seed + 11)
        for r, ti in zip(reqs, t):
            r.arrival = float(ti)
            r.done = None
        st = srv.run(reqs, realtime=True)
        out["loads"].append({"lambda_over_mu": ld, "lambda_requests_per_s": ld * mu, "p50_ms": st["p50_ms"],
                             "p99_ms": st["p99_ms"], "atoms_per_s": st["atoms_per_s"], "failed": st["failed"],
                             "lists_reused": st["lists_reused"]})
    srv.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="all", choices=["all", "capsid", "trajectory", "serving"])
    ap.add_argument("--quick", action="store_true", help="headline workload only (no capsid, trajectory, serving)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "all":
        run_gpu(args)
        return
    import torch
    from paper_2401_10462_gb300 import api
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    tm = Timer(api, torch, dev, 0, stream, flush)
    if args.workload == "capsid":
        print(json.dumps(capsid_measure(args, tm, json.load(open(WORK_MODEL)), measure_peaks(0))), flush=True)
    elif args.workload == "trajectory":
        print(json.dumps(trajectory_measure(args, 0)), flush=True)
    else:
        print(json.dumps({"workload": "serving stream, 4,096 requests of 300-50,000 atoms",
                          **serving_measure(4096, 32, loads=(0.5, 0.8, 0.95))}), flush=True)


if __name__ == "__main__":
    main()
