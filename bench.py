#!/usr/bin/env python
"""Benchmark of the additive multilevel Helmholtz cycle on GB300.

Default workload: the 2D complex128 variant-sweep configuration -- depth 6
(729 x 729 fine cells, 529,984 interior unknowns), k = 20 pi, exterior
scaling layer of 10% per side with theta = pi/6, f = three Gaussians of width
0.02 (seed 1).  A step is one BPX additive FAS cycle (omega = 0.6 on every
level) through the C ABI: fused fine sweep, coarse sweeps, prolongation, and
the fused fine residual norm.  The metric is fine-grid interior DoF-updates/s
(interior vertices x cycles / s).  L2 is flushed (256 MB write) before every
timed step; steps are timed with CUDA events on the solver's stream.

``--impl reference`` times the FP64 CPU oracle (test infrastructure) on the
host cores on a bounded sample of the same workload.  Under torchrun with
N > 1 every rank runs an independent replica of the solve (a single solve
does not shard); value is the sum over ranks divided by the slowest rank's
time.
"""
from __future__ import annotations

import argparse
import hashlib
import itertools
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1508_03954_gb300 import workloads as W  # noqa: E402

METRIC = "additive-cycle DoF-updates/s"
UNIT = "DoF-updates/s"
# FP64 peak of GB300 from unit counts and clock: 152 SMs x 2 FP64 FMA/clk/SM
# x 2 flops x 2.07 GHz (the nominal 1.25 TFLOP/s of the data sheet).
FP64_PEAK_FLOPS = 152 * 2 * 2 * 2.07e9
FP32_PEAK_FLOPS = 152 * 128 * 2 * 2.07e9


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------- algorithmic counts
def complex_row_fraction(d, depth, w):
    """Fraction of interior fine vertices whose stencil row has complex
    entries (some adjacent cell lies in the scaling layer)."""
    n = 3 ** depth
    i = np.arange(n)
    if w >= 0.5:
        return 1.0
    rot = np.minimum(2 * i + 1, 2 * n - 2 * i - 1) < 2.0 * w * n
    v = np.arange(1, n)
    cplx_axis = rot[v - 1] | rot[v]
    real_frac_axis = 1.0 - cplx_axis.mean()
    return 1.0 - real_frac_axis ** d


def fine_sweep_counts(d, depth, w, bpx, omega_real, word=16, galerkin=True):
    """(flops, bytes) the method needs for one finest-level sweep.

    Per interior fine vertex (an FMA is 2 flops; real x complex MAC = 4 flops,
    complex x complex MAC = 8 flops): the residual row of 3^d entries (complex
    where a neighbouring cell is scaled, real otherwise, b folded into the
    accumulation); d-linear interpolation of the pending coarse correction
    ((5/3)^d MACs on average); restriction ((5/3)^d MACs per fine vertex);
    the coarse right-hand side either as G u_{l-1} (one 3^d Galerkin row per
    coarse vertex, galerkin=True) or as the hierarchical residual b - H uhat
    with the surplus uhat = u - P I u (galerkin=False); Jacobi (complex or
    real scaling); BPX surplus of du ((5/3)^d MACs + subtraction); the update
    and |r|^2.
    Bytes: U read, b read, U' written on the fine level (3 words per vertex),
    pending correction read and b, u written on the next coarser level (3
    words per coarse vertex)."""
    n = 3 ** depth
    ns = 3 ** d
    fc = complex_row_fraction(d, depth, w)
    row = fc * ns * 8 + (1 - fc) * ns * 4
    interp = (5.0 / 3.0) ** d * 4
    jac = fc * 6 + (1 - fc) * (2 if omega_real else 6)
    if galerkin:
        coarse_rhs = fc * 8 + (1 - fc) * 4          # one G entry per fine vertex on average
    else:
        coarse_rhs = row + 2 + interp + 2           # second row on uhat, surplus
    per = row + interp + interp + coarse_rhs + jac + (interp + 2 if bpx else 0) + 2 + 4
    flops = per * (n - 1) ** d
    nbytes = 3 * word * (n + 1) ** d + 3 * word * (n // 3 + 1) ** d
    return flops, nbytes


def axis_complex_fraction(depth, w):
    """Fraction of interior indices of one axis whose 1D rows are complex
    (a neighbouring cell of that axis lies in the scaling layer)."""
    n = 3 ** depth
    if w >= 0.5:
        return 1.0
    i = np.arange(n)
    rot = np.minimum(2 * i + 1, 2 * n - 2 * i - 1) < 2.0 * w * n
    v = np.arange(1, n)
    return float((rot[v - 1] | rot[v]).mean())


def fine_sweep3_counts(depth, w, bpx=True):
    """(FP64 flops, bytes) the separable 3D complex128 fine sweep needs per
    launch, per owned vertex and without halo recomputation (an FMA is 2
    flops, an add or a multiply 1; a complex x complex MAC is 8 flops).
    Per interior vertex and complex value:
      residual H = M_x[M_y(K_z - phi M_z) + K_y M_z] + K_x M_y M_z with
        symmetric real rows: z-pair 14, y-pair 24, x-pass with b - 20
        (complex rows along an axis: 48, 72, 50);
      pending correction u = U + P c: bilinear per coarse plane + z weights, 12.7;
      Jacobi 2 (6 with a complex factor), update 2, |r|^2 4;
      restriction R r (separable, x at c-columns, y at c-rows, z by
        accumulation), 7.6;
      Galerkin rows G u_{l-1}: 27 real MACs per coarse vertex, 4.
    With the BPX transfer the fine sweep stores du and I du; P I du is
    subtracted in the correction stage on the next coarser level (through
    the pending correction), so it is not part of this kernel's work.
    Bytes: U, b read and U' written (3 x 16 B per fine vertex); pending
    correction read, b and u written on the next coarser level (3 x 16 B per
    coarse vertex)."""
    n = 3 ** depth
    f = axis_complex_fraction(depth, w)
    per = 14 + 24 + 20 + f * ((48 - 14) + (72 - 24) + (50 - 20))
    per += 12.7 + 2 + 4 * (1 - (1 - f) ** 3) + 2 + 4 + 7.6 + 4
    flops = per * (n - 1) ** 3
    nbytes = 3 * 16 * (n + 1) ** 3 + 3 * 16 * (n // 3 + 1) ** 3
    return flops, nbytes


FINE_SWEEP3_SOURCES = ("mg_sweep3sd.cuh", "mg_sweep3s.cuh", "mg_defect3.cuh", "mg_kernels.cuh")


def fine_sweep3_roofline(cfg, sweep_ms, peaks, peak_src):
    """Roofline of the dominant kernel of the headline cycle: the finest
    level's separable complex128 sweep, bound by the FP64 pipe."""
    flops, nbytes = fine_sweep3_counts(cfg["depth"], cfg["layer_width"], bpx=True)
    t = sweep_ms / 1e3
    achieved = flops / t
    csrc = os.path.join(ROOT, "paper_1508_03954_gb300", "csrc")
    traffic, sha = recorded_traffic("fine_sweep3_c128_3d_depth5", [os.path.join(csrc, f) for f in FINE_SWEEP3_SOURCES])
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_FLOPS, "traffic": traffic,
            "kernel": "sweep3sd_kernel (finest level, separable, FP64)",
            "peak_source": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived)",
            "sweep_ms": sweep_ms, "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": nbytes,
            "hbm": {"achieved_gbs": nbytes / t / 1e9, "peak_gbs": peaks.get("hbm_gbs"),
                    "frac": nbytes / t / 1e9 / peaks.get("hbm_gbs", 6800.0), "peak_source": peak_src},
            "source_sha256_16": sha}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------- traffic record
FINE_SWEEP_SOURCES = ("mg_kernels.cuh", "mg_sweep2d.cuh", "mg_persist.cuh")


def recorded_traffic(kernel_key, source_files):
    """DRAM bytes per launch of the timed kernel from the committed ncu summary,
    if it was taken with the current source (sha256 over the CUDA sources that
    define the kernel)."""
    h = hashlib.sha256()
    for f in source_files:
        with open(f, "rb") as fh:
            h.update(fh.read())
    sha = h.hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", f"{kernel_key}.md")
    if not os.path.exists(path):
        return None, sha
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    s = re.search(r"source_sha256_16:\s*([0-9a-f]+)", txt)
    if m and s and s.group(1) == sha:
        return float(m.group(1)), sha
    return None, sha


# ---------------------------------------------------------------- oracle timing
# The oracle (numpy, FP64) is far too slow for the full 3D depth-5 workload
# (about two minutes and 3 GB per cycle on one core), so its timings run the
# depth-4 instance of the same workload (k = 8 pi, 10% layer, centred
# Gaussian; 512,000 interior unknowns) and report DoF-updates/s.
ORACLE_CYCLE_S = {5: 115.0, 4: 3.4, 3: 0.13}   # one host core, per cycle


def _oracle_problem(depth):
    import oracle as O
    cfg = W.config3(depth)
    o = O.Hierarchy(cfg["d"], depth, cfg["k2"], cfg["theta"], cfg["layer_width"])
    o.set_rhs_nodal(cfg["f"])
    return O, o


def _oracle_cycles(depth, ncycles, budget_s):
    """Oracle cycles (BPX, omega = 0.6) on one core: (cycles done, seconds)."""
    O, o = _oracle_problem(depth)
    omega = np.full(depth, 0.6)
    done, t0 = 0, time.perf_counter()
    while done < ncycles:
        o.cycle(omega, O.ADD, O.HIERARCHICAL)
        done += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    return done, time.perf_counter() - t0


_WORKER = {}


def _oracle_worker_init(depth):
    _WORKER["p"] = _oracle_problem(depth)
    _WORKER["depth"] = depth


def _oracle_worker_cycles(ncycles):
    O, o = _WORKER["p"]
    omega = np.full(_WORKER["depth"], 0.6)
    t0 = time.perf_counter()
    for _ in range(ncycles):
        o.cycle(omega, O.ADD, O.HIERARCHICAL)
    return ncycles, time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _oracle_pool(depth, cores):
    """One oracle process per host core (spawned: no CUDA state is
    inherited), each holding its own copy of the problem."""
    import multiprocessing as mp
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    return mp.get_context("spawn").Pool(cores, initializer=_oracle_worker_init, initargs=(depth,))


def cpu_baseline_line(budget_s=12.0, depth=4):
    """The oracle on the host: one core (about budget_s of cycles) and every
    core of the process's affinity mask (one independent copy of the problem
    per core, cycles timed in parallel; throughput = all cycles / the slowest
    copy's time)."""
    units = (3 ** depth - 1) ** 3
    done1, dt1 = _oracle_cycles(depth, 1000, budget_s)
    single = units * done1 / dt1
    cores = host_cores()
    per = max(1, int(budget_s / max(dt1 / done1, 1e-3)))
    with _oracle_pool(depth, cores) as pool:
        pool.map(_oracle_worker_cycles, [0] * cores)        # set-up done in every worker
        res = pool.map(_oracle_worker_cycles, [per] * cores)
    dt_all = max(r[1] for r in res)
    allc = units * sum(r[0] for r in res) / dt_all
    return {"value": allc, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"BPX cycles (omega 0.6) of the depth-4 instance of the 3D workload ({units} "
                      f"interior unknowns): {per} per core on {cores} cores in {dt_all:.1f} s "
                      f"(one copy per core); one core alone: {done1} cycles in {dt1:.1f} s",
            "single_core": {"value": single, "cores": 1}}


def run_reference(args, rank):
    """The oracle as the reference arm: each step runs one cycle on every
    host core (one copy of the problem per core), on the deepest instance
    of the 3D workload whose steps fit in about two and a half minutes."""
    if rank != 0:
        return
    depth = 3
    for dd in (4, 3):
        depth = dd
        if (args.steps + args.warmup) * ORACLE_CYCLE_S[dd] * 1.3 <= 150:
            break
    cores = host_cores()
    units = (3 ** depth - 1) ** 3
    with _oracle_pool(depth, cores) as pool:
        pool.map(_oracle_worker_cycles, [0] * cores)
        for _ in range(args.warmup):
            pool.map(_oracle_worker_cycles, [1] * cores)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.map(_oracle_worker_cycles, [1] * cores)
        dt = time.perf_counter() - t0
    val = units * cores * args.steps / dt
    sample = (f"one FP64 oracle BPX cycle per step on each of {cores} host cores (one copy each) on the "
              f"depth-{depth} instance of the 3D workload ({units} interior unknowns)")
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128 (f64)", "data": "synthetic",
            "impl": "reference", "config": workload_config(1),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- replicas
def max_over_ranks(dist, x, device):
    """The largest x over all ranks (x itself without a process group); the
    slowest replica sets the whole job's time."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_step, steps, world, max_ms):
    """Units all replicas processed divided by the slowest replica's time."""
    return units_per_step * steps * world / (max_ms / 1e3)


def workload_config(world):
    return {"workload": "3D complex128 cycle: depth 5 (243^3 cells, 14,172,488 interior unknowns), "
                        "k=8pi, 10% ECS layer theta=pi/6, centred Gaussian width 0.05; step = one BPX "
                        "additive FAS cycle, omega=0.6 on every level",
            "l2": "inputs larger than L2 (232 MB per fine array); L2 also flushed before every timed step",
            "parallelism": "replicas" if world > 1 else "single GPU"}


# ---------------------------------------------------------------- other forms
# complex64 cycles per FP64 outer step of the refinement and batched forms
# (the best of 4, 8, 16, 32 for the 2D, 3D and batched definite problems on
# GB300: fewer FP64 outer residuals for about the same number of cycles)
INNER = 16


def _wall(torch, fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return r, time.perf_counter() - t0


def time_cycles(torch, s, variant, omega, transfer, steps, warmup, flush=None, clocks=None, dist=None):
    """Device time of `steps` cycles (CUDA events on the solver's stream
    around each cycle, L2 flushed before each), after `warmup` untimed ones.
    Returns (total ms, launches in the timed region, clock record)."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        s.cycle(variant, omega, transfer)
    torch.cuda.synchronize()
    s.get_stats()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
    for k in range(steps):
        if flush is not None:
            flush.fill_(float(k & 7))
        starts[k].record(stream)
        s.cycle(variant, omega, transfer)
        ends[k].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop() if clocks is not None else None
    launches, _, _ = s.get_stats()
    return sum(a.elapsed_time(b) for a, b in zip(starts, ends)), launches, clk


def fine_sweep_ms(torch, s, variant, omega, transfer, cycles, flush=None):
    """The finest-level sweep alone: the same cycles with an event pair
    around the fine sweep (instrumented pass; mean ms per sweep)."""
    s.set_timing(True)
    for _ in range(3):
        s.cycle(variant, omega, transfer)
    torch.cuda.synchronize()
    s.get_stats()
    for k in range(cycles):
        if flush is not None:
            flush.fill_(float(k & 7))
        s.cycle(variant, omega, transfer)
    _, nsweeps, ms = s.get_stats()
    s.set_timing(False)
    return ms / max(nsweeps, 1)


def form_cycle_2d(mg, torch, peaks, steps=500):
    """The 2D complex128 variant-sweep workload (depth 6, 529,984 interior
    unknowns, k = 20 pi, 10% layer, three Gaussians of seed 1): device time
    per BPX cycle (omega 0.6, L2 flushed before each), and the fine sweep
    against the FP64 roofline.  The level is L2-resident between cycles."""
    cfg = W.config2()
    d, depth = cfg["d"], cfg["depth"]
    s = mg.Solver(d, depth, cfg["k2"], cfg["theta"], cfg["layer_width"])
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    s.set_rhs(cfg["f"])
    omega = np.full(depth, 0.6)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    total, _, _ = time_cycles(torch, s, mg.MG_BPX, omega, mg.MG_HIERARCHICAL, steps, 20, flush)
    sweep = fine_sweep_ms(torch, s, mg.MG_BPX, omega, mg.MG_HIERARCHICAL, min(steps, 300), flush)
    s.close()
    flops, nbytes = fine_sweep_counts(d, depth, cfg["layer_width"], bpx=True, omega_real=True)
    interior = (3 ** depth - 1) ** d
    return {"ms_per_cycle": total / steps, "dof_updates_per_s": interior * steps / (total / 1e3),
            "fine_sweep_ms": sweep, "fine_sweep_fp64_tflops": flops / (sweep / 1e3) / 1e12,
            "fine_sweep_frac_of_fp64_peak": flops / (sweep / 1e3) / FP64_PEAK_FLOPS,
            "fine_sweep_hbm_frac": nbytes / (sweep / 1e3) / 1e9 / peaks.get("hbm_gbs", 6800.0)}


def form_configured_2d(mg, torch):
    """The configured indefinite 2D depth-6 problem from u = 0 (it diverges:
    interior theta = 0)."""
    c = W.config2()
    s = mg.Solver(2, 6, c["k2"], c["theta"], c["layer_width"])
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    s.set_rhs(c["f"])
    st, n, rel = s.solve(mg.MG_BPX, np.full(6, 0.6), mg.MG_HIERARCHICAL, 1e-8, 300)
    s.close()
    return {"status": mg.STATUS_NAMES[st], "cycles": n, "rel_res": rel}


def form_refine_2d(mg, torch):
    """Time to 1e-8 on the 2D depth-6 definite companion (k^2 -> -k^2):
    complex64 cycles in FP64 defect correction against plain complex128
    cycles."""
    c = W.definite(W.config2())
    om = mg.omega_scheme(mg.MG_OMEGA_EXP, 0.6, 6)
    s = mg.Solver(2, 6, c["k2"], c["theta"], c["layer_width"])
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    s.set_rhs(c["f"])
    s.set_precision(mg.MG_C64_REFINE, INNER)
    s.solve(mg.MG_ADD, om, mg.MG_DLINEAR, 1e-8, 4000)
    s.set_solution(np.zeros(s.shape, complex))
    (st, n, rel), dt = _wall(torch, lambda: s.solve(mg.MG_ADD, om, mg.MG_DLINEAR, 1e-8, 4000))
    a = {"c64_refine": {"status": mg.STATUS_NAMES[st], "inner_cycles": n, "inner_per_outer": INNER,
                        "rel_res": rel, "seconds": dt}}
    s.set_precision(mg.MG_C128, 4)
    s.set_solution(np.zeros(s.shape, complex))
    (st, n, rel), dt = _wall(torch, lambda: s.solve(mg.MG_ADD, om, mg.MG_DLINEAR, 1e-8, 300))
    a["c128_plain"] = {"status": mg.STATUS_NAMES[st], "cycles": n, "rel_res": rel, "seconds": dt,
                       "note": "stalls at the FAS fixed point shifted by the non-Galerkin layer edge"}
    s.close()
    return a


def form_refine_3d(mg, torch, peaks):
    """Time to 1e-8 on the 3D depth-5 definite companion: complex64 cycles in
    FP64 defect correction against plain complex128 cycles, with the
    complex64 fine sweep's HBM fraction from an event-timed pass."""
    c = W.definite(W.config3())
    om = mg.omega_scheme(mg.MG_OMEGA_EXP, 0.6, 5)
    s = mg.Solver(3, 5, c["k2"], c["theta"], c["layer_width"])
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    s.set_rhs(c["f"])
    s.set_precision(mg.MG_C64_REFINE, INNER)
    s.solve(mg.MG_ADD, om, mg.MG_DLINEAR, 1e-8, INNER)
    s.set_solution(np.zeros(s.shape, complex))
    (st, n, rel), dt = _wall(torch, lambda: s.solve(mg.MG_ADD, om, mg.MG_DLINEAR, 1e-8, 2000))
    s.set_solution(np.zeros(s.shape, complex))
    s.set_timing(True)
    s.get_stats()
    s.solve(mg.MG_ADD, om, mg.MG_DLINEAR, 1e-30, 2 * INNER)
    _, k, ms = s.get_stats()
    s.set_timing(False)
    nbytes = 3 * 8 * (3 ** 5 + 1) ** 3 + 3 * 8 * (3 ** 4 + 1) ** 3
    sweep_s = ms / max(k, 1) / 1e3
    cc = {"c64_refine": {"status": mg.STATUS_NAMES[st], "inner_cycles": n, "inner_per_outer": INNER,
                         "rel_res": rel, "seconds": dt, "fine_sweep_ms": sweep_s * 1e3,
                         "fine_sweep_hbm": {"achieved_gbs": nbytes / sweep_s / 1e9,
                                            "peak_gbs": peaks.get("hbm_gbs"),
                                            "frac": nbytes / sweep_s / 1e9 / peaks.get("hbm_gbs", 6800.0),
                                            "algorithmic_bytes": nbytes}}}
    s.set_precision(mg.MG_C128, 4)
    s.set_solution(np.zeros(s.shape, complex))
    (st, n, rel), dt = _wall(torch, lambda: s.solve(mg.MG_ADD, om, mg.MG_DLINEAR, 1e-8, 60))
    cc["c128_plain"] = {"status": mg.STATUS_NAMES[st], "cycles": n, "rel_res": rel, "seconds": dt,
                        "dof_updates_per_s": (3 ** 5 - 1) ** 3 * n / dt}
    s.close()
    return cc


def form_aligned_layer(mg, torch):
    """Time to 1e-8 where both arms converge: the definite companions of the
    2D depth-6 and 3D depth-5 workloads with the layer edge on coarse grid
    lines (width 1/3, so rediscretisation equals the Galerkin product on
    every level and the plain FAS cycle's fixed point is the discrete
    solution).  Arms: complex64 cycles inside FP64 defect correction (16 per
    outer step) and plain complex128 cycles, both additive with exponential
    damping (omega 0.6), from u = 0.  Seconds are host wall time around the
    synchronising solve; cycles are inner cycles for the refinement arm."""
    out = {}
    for name, cfg in (("2d_depth6", W.config2()), ("3d_depth5", W.config3())):
        c = W.definite(cfg)
        d, depth = c["d"], c["depth"]
        om = mg.omega_scheme(mg.MG_OMEGA_EXP, 0.6, depth)
        s = mg.Solver(d, depth, c["k2"], c["theta"], 1.0 / 3.0)
        s.set_stream(torch.cuda.current_stream().cuda_stream)
        s.set_rhs(c["f"])
        res = {}
        for arm, prec, cap in (("c64_refine", mg.MG_C64_REFINE, 4000), ("c128_plain", mg.MG_C128, 1000)):
            s.set_precision(prec, INNER)
            s.solve(mg.MG_ADD, om, mg.MG_DLINEAR, 1e-8, min(cap, 2 * INNER))  # warm-up (graphs)
            s.set_solution(np.zeros(s.shape, complex))
            (st, n, rel), dt = _wall(torch, lambda: s.solve(mg.MG_ADD, om, mg.MG_DLINEAR, 1e-8, cap))
            res[arm] = {"status": mg.STATUS_NAMES[st], "cycles": n, "rel_res": rel, "seconds": dt}
        res["speedup_c64_refine"] = res["c128_plain"]["seconds"] / res["c64_refine"]["seconds"]
        out[name] = res
        s.close()
    return out


def form_multichannel(mg, torch, cycles=20):
    """Coupled multichannel cycles (Section 7.5; the channel counts of its
    Table 4): c = 1, 2, 4, 8, 16 channels fused on one grid, 2D depth 6
    (p = 2) and 3D depth 4 (p = 3), 10% layer with theta = pi/6, a definite
    synthetic coupling matrix (channel shifts -(5 + 3 i)^2 on the diagonal,
    couplings 0.05 |phi| e^{-|i-j|} off it: the closer to the diagonal, the
    stronger, as Section 2 describes), a Gaussian rhs per channel.  Per run:
    device time per BPX cycle (CUDA events over `cycles` cycles) and
    unknown-updates/s (vertices x channels)."""
    rows = []
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for d, depth in ((2, 6), (3, 4)):
        n = 3 ** depth
        for c in (1, 2, 4, 8, 16):
            ph = -np.array([(5.0 + 3.0 * i) ** 2 for i in range(c)])
            Phi = np.diag(ph).astype(complex)
            for i in range(c):
                for j in range(c):
                    if i != j:
                        Phi[i, j] = 0.05 * math.sqrt(abs(ph[i] * ph[j])) * math.exp(-abs(i - j))
            g = mg.MultiChannel(d, depth, Phi, W.THETA, 0.1)
            g.set_stream(stream.cuda_stream)
            f = np.stack([W.gaussian(d, depth, (0.5,) * d, 0.05)] * c, axis=-1).astype(np.complex128)
            g.set_rhs(f)
            g.residual_norm()  # reference: the residual of u = 0
            om = np.full(depth, 0.6)
            for _ in range(3):
                g.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)
            torch.cuda.synchronize()
            ev[0].record(stream)
            for _ in range(cycles):
                g.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)
            ev[1].record(stream)
            torch.cuda.synchronize()
            ms = ev[0].elapsed_time(ev[1]) / cycles
            _, rel = g.residual_norm()
            rows.append({"p": d, "depth": depth, "channels": c, "ms_per_cycle": ms,
                         "unknown_updates_per_s": c * (n - 1) ** d / (ms / 1e3),
                         "rel_res_after_cycles": rel, "cycles_done": cycles + 3})
            g.close()
    return {"cycles": cycles, "variant": "BPX, omega 0.6", "runs": rows}


def form_batched(mg, torch):
    """256 problems of depth 4-6 (definite companions) in one persistent
    launch per outer step against the same problems one after another."""
    specs = W.config4_specs(256)
    probs = [W.definite(W.config4_problem(sp)) for sp in specs]
    bt = mg.Batch(probs)
    bt.set_stream(torch.cuda.current_stream().cuda_stream)
    for p, pr in enumerate(probs):
        bt.solvers[p].set_rhs(pr["f"])
    oms = [mg.omega_scheme(mg.MG_OMEGA_EXP, 0.6, pr["depth"]) for pr in probs]
    tc, bp, ms = bt.autotune(mg.MG_ADD, oms, mg.MG_DLINEAR, INNER)
    (st, cyc, rel), dt = _wall(torch, lambda: bt.solve(mg.MG_ADD, oms, mg.MG_DLINEAR, 1e-8, 400, INNER))
    unknowns = sum((3 ** pr["depth"] - 1) ** 2 for pr in probs)
    upd = sum((3 ** pr["depth"] - 1) ** 2 * cyc[p] for p, pr in enumerate(probs))
    # algorithmic bytes of one outer step per fine vertex: the FP64 residual
    # (u, b read, complex64 rhs written: 40 B), INNER complex64 cycles (U, b
    # read, U' written, ~12% more on the coarse levels: 27 B each) and the FP64
    # update (u, e read, u written: 40 B)
    outer_bytes = sum((3 ** pr["depth"] + 1) ** 2 for pr in probs) * (40 + 27 * INNER + 40)
    hbm_gbs = outer_bytes / (ms / 1e3) / 1e9
    bb = {"problems": 256, "fine_unknowns": unknowns,
          "autotuned": {"tile": tc, "blocks_per_sm": bp, "ms_per_outer_step": ms},
          "outer_step_hbm": {"algorithmic_bytes": outer_bytes, "achieved_gbs": hbm_gbs,
                             "frac": hbm_gbs / 6703.8},
          "batched": {"seconds": dt, "all_ok": all(x == mg.MG_OK for x in st), "max_rel_res": max(rel),
                      "dof_updates_per_s": upd / dt}}

    def seq():
        res = []
        for p in range(256):
            sv = bt.solvers[p]
            sv.set_solution(np.zeros(sv.shape, complex))
            sv.set_precision(mg.MG_C64_REFINE, INNER)
            res.append(sv.solve(mg.MG_ADD, oms[p], mg.MG_DLINEAR, 1e-8, 4000))
        return res
    r, dt2 = _wall(torch, seq)
    bb["sequential"] = {"seconds": dt2, "all_ok": all(x[0] == mg.MG_OK for x in r)}
    bt.close()
    return bb


def form_adjoint(mg, torch):
    """Forward and adjoint solves with the gradients of J (2D depth 6, the
    definite companion E = 0 of the adjoint workload, tolerance 1e-10)."""
    from paper_1508_03954_gb300.adjoint import SolveOptions, far_field
    c = W.config5()
    E = 0.0  # definite companion (k^2 = -V)
    s = mg.Solver(2, 6, E - c["V"], c["theta"], c["layer_width"])
    s.set_stream(torch.cuda.current_stream().cuda_stream)
    xyz, g = W.circle_samples(256)
    opts = SolveOptions(variant=mg.MG_ADD, transfer=mg.MG_DLINEAR, omega=mg.omega_scheme(mg.MG_OMEGA_EXP, 0.6, 6),
                        tol=1e-10, max_cycles=20000, precision=mg.MG_C64_REFINE, inner_cycles=INNER)
    V = torch.from_numpy(c["V"]).cuda().requires_grad_(True)
    f = torch.from_numpy(np.real(c["f"])).cuda().requires_grad_(True)

    def fwd_bwd():
        J = far_field(V, f, s, E, xyz, g, opts)
        J.backward()
        return J.item()
    fwd_bwd()
    V.grad = None
    f.grad = None
    Jv, dt = _wall(torch, fwd_bwd)
    s.close()
    return {"J": Jv, "seconds_forward_backward": dt, "tol": 1e-10}


def form_table(mg, torch, peaks):
    """Every secondary form by name (each printed on a line of its own)."""
    return {"cycle_2d_depth6": lambda: form_cycle_2d(mg, torch, peaks),
            "configured_2d_depth6": lambda: form_configured_2d(mg, torch),
            "time_to_1e-8_2d_depth6_definite": lambda: form_refine_2d(mg, torch),
            "time_to_1e-8_3d_depth5_definite": lambda: form_refine_3d(mg, torch, peaks),
            "time_to_1e-8_aligned_layer": lambda: form_aligned_layer(mg, torch),
            "batched_256_definite": lambda: form_batched(mg, torch),
            "multichannel": lambda: form_multichannel(mg, torch),
            "adjoint_2d_depth6": lambda: form_adjoint(mg, torch),
            "csg_sweep": lambda: csg_sweep(mg, torch),
            "channel_table2": lambda: channel_table2(mg, torch),
            "four_d": lambda: four_d(mg, torch, peaks),
            "dimension_study": lambda: dimension_study(mg, torch),
            "adaptive": lambda: adaptive(mg, torch),
            "adaptive_3d": lambda: adaptive(mg, torch, d=3, depth=5, cycles=30),
            "channel_table2_adaptive": lambda: channel_table2_adaptive(mg, torch)}


def run_forms(mg, torch, peaks, names, out_path=None):
    """Run the named forms, each guarded (an exception is recorded as its
    result), print each as one compact JSON line and optionally collect them
    in a file.  Returns {name: seconds}."""
    table = form_table(mg, torch, peaks)
    collected, secs = {}, {}
    for name in names:
        t0 = time.perf_counter()
        try:
            res = table[name]()
        except Exception as e:  # a failing form must not cost the headline line
            res = {"error": f"{type(e).__name__}: {e}"}
        secs[name] = round(time.perf_counter() - t0, 2)
        collected[name] = res
        print(json.dumps({"form": name, "result": res}, separators=(",", ":")), flush=True)
    if out_path:
        with open(out_path, "w") as fh:
            json.dump(collected, fh, indent=1)
    return secs


def csg_sweep(mg, torch, cycles=300):
    """The paper's complex-scaled-grid regime (Section 7.3): every cell rotated
    (layer width 0.5), Dirichlet boundary, omega = 0.8 on every level, kh = 5/9
    (k = 5, 15, 45, 135 on depths 2..5), rotation angles 0..45 degrees, the
    four variants; rhs a centred Gaussian of width 0.05, u0 = 0.  Per run: the
    cycles to a relative residual of 1e-8 (None if not reached), the relative
    residual after the run, and the mean reduction per cycle over cycles
    10 .. (1e-8 or the end)."""
    variants = {"add": (mg.MG_ADD, mg.MG_DLINEAR), "hb": (mg.MG_HB, mg.MG_DLINEAR),
                "bpx": (mg.MG_BPX, mg.MG_HIERARCHICAL), "hb-hier": (mg.MG_HB, mg.MG_HIERARCHICAL)}
    rows = []
    t0 = time.perf_counter()
    for k, depth in ((5, 2), (15, 3), (45, 4), (135, 5)):
        for deg in (0, 30, 35, 40, 45):
            k2 = W.constant_k2(2, depth, float(k * k))
            f = W.gaussian(2, depth, (0.5, 0.5), 0.05)
            s = mg.Solver(2, depth, k2, math.radians(deg), 0.5)
            s.set_rhs(f)
            om = np.full(depth, 0.8)
            for name, (v, t) in variants.items():
                s.set_solution(np.zeros(s.shape, complex))
                s.residual_norm()  # reference residual of u0
                hist, hit = [], None
                for c in range(cycles + 1):
                    s.cycle(v, om, t)
                    rel = s.last_cycle_norm()[1]  # residual of the iterate after c cycles
                    hist.append(rel)
                    if hit is None and rel <= 1e-8:
                        hit = c
                        break
                    if not np.isfinite(rel) or rel > 1e30:
                        break
                end = len(hist) - 1
                rate = float("nan")
                if end > 10 and hist[10] > 0 and np.isfinite(hist[end]):
                    rate = (hist[end] / hist[10]) ** (1.0 / (end - 10))
                rows.append({"k": k, "depth": depth, "theta_deg": deg, "variant": name,
                             "cycles_to_1e-8": hit, "rel_res": float(hist[-1]), "cycles_run": end,
                             "rate_per_cycle": float(rate)})
            s.close()
    return {"cycles_max": cycles, "omega": 0.8, "layer_width": 0.5, "seconds": time.perf_counter() - t0,
            "runs": rows}


def channel_table2(mg, torch, iters=50):
    """The channel problem of Section 7.4 on h = 1/81 (Table 2, regular
    grid): a 30 degree layer within 1/3 of the top and right faces, the
    interior rotated by theta, varying phi and the Gaussian source chi of
    Eq. 08-gaussian, u0 = 0, 50 iterations of pure Jacobi (two-phase factors
    at theta = 0, 0.4 otherwise), the additive transition scheme (0.4) and BPX
    (0.4).  Per run: the max-norm residual reduction and the device time per
    iteration (CUDA events around the 50 cycles)."""
    rows = []
    t0 = time.perf_counter()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for deg in (0, 18, 25, 35, 45):
        c = W.channel(deg)
        s = mg.Solver(2, c["depth"], c["k2"], c["theta"], c["layer_width"], c["theta_interior"])
        s.set_stream(torch.cuda.current_stream().cuda_stream)
        s.set_rhs(c["f"])
        for solver in ("jacobi", "transition", "bpx"):
            s.set_solution(np.zeros(s.shape, complex))
            r0 = s.residual_max()
            sched = []
            for it in range(1, iters + 1):
                if solver == "jacobi":
                    w = (W.CHANNEL_OMEGA1 if it % 2 else W.CHANNEL_OMEGA2) if deg == 0 else 0.4
                    sched.append((mg.omega_scheme(mg.MG_OMEGA_JACOBI, w, 4), mg.MG_ADD, mg.MG_DLINEAR))
                elif solver == "transition":
                    sched.append((mg.omega_scheme(mg.MG_OMEGA_TRANSITION, 0.4, 4, it), mg.MG_ADD, mg.MG_DLINEAR))
                else:
                    sched.append((mg.omega_scheme(mg.MG_OMEGA_UCG, 0.4, 4), mg.MG_ADD, mg.MG_HIERARCHICAL))
            torch.cuda.synchronize()
            ev[0].record()
            for om, v, t in sched:
                s.cycle(v, om, t)
            ev[1].record()
            torch.cuda.synchronize()
            red = s.residual_max() / r0
            rows.append({"theta_deg": deg, "solver": solver, "reduction_max_norm": float(red),
                         "diverged": bool(not red < 1.0), "us_per_iteration": ev[0].elapsed_time(ev[1]) * 1e3 / iters})
        s.close()
    return {"iterations": iters, "depth": 4, "seconds": time.perf_counter() - t0, "runs": rows}


def channel_table2_adaptive(mg, torch, iters=50, depth=7, min_level=3):
    """The channel problem of Section 7.4 on dynamically adaptive grids
    (Table 2, adaptive column): the solve starts on the regular grid of
    h = 1/27 (the coarsest level with h <= h_max = 0.1) and every iteration
    is one cycle followed by one step of feature-based refinement (Section
    5.3: 10% refined, 2% erased, 20 bins, veto 1e-2), cells down to
    h = 1/2187 (the first level below h_min = 0.001).  Solvers and factors
    as on the regular grid, looked up by succ(v).  The residual veto runs in
    both readings: absolute (|r / diag| > 1e-2) and relative to the vertex's
    value (|r / diag| > 1e-2 |u|).  Per run: max-norm residual reduction
    after 50 iterations against the start grid's initial residual,
    fine-grid vertices at the end, finest level reached, and the time per
    iteration (CUDA events: cycle, adaptation step with its host round
    trip, total)."""
    rows = []
    t0 = time.perf_counter()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for deg in (0, 18, 25, 35, 45):
        c = W.channel(deg, depth)
        ref = {lev: np.full((3 ** lev,) * 2, lev < min_level) for lev in range(1, depth)}
        for solver, relative in itertools.product(("jacobi", "transition", "bpx"), (False, True)):
            s = mg.Solver.adaptive(2, depth, c["k2"], c["theta"], c["layer_width"], ref, c["theta_interior"])
            s.set_stream(torch.cuda.current_stream().cuda_stream)
            s.set_rhs(c["f"])
            s.set_solution(np.zeros(s.shape, complex))
            r0 = s.residual_max()
            torch.cuda.synchronize()
            ev[0].record()
            st = (0, 0, 0, 0)
            diverged = False
            t_cycle = t_adapt = 0.0
            for it in range(1, iters + 1):
                ev[2].record()
                if solver == "jacobi":
                    w = (W.CHANNEL_OMEGA1 if it % 2 else W.CHANNEL_OMEGA2) if deg == 0 else 0.4
                    s.cycle(mg.MG_ADD, mg.omega_scheme(mg.MG_OMEGA_JACOBI, w, depth), mg.MG_DLINEAR)
                elif solver == "transition":
                    s.cycle(mg.MG_ADD, mg.omega_scheme(mg.MG_OMEGA_TRANSITION, 0.4, depth, it), mg.MG_DLINEAR)
                else:
                    s.cycle(mg.MG_ADD, mg.omega_scheme(mg.MG_OMEGA_UCG, 0.4, depth), mg.MG_HIERARCHICAL)
                ev[3].record()
                try:
                    st = s.adapt(min_level, 0.1, 0.02, 20, 1e-2, veto_relative=relative)
                except mg.MgError:
                    diverged = True  # non-finite indicator: the grid stays
                ev[1].record()
                torch.cuda.synchronize()
                t_cycle += ev[2].elapsed_time(ev[3])
                t_adapt += ev[3].elapsed_time(ev[1])
            red = s.residual_max() / r0
            rows.append({"theta_deg": deg, "solver": solver, "veto": "relative" if relative else "absolute",
                         "reduction_max_norm": float(red), "diverged": bool(diverged or not red < 1.0),
                         "fine_vertices": st[2], "finest_level": st[3],
                         "ms_per_iteration": ev[0].elapsed_time(ev[1]) / iters,
                         "ms_cycle": t_cycle / iters, "ms_adapt": t_adapt / iters})
            s.close()
    return {"iterations": iters, "depth": depth, "min_level": min_level, "seconds": time.perf_counter() - t0,
            "runs": rows}


def poisson_rhs(d, depth):
    """Section 7.1: f = d pi^2 prod_i sin(pi x_i) (phi = 0, theta = 0)."""
    n = 3 ** depth
    s1 = np.sin(math.pi * np.arange(n + 1) / n)
    s = np.ones((1,) * d)
    for ax in range(d):
        shape = [1] * d
        shape[ax] = n + 1
        s = s * s1.reshape(shape)
    return (d * math.pi ** 2 * s).astype(np.complex128)


def four_d(mg, torch, peaks, depth=4, cycles=50):
    """The four-dimensional path at depth 4 (82^4 vertices, 80^4 unknowns):
    device time per additive cycle (exponential damping, omega = 0.8, one
    CUDA graph per cycle) and the fine operator's ten-pass chain timed alone
    with events (instrumented pass).  The chain moves 384 B per vertex
    (7 passes read 1 and write 1 array, 2 read 2, the last reads 3), the
    operator's own operands are 48 B (u, b read, r written).  It is bound by
    FP64 issue: with real rows (Poisson, no layer) a pass is 3 real x complex
    taps (10 flops), plus 3 complex adds of partial sums and the subtraction
    from b: 108 FP64 flops per vertex."""
    d = 4
    s = mg.Solver(d, depth, W.constant_k2(d, depth, 0.0), 0.0, 0.0)
    stream = torch.cuda.current_stream()
    s.set_stream(stream.cuda_stream)
    s.set_rhs(poisson_rhs(d, depth))
    om = mg.omega_scheme(mg.MG_OMEGA_EXP, 0.8, depth)
    for _ in range(3):
        s.cycle(mg.MG_ADD, om, mg.MG_DLINEAR)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(cycles):
        s.cycle(mg.MG_ADD, om, mg.MG_DLINEAR)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / cycles
    s.get_stats()
    s.set_timing(True)
    for _ in range(10):
        s.cycle(mg.MG_ADD, om, mg.MG_DLINEAR)
    _, nfine, fine_ms = s.get_stats()
    s.set_timing(False)
    apply_ms = fine_ms / max(nfine, 1)
    nv = (3 ** depth + 1) ** d
    interior = (3 ** depth - 1) ** d
    chain_gbs = 384.0 * nv / (apply_ms / 1e3) / 1e9
    # time to 1e-8 from u = 0: complex128 cycles against complex64 cycles in
    # FP64 defect correction (16 per outer step)
    solves = {}
    for name, prec in (("c128", mg.MG_C128), ("c64_refine", mg.MG_C64_REFINE)):
        s.set_precision(prec, 16)
        s.set_solution(torch.zeros(s.nv, dtype=torch.complex128, device="cuda"))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, n, rel_end = s.solve(mg.MG_ADD, om, mg.MG_DLINEAR, 1e-8, 2000)
        torch.cuda.synchronize()
        solves[name] = {"status": mg.STATUS_NAMES[st], "cycles": n, "rel_res": rel_end,
                        "seconds": time.perf_counter() - t0}
    s.close()
    flops = 108.0 * nv
    return {"depth": depth, "vertices": nv, "ms_per_cycle": ms, "dof_updates_per_s": interior / (ms / 1e3),
            "time_to_1e-8": solves,
            "fine_apply_ms": apply_ms, "fine_apply_fp64_tflops": flops / (apply_ms / 1e3) / 1e12,
            "fine_apply_frac_of_fp64_peak": flops / (apply_ms / 1e3) / FP64_PEAK_FLOPS,
            "fine_apply_chain_gbs": chain_gbs,
            "fine_apply_chain_frac_of_hbm": chain_gbs / peaks.get("hbm_gbs", 6800.0),
            "fine_apply_operand_gbs": 48.0 * nv / (apply_ms / 1e3) / 1e9}


def dimension_study(mg, torch, cycles=300):
    """Regular-grid counterpart of the dimension study of Section 7.1: the
    Poisson problem (phi = 0, theta = 0, f = d pi^2 prod sin(pi x_i), u0 = 0)
    for p = 2, 3, 4 on every depth up to the largest of each dimension,
    additive multigrid with exponential damping, the transition scheme and
    undamped coarse grid corrections for omega = 0.6, 0.8, 1.0.  Per run:
    cycles to a relative residual of 1e-8 (None if not within the limit or
    diverged) and the mean reduction per cycle from cycle 5 on."""
    rows = []
    t0 = time.perf_counter()
    depths = {2: (2, 3, 4, 5, 6), 3: (2, 3, 4, 5), 4: (2, 3, 4)}
    schemes = {"exp": mg.MG_OMEGA_EXP, "transition": mg.MG_OMEGA_TRANSITION, "ucg": mg.MG_OMEGA_UCG}
    for d, ds in depths.items():
        for depth in ds:
            s = mg.Solver(d, depth, W.constant_k2(d, depth, 0.0), 0.0, 0.0)
            s.set_rhs(poisson_rhs(d, depth))
            for name, sch in schemes.items():
                for w in (0.6, 0.8, 1.0):
                    s.set_solution(np.zeros(s.shape, complex))
                    s.residual_norm()
                    hist, hit = [], None
                    for k in range(1, cycles + 2):
                        s.cycle(mg.MG_ADD, mg.omega_scheme(sch, w, depth, k), mg.MG_DLINEAR)
                        rel = s.last_cycle_norm()[1]  # residual after k - 1 cycles
                        hist.append(rel)
                        if rel <= 1e-8:
                            hit = k - 1
                            break
                        if not np.isfinite(rel) or rel > 1e6:
                            break
                    end = len(hist) - 1
                    rate = float("nan")
                    if end > 5 and hist[5] > 0 and np.isfinite(hist[end]):
                        rate = (hist[end] / hist[5]) ** (1.0 / (end - 5))
                    rows.append({"p": d, "depth": depth, "scheme": name, "omega": w, "cycles_to_1e-8": hit,
                                 "rel_res": float(hist[-1]), "rate_per_cycle": float(rate)})
            s.close()
    return {"cycles_max": cycles, "variant": "add, d-linear", "seconds": time.perf_counter() - t0, "runs": rows}


def adaptive(mg, torch, d=2, depth=6, cycles=100):
    """Adaptive spacetree against the regular grid of the same finest depth
    (2D depth 6, h_min = 1/729; 3D depth 5, h_min = 1/243): a definite
    problem (k^2 = -(15 pi)^2, no layer) with the localised source
    exp(-sum (125 x_a)^2) of Eq. 08-gaussian at the origin; the adaptive grid
    refines level-l cells whose centre lies within 0.7 * 0.7^(l-1) of the
    origin (2D: 2.5% of the regular unknowns).  BPX with undamped factors
    0.6.  Per grid: fine-grid unknowns, device time per cycle (CUDA events
    around `cycles` cycles), cycles and seconds to 1e-8, and the adaptive
    solution's largest deviation from the regular one at the vertices of
    the finest adaptive level."""
    n = 3 ** depth
    x = np.arange(n + 1) / n
    r2 = np.zeros((n + 1,) * d)
    for ax in range(d):
        shape = [1] * d
        shape[ax] = n + 1
        r2 = r2 + (125.0 * x.reshape(shape)) ** 2
    f = np.exp(-r2).astype(np.complex128)
    k2 = W.constant_k2(d, depth, -(15 * math.pi) ** 2)
    ref = W.source_refinement(d, depth)
    om = mg.omega_scheme(mg.MG_OMEGA_UCG, 0.6, depth)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    out, sols = {}, {}
    for name in ("regular", "adaptive"):
        s = mg.Solver.adaptive(d, depth, k2, 0.0, 0.0, ref) if name == "adaptive" else mg.Solver(d, depth, k2, 0.0, 0.0)
        s.set_stream(stream.cuda_stream)
        s.set_rhs(f)
        for _ in range(3):
            s.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(cycles):
            s.cycle(mg.MG_BPX, om, mg.MG_HIERARCHICAL)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / cycles
        s.set_solution(np.zeros(s.shape, complex))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, nc, rel = s.solve(mg.MG_BPX, om, mg.MG_HIERARCHICAL, 1e-8, 3000)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        sols[name] = s.get_solution()
        out[name] = {"ms_per_cycle": ms, "status": mg.STATUS_NAMES[st], "cycles_to_1e-8": nc, "rel_res": rel,
                     "seconds_to_1e-8": sec}
        s.close()
    # grid structure from the flags: cells of level l + 1 are the children of
    # refined level-l cells; a vertex carries an unknown when its 2^d cells exist
    cells = np.ones((3,) * d, dtype=bool)
    unknown, exists = {}, {}
    for lev in range(1, depth + 1):
        m = 3 ** lev
        cnt = np.zeros((m + 1,) * d, dtype=int)
        for corner in itertools.product((0, 1), repeat=d):
            cnt[tuple(slice(o, o + m) for o in corner)] += cells
        inner = np.zeros_like(cnt, dtype=bool)
        inner[(slice(1, -1),) * d] = True
        unknown[lev], exists[lev] = inner & (cnt == 2 ** d), cnt > 0
        if lev < depth:
            cells = cells & ref[lev]
            for ax in range(d):
                cells = np.repeat(cells, 3, axis=ax)
    own = sum(int((unknown[lev] & ~unknown[lev + 1][(slice(None, None, 3),) * d]).sum()) for lev in range(1, depth))
    own += int(unknown[depth].sum())
    out["adaptive"]["fine_unknowns"] = own
    out["regular"]["fine_unknowns"] = (n - 1) ** d
    for name in out:
        out[name]["dof_updates_per_s"] = out[name]["fine_unknowns"] / (out[name]["ms_per_cycle"] / 1e3)
    m = exists[depth]
    dev = np.abs(sols["adaptive"][m] - sols["regular"][m]).max() / np.abs(sols["regular"]).max()
    out["max_deviation_on_finest_region"] = float(dev)
    return out


# ---------------------------------------------------------------- main
FORMS_DEFAULT = ("cycle_2d_depth6", "configured_2d_depth6", "time_to_1e-8_2d_depth6_definite",
                 "time_to_1e-8_3d_depth5_definite", "time_to_1e-8_aligned_layer", "batched_256_definite",
                 "adjoint_2d_depth6", "multichannel",
                 "csg_sweep", "channel_table2", "four_d", "adaptive", "adaptive_3d")


def profile_sequence(mg, torch, which):
    """A short fixed launch sequence for ncu (no timing, no output but a
    status line)."""
    if which == "cycle3d":
        c = W.config3()
        s = mg.Solver(3, 5, c["k2"], c["theta"], c["layer_width"])
        s.set_rhs(c["f"])
        for _ in range(3):
            s.cycle(mg.MG_BPX, np.full(5, 0.6), mg.MG_HIERARCHICAL)
    elif which == "refine3d":
        c = W.definite(W.config3())
        s = mg.Solver(3, 5, c["k2"], c["theta"], c["layer_width"])
        s.set_rhs(c["f"])
        s.set_precision(mg.MG_C64_REFINE, INNER)
        s.solve(mg.MG_ADD, mg.omega_scheme(mg.MG_OMEGA_EXP, 0.6, 5), mg.MG_DLINEAR, 1e-30, INNER)
    else:
        # 2D depth 8 (6561^2 cells, 43 M vertices), definite k^2 = -(20 pi)^2,
        # 10% layer, one Gaussian source
        depth = 8
        s = mg.Solver(2, depth, W.constant_k2(2, depth, -(20 * math.pi) ** 2), W.THETA, 0.1)
        s.set_rhs(W.gaussian(2, depth, (0.45, 0.55), 0.05))
        s.set_precision(mg.MG_C64_REFINE, INNER)
        s.solve(mg.MG_ADD, mg.omega_scheme(mg.MG_OMEGA_EXP, 0.6, depth), mg.MG_DLINEAR, 1e-30, INNER)
    torch.cuda.synchronize()
    print(json.dumps({"profile": which, "ok": True}), flush=True)
    s.close()


def headline_line(value, steps, warmup, total_ms, world, roofline, e2e, launches, clk, cpu=None):
    """The one JSON line the run ends with (compact: a few hundred bytes of
    numbers; every secondary form goes on a line of its own before it)."""
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128 (f64)", "data": "synthetic",
            "config": workload_config(world), "roofline": roofline, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--forms", default=",".join(FORMS_DEFAULT),
                    help="comma-separated secondary forms to run after the headline")
    ap.add_argument("--forms-out", default=None, help="also write the forms' results to this JSON file")
    ap.add_argument("--form", choices=sorted(form_table(None, None, {}).keys()), default=None,
                    help="run only this form and print its result (profiling)")
    ap.add_argument("--four-d-depth", type=int, default=4, help="depth of the four_d form (profiling)")
    ap.add_argument("--profile", choices=["cycle3d", "refine3d", "refine2d8"], default=None,
                    help="run a short fixed sequence for a profiler and exit: cycle3d = three complex128 "
                         "BPX cycles of the headline workload, refine3d = one outer step (16 complex64 "
                         "cycles) of the 3D depth-5 refinement form, refine2d8 = one outer step of the "
                         "2D depth-8 refinement form (the fine level's strips take two columns per lane)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local_rank)

    from paper_1508_03954_gb300 import build as B
    from paper_1508_03954_gb300 import mg
    B.build()
    mg.load()
    peaks, peak_src = measured_peaks()
    if args.profile is not None:
        profile_sequence(mg, torch, args.profile)
        return
    if args.form is not None:
        if args.form == "four_d":
            res = four_d(mg, torch, peaks, depth=args.four_d_depth)
        else:
            res = form_table(mg, torch, peaks)[args.form]()
        print(json.dumps({"form": args.form, "result": res}), flush=True)
        return

    # headline: the 3D complex128 cycle (depth 5), one BPX cycle per step
    cfg = W.config3()
    d, depth = cfg["d"], cfg["depth"]
    s = mg.Solver(d, depth, cfg["k2"], cfg["theta"], cfg["layer_width"])
    stream = torch.cuda.current_stream()
    s.set_stream(stream.cuda_stream)
    s.set_rhs(torch.from_numpy(cfg["f"]).cuda())
    omega = np.full(depth, 0.6)
    variant, transfer = mg.MG_BPX, mg.MG_HIERARCHICAL
    interior = (3 ** depth - 1) ** d
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    total_ms, launches, clk = time_cycles(torch, s, variant, omega, transfer, args.steps, args.warmup,
                                          flush, ClockSampler(local_rank), dist)
    total_ms = max_over_ranks(dist, total_ms, "cuda")
    value = whole_job_rate(interior, args.steps, world, total_ms)

    # the dominant kernel alone: event pair around the fine sweep (separate pass)
    sweep = fine_sweep_ms(torch, s, variant, omega, transfer, min(max(args.steps, 10), 100), flush)

    # end to end through the public API with page-locked host buffers
    u_h = torch.zeros(s.shape, dtype=torch.complex128).pin_memory()
    f_h = torch.from_numpy(cfg["f"]).pin_memory()
    out_h = torch.empty(s.shape, dtype=torch.complex128).pin_memory()
    s.set_solution(u_h)
    e2e_ms = 0.0
    ne = max(1, args.e2e_steps)
    for k in range(ne + 3):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.set_solution(u_h)
        s.set_rhs(f_h)
        s.cycle(variant, omega, transfer)
        s.get_solution(out_h)
        b.record(stream)
        b.synchronize()
        if k >= 3:
            e2e_ms += a.elapsed_time(b)
    e2e_value = whole_job_rate(interior, ne, world, max_over_ranks(dist, e2e_ms, "cuda"))
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * 16 * s.nv,
           "d2h_bytes_per_step": 16 * s.nv,
           "what": "mg_set_solution + mg_set_rhs from pinned host, mg_cycle, mg_get_solution to pinned host"}
    s.close()

    roofline = fine_sweep3_roofline(cfg, sweep, peaks, peak_src)
    if rank == 0 and world == 1 and not args.no_forms:
        names = [x for x in args.forms.split(",") if x]
        run_forms(mg, torch, peaks, names, args.forms_out)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline_line()
        except Exception as e:
            cpu = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0:
        line = headline_line(value, args.steps, args.warmup, total_ms, world, roofline, e2e, launches, clk, cpu)
        print(json.dumps(line, separators=(",", ":")), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
