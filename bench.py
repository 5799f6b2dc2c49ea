"""Benchmark of the DG right-hand side / SSP-RK3 step on GB300.

Metric: DOF-updates/s = nodes x 7 fields x 3 right-hand-side evaluations per
SSP-RK3 step / time.  One bench "step" is one SSP-RK3 step of the whole hot
path on the 2D periodic drop workload (64 x 64 quadrilaterals, p = 3, water
drop R = 0.15 in air at a seeded centre, u = (1, 0.5), P = 1e5, eps = 0.75 h),
with the state resident in HBM.  L2 (129 MB) is flushed between timed steps by
writing a 512 MB buffer, because the state (3.7 MB) would otherwise stay in L2.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--precision fp64]
Under torchrun each rank advances its own independent replica (weak scaling,
no collective on the data path).  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DG RHS DOF-updates/s (fp32-bulk vs fp64 at stated L2 err); adjoint/forward time"
UNIT = "DOF-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32bulk", choices=["fp32bulk", "fp64"])
    ap.add_argument("--accuracy-steps", type=int, default=500,
                    help="steps of the FP32-bulk vs FP64 accuracy comparison (the workload's 500)")
    ap.add_argument("--batch-steps", type=int, default=10,
                    help="timed steps of the batched ensemble (0 skips the batched block)")
    ap.add_argument("--rt-steps", type=int, default=10,
                    help="timed steps of the 256 x 256, p = 4 Rayleigh-Taylor block (0 skips it)")
    ap.add_argument("--rt-accuracy-steps", type=int, default=2000,
                    help="steps of the Rayleigh-Taylor FP32-bulk vs FP64 accuracy run (the workload's 2000)")
    ap.add_argument("--batch-accuracy-steps", type=int, default=200,
                    help="steps of the batched accuracy run (the ensemble's 200; sampled problems vs FP64)")
    ap.add_argument("--batch-problems", type=int, default=256,
                    help="ensemble size of the batched block (smaller values for profiling)")
    ap.add_argument("--adjoint-n", type=int, default=128,
                    help="elements per direction of the adjoint block (smaller values for profiling)")
    ap.add_argument("--kin-steps", type=int, default=200,
                    help="timed RK4 steps of the kinematic Rider-Kothe block (0 skips it)")
    ap.add_argument("--reinit-iters", type=int, default=50,
                    help="pseudo-time steps of the timed re-initialisation block (0 skips it)")
    ap.add_argument("--rt-paper-steps", type=int, default=10,
                    help="timed steps on the paper's Rayleigh-Taylor domain with the pressure top (0 skips)")
    ap.add_argument("--rb-steps", type=int, default=100,
                    help="timed steps of the rising-bubble block (20 x 40 quads, p = 4; 0 skips it)")
    ap.add_argument("--slab-steps", type=int, default=1000,
                    help="steps of the 1D slab block (0 skips it)")
    ap.add_argument("--tri-steps", type=int, default=200,
                    help="timed RK4 steps of the kinematic block on triangles (0 skips it)")
    ap.add_argument("--tri-n", type=int, default=64,
                    help="cells per direction of the timed triangle block (smaller values for profiling)")
    ap.add_argument("--adjoint-steps", type=int, default=200,
                    help="trajectory length of the adjoint timing (0 skips it)")
    ap.add_argument("--cpu-sample-steps", type=int, default=0,
                    help="oracle steps for the cpu_baseline leg (0 = size for ~15 s)")
    return ap.parse_args()


def workload(seed: int):
    from paper_2306_05002_gb300 import workloads as W
    return W.drop_2d(n=64, p=3, seed=seed)


def config_of(wl, extra=None):
    c = {"workload": f"2D periodic drop advection {wl.nx}x{wl.ny} quads p={wl.p} (water drop R=0.15 in air, "
                     f"u=(1,0.5), P=1e5, eps=0.75h, Gamma=|u|, SSP-RK3)",
         "elements": wl.E, "p": wl.p, "nodes": wl.N, "dof_per_rhs": 7 * wl.N,
         "dof_paper_convention": wl.N,  # nodes per scalar field, as the paper counts (Sec. 4.1)
         "dt": wl.dt,
         "l2": "flushed between timed steps (512 MB write)"}
    if extra:
        c.update(extra)
    return c


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout: float = 10.0):
        """Wait for the first sample (the first nvidia-smi on a freshly started box takes a while to
        start), so that the samples cover the timed region."""
        t0 = time.perf_counter()
        while self.proc and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.05)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[2:]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# Spin cycles of the gate kernel ahead of each timed step (~19 ms at 2.07 GHz): longer than the
# host takes to enqueue the flush, the events and the step even in the first process on a fresh
# box (~5 ms per step there), so the GPU never waits for the host inside the event interval.
GATE_CYCLES = 40_000_000


# --------------------------------------------------------------------------- roofline helpers

KERNEL_SOURCES = {"fp64": ["paper_2306_05002_gb300/csrc/dg_kernels_fp64.cuh",
                           "paper_2306_05002_gb300/csrc/dg_common.cuh"],
                  "fp32bulk": ["paper_2306_05002_gb300/csrc/dg_kernels_fp32.cuh",
                               "paper_2306_05002_gb300/csrc/dg_kernels_fp64.cuh",
                               "paper_2306_05002_gb300/csrc/dg_common.cuh",
                               "paper_2306_05002_gb300/csrc/dg_pdl.cuh"]}


def kernel_source_hash(precision="fp64"):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[precision]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, wl_name: str, precision: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{wl_name}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"source_hash:\s*([0-9a-f]+)", txt)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m or not t or m.group(1) != kernel_source_hash(precision):
        return None
    return float(t.group(1))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# FP64 FMA peak: measured on the GPU by the library's FMA-chain probe (dg_peak_flops) at the start
# of the run; before that (or if the probe fails), the figure from unit counts and clock:
# 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz.
FP64_PEAK_DERIVED = 152 * 2 * 2 * 2.07e9 / 1e12
MEASURED_PIPES = {}


def fp64_peak():
    return MEASURED_PIPES.get("fp64_tflops", FP64_PEAK_DERIVED)


def fp64_peak_source():
    if "fp64_tflops" in MEASURED_PIPES:
        return "measured: dg_peak_flops FP64 FMA chains on this GPU (every resident thread, 8 chains), of measured"
    return "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (ncu: 2 DFMA/clk/SM)"


def measure_pipes(dg):
    """FP64 and FP32 FMA rates of this GPU (best of three probe runs each)."""
    try:
        MEASURED_PIPES["fp64_tflops"] = max(dg.peak_flops("fp64") for _ in range(3))
        MEASURED_PIPES["fp32_tflops"] = max(dg.peak_flops("fp32") for _ in range(3))
    except Exception as exc:  # report the derived figure instead
        MEASURED_PIPES["error"] = str(exc)[:200]


# Per-unit algorithmic figures.  FP32-bulk (HBM-bound): 168 B per node and RK stage -- read the
# stage state and w^n, write the new stage, 7 FP64 words each -- i.e. 24 B per DOF-update; the fused
# stage kernel completes one stage per launch, so its units are the nodes.  FP64 (FP64-pipe-bound):
# the library's per-kernel flop counts (dg_kernel_costs, from the scheme's formulas).
BYTES_PER_NODE_STAGE = 168


NAMES = {"fp64": ["k_volume", "k_surface"],
         "fp32bulk": ["k_volume32", "k_surface32", "k_surfvol32", "k_volume32(fp64 state in)",
                      "k_surface32(fp64 state out)"]}


def roofline(precision, names, kms, flops, bytes_, nodes):
    # FP64 runs a volume and a surface kernel per stage (the dominant one is the roofline kernel);
    # a single-step FP32-bulk call runs the first-stage volume kernel (FP64 state in), two fused
    # stage kernels and the last-stage surface kernel (FP64 state out): the roofline kernel is the
    # fused one, which completes a whole stage per launch
    per_step = [3, 3] if precision == "fp64" else [0, 0, 2, 1, 1]
    n = min(len(kms), len(per_step), len(names))
    names, kms, flops, bytes_ = names[:n], kms[:n], flops[:n], bytes_[:n]
    dom = max(range(n), key=lambda i: kms[i] * per_step[i])
    if precision == "fp64":
        ach = flops[dom] / (kms[dom] * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": names[dom], "achieved": ach, "peak": fp64_peak(),
                "unit": "TFLOP/s", "frac": ach / fp64_peak(),
                "per_unit": "dg_kernel_costs flops per launch", "peak_source": fp64_peak_source()}
    else:
        dom = names.index("k_surfvol32")
        hbm = peaks().get("hbm_gbs", 6800.0)
        ach = BYTES_PER_NODE_STAGE * nodes / (kms[dom] * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": names[dom], "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "per_unit": f"{BYTES_PER_NODE_STAGE} B per node and stage x {nodes} nodes",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy), of measured"}
    roof.update({"kernel_ms": dict(zip(names, kms)), "launches_per_step": dict(zip(names, per_step)),
                 "kernel_flops_per_launch": dict(zip(names, flops)),
                 "kernel_bytes_per_launch": dict(zip(names, bytes_))})
    return roof


# --------------------------------------------------------------------------- ranks

def reduce_max(values, device):
    """Element-wise maximum over all ranks (a no-op without torch.distributed)."""
    import torch
    import torch.distributed as tdist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if tdist.is_available() and tdist.is_initialized() and tdist.get_world_size() > 1:
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return t.tolist()


def weak_scaling_value(units_per_rank: float, steps: int, world: int, ms_max: float) -> float:
    """Whole-job throughput: every rank advances its own replica; the slowest rank sets the time."""
    return units_per_rank * steps * world / (ms_max * 1e-3)


# --------------------------------------------------------------------------- oracle leg

def oracle_rate(wl, steps: int, threads: int = 0):
    import oracle
    pb = oracle.Problem(**wl.problem_kwargs())
    t0 = time.perf_counter()
    oracle.rk3(pb, wl.w, wl.dt, steps, threads=threads)
    dt = time.perf_counter() - t0
    return 7 * wl.N * 3 * steps / dt, dt


def oracle_sample(single, omp, omp_steps: int = 1, of: str = ""):
    """The oracle on a bounded sample of a large workload, as DOF-updates/s: one right-hand side
    of each problem in `single` on one core, and `omp_steps` SSP-RK3 steps of each problem in
    `omp` on every host core (the OpenMP build; bit-identical results).  `of` names the sample."""
    import oracle
    oracle.lib()  # built (or loaded) before any timing
    units = secs = 0.0
    for wl in single:
        pb = oracle.Problem(**wl.problem_kwargs())
        t0 = time.perf_counter()
        oracle.rhs(pb, wl.w)
        secs += time.perf_counter() - t0
        units += 7 * wl.N
    out = {"single_core": {"value": units / secs, "unit": UNIT, "cores": 1,
                           "sample": f"one right-hand side of {of or 'each problem'} ({secs:.1f} s)"}}
    try:
        cores = oracle.lib(openmp=True).orc_threads(os.cpu_count() or 1)
        units = secs = 0.0
        for wl in omp:
            pb = oracle.Problem(**wl.problem_kwargs())
            t0 = time.perf_counter()
            oracle.rk3(pb, wl.w, wl.dt, omp_steps, threads=cores)
            secs += time.perf_counter() - t0
            units += 7 * wl.N * 3 * omp_steps
        out["openmp"] = {"value": units / secs, "unit": UNIT, "cores": cores,
                         "sample": f"{omp_steps} SSP-RK3 step(s) of {len(omp)} problem(s) ({secs:.1f} s)"}
    except Exception as exc:
        out["openmp"] = {"unavailable": str(exc)[:200]}
    out["kind"] = "oracle"
    out["host"] = host_cpu()
    return out


def host_cpu():
    """The host CPU the oracle runs on: model name (lscpu, else the machine type) and core count."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    import platform
    return {"model": model or platform.machine(), "nproc": os.cpu_count()}


def cpu_baseline(wl, steps: int):
    if steps <= 0:
        _, t1 = oracle_rate(wl, 1)
        steps = max(1, min(200, int(15.0 / max(t1, 1e-3))))
    rate, secs = oracle_rate(wl, steps)
    line = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} SSP-RK3 steps of the same workload ({secs:.1f} s, single-threaded plain C FP64)",
            "host": host_cpu()}
    # the same oracle source built with its element loops parallel (OpenMP), on every host core
    try:
        import oracle
        cores = os.cpu_count() or 1
        used = oracle.lib(openmp=True).orc_threads(cores)
        oracle_rate(wl, 1, threads=used)
        r_omp, s_omp = oracle_rate(wl, steps, threads=used)
        line["openmp"] = {"value": r_omp, "unit": UNIT, "cores": used, "kind": "oracle (OpenMP over elements)",
                          "sample": f"the same {steps} steps ({s_omp:.1f} s)"}
    except Exception as exc:  # a host compiler without OpenMP: report the plain run only
        line["openmp"] = {"unavailable": str(exc)[:200]}
    return line


def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = workload(2)
    for _ in range(max(0, min(args.warmup, 1))):
        oracle_rate(wl, 1)
    per_step = []
    for _ in range(args.steps):
        r, secs = oracle_rate(wl, 1)
        per_step.append(secs)
    total = sum(per_step)
    value = 7 * wl.N * 3 * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(wl, {"l2": "n/a (CPU)"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} SSP-RK3 steps, one per timed step", "host": host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- our leg

def time_path(dg, wl, precision, steps, warmup, flush, stream, local_rank, sample_clocks):
    """K timed SSP-RK3 steps through dg_step, L2 flushed before each; returns timings and kernel data."""
    import torch
    solver = dg.Solver(wl, precision=precision)
    w = torch.from_numpy(wl.w.copy()).cuda()
    for _ in range(warmup):  # the timed steps' operations, so that none is a first use when timed
        torch.cuda._sleep(GATE_CYCLES)
        flush.zero_()
        solver.dg_step(w, wl.dt, 1)
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank) if sample_clocks else None
    if clocks:
        clocks.start()
        clocks.wait_first()
        time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for ev in starts + ends:  # create the events (lazily made at their first record) before timing
        ev.record(stream)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    t_enq = time.perf_counter()
    for k in range(steps):
        # a spin kernel of GATE_CYCLES ahead of each step keeps the GPU busy while the host enqueues
        # the flush, the events and the step, so the events measure the step's device time even
        # when the host is slow to enqueue (the first process on a fresh box)
        torch.cuda._sleep(GATE_CYCLES)
        flush.zero_()
        starts[k].record(stream)
        solver.dg_step(w, wl.dt, 1)
        ends[k].record(stream)
    enqueue_s = time.perf_counter() - t_enq
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    ms = sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends))
    clk = clocks.stop() if clocks else None
    status = solver.dg_status_read()
    kms = solver.dg_time_kernels(w, nrep=20)
    flops, bytes_ = solver.dg_kernel_costs()
    return dict(solver=solver, w=w, ms=ms, wall=wall, clocks=clk, status=status, kms=kms, flops=flops,
                bytes=bytes_, enqueue_s=enqueue_s)


def primitives_host(wl, w):
    """Pressure and velocity from an FP64 state on the host (stiffened gas, Sec. 2)."""
    g1, g2 = wl.gamma
    C1 = g1 * wl.pinf[0] / (g1 - 1.0)
    C2 = g2 * wl.pinf[1] / (g2 - 1.0)
    rho = w[2] + w[3]
    rhoe = w[6] - 0.5 * (w[4] ** 2 + w[5] ** 2) / rho
    P = (rhoe - (w[0] * C1 + (1 - w[0]) * C2)) / (w[0] / (g1 - 1.0) + (1 - w[0]) / (g2 - 1.0))
    return P, w[4] / rho, w[5] / rho


def l2_errors(wl, w32, w64):
    """Relative L2 error of alpha (= phi), P and the velocity of an FP32-bulk state against the FP64
    state of the same run (the FP64 path matches the FP64 oracle to 1e-12 per right-hand side)."""
    import numpy as np
    P32, u32, v32 = primitives_host(wl, w32)
    P64, u64, v64 = primitives_host(wl, w64)
    l2 = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    vel = float(np.sqrt(np.sum((u32 - u64) ** 2 + (v32 - v64) ** 2) / max(np.sum(u64 ** 2 + v64 ** 2), 1e-300)))
    return {"l2_rel_alpha": l2(w32[0], w64[0]), "l2_rel_p": l2(P32, P64), "l2_rel_u": vel}


def run_steps(dg, wl, precision, steps):
    """The FP64 state after `steps` SSP-RK3 steps in one dg_step call."""
    import torch
    s = dg.Solver(wl, precision=precision)
    d = torch.from_numpy(wl.w.copy()).cuda()
    s.dg_step(d, wl.dt, steps)
    out = d.cpu().numpy()
    s.close()
    return out


def accuracy(dg, wl, steps):
    """Relative L2 error of phi, P, u of the FP32-bulk path against the FP64 path after `steps`, and
    the time per step of that FP32-bulk run (all steps in one dg_step call: 3 launches a step, the
    state L2-resident, no flush)."""
    import torch
    out = {"steps": steps, "reference": "FP64 GPU path (matches the FP64 oracle to 1e-12 per RHS)"}
    s = dg.Solver(wl, precision="fp32bulk")
    d = torch.from_numpy(wl.w.copy()).cuda()
    s.dg_step(d, wl.dt, 2)  # warm-up: graphs captured
    d.copy_(torch.from_numpy(wl.w.copy()))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    s.dg_step(d, wl.dt, steps)
    e1.record()
    torch.cuda.synchronize()
    us = 1e3 * e0.elapsed_time(e1) / steps
    w32 = d.cpu().numpy()
    s.close()
    out.update(l2_errors(wl, w32, run_steps(dg, wl, "fp64", steps)))
    out["one_call"] = {"us_per_step": us, "value": 21 * wl.N / (us * 1e-6), "unit": UNIT}
    return out


def batched_block(dg, steps, nprob=256, acc_steps=200):
    """Batched ensemble of 256 independent drop/bubble problems (meshes 16^2..128^2, p in 2..5,
    seed 4): one batched FP32-bulk step vs the same problems stepped one by one (FP32-bulk and
    FP64).  The working set (several GB) is far larger than L2, so no flush is needed."""
    import torch
    from paper_2306_05002_gb300 import workloads as W
    wls = W.ensemble(n=nprob, seed=4)
    nodes = sum(wl.N for wl in wls)
    units = 7 * 3 * nodes
    states = [torch.from_numpy(wl.w.copy()).cuda() for wl in wls]
    dts = [wl.dt for wl in wls]
    bs = dg.BatchSolver(wls)
    for _ in range(2):
        bs.dg_batch_step(states, dts, 1)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(steps):
        bs.dg_batch_step(states, dts, 1)
    t1.record()
    torch.cuda.synchronize()
    ms_b = t0.elapsed_time(t1) / steps
    tiles = bs.dg_batch_tiles()
    bs.close()

    def one_by_one(precision, nrep):
        solvers = [dg.Solver(wl, precision=precision) for wl in wls]
        for s_, w_, wl in zip(solvers, states, wls):
            s_.dg_step(w_, wl.dt, 1)
        torch.cuda.synchronize()
        t0.record()
        for _ in range(nrep):
            for s_, w_, wl in zip(solvers, states, wls):
                s_.dg_step(w_, wl.dt, 1)
        t1.record()
        torch.cuda.synchronize()
        for s_ in solvers:
            s_.close()
        return t0.elapsed_time(t1) / nrep

    ms_32 = one_by_one("fp32bulk", 2)
    ms_64 = one_by_one("fp64", 1)

    # accuracy: the batch after acc_steps steps from the initial states, against single-problem FP64
    # runs of a sample (the first and last problem of each order)
    acc = None
    if acc_steps > 0:
        bs = dg.BatchSolver(wls)
        fresh = [torch.from_numpy(wl.w.copy()).cuda() for wl in wls]
        bs.dg_batch_step(fresh, dts, acc_steps)
        torch.cuda.synchronize()
        bs.close()
        picks = []
        for p in sorted({wl.p for wl in wls}):
            idx = [k for k, wl in enumerate(wls) if wl.p == p]
            picks += sorted({idx[0], idx[-1]})
        per = []
        for k in picks:
            e = l2_errors(wls[k], fresh[k].cpu().numpy(), run_steps(dg, wls[k], "fp64", acc_steps))
            per.append(dict(problem=wls[k].name, **e))
        acc = {"steps": acc_steps, "sample": "first and last problem of each order", "problems": per}
        for key in ("l2_rel_alpha", "l2_rel_p", "l2_rel_u"):
            vals = [e[key] for e in per]
            acc["max_" + key] = float("nan") if any(v != v for v in vals) else max(vals)
        del fresh
    return {"workload": f"{nprob} independent 2D periodic drop/bubble problems, N x N quads with N ~ U{{16..128}}, "
                        "p ~ U{2,3,4,5}, R ~ U[0.05,0.2], seeded centres (seed 4), u=(1,0.5), eps=0.75h, own dt",
            "problems": len(wls), "nodes": nodes, "steps": steps,
            "value": units / (ms_b * 1e-3), "unit": UNIT, "ms_per_step": ms_b,
            "one_by_one_fp32bulk": {"value": units / (ms_32 * 1e-3), "ms_per_step": ms_32},
            "one_by_one_fp64": {"value": units / (ms_64 * 1e-3), "ms_per_step": ms_64},
            "speedup_vs_fp64": ms_64 / ms_b, "l2": "working set > L2 (no flush needed)",
            "roofline": batch_roofline(nodes, ms_b),
            "tiles": tiles, "accuracy": acc,
            "cpu_oracle": oracle_sample(wls[:32], wls, of="the first 32 problems")}


def batch_roofline(nodes, ms_step):
    """Step-level HBM roofline of the batched form: 168 B per node and RK stage (the per-unit figure
    of the single-problem path) over the whole step's duration, launch gaps and all orders' kernels
    included -- a lower bound on the fraction the kernels reach while they run."""
    hbm = peaks().get("hbm_gbs", 6800.0)
    ach = BYTES_PER_NODE_STAGE * nodes * 3 / (ms_step * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "whole batched step (volume, fused and surface kernels of every order)",
            "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "per_unit": f"{BYTES_PER_NODE_STAGE} B per node and stage x 3 stages x {nodes} nodes",
            "duration": "step time (CUDA events over the batched steps)",
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy), of measured"}


def rt_block(dg, steps, n=256, paper=False, cpu=False, acc_steps=0, bubble=False):
    """Viscous Rayleigh-Taylor set-up (256 x 256 quads, p = 4, walls, gravity, surface tension,
    seed 3): FP32-bulk and FP64 step times and the FP32-bulk error after the timed steps.
    The state (92 MB FP64, 1.64M nodes) and the workspace exceed L2 together; no flush.
    paper: the paper's domain [0, 1] x [0, 4] on n x 4n quads instead (slip sides, no-slip bottom,
    the Riemann-invariant pressure top, no surface tension).  cpu: also the oracle on a bounded
    sample (one right-hand side on one core, one step on every core).  acc_steps > 0: also the
    FP32-bulk errors (alpha, P, u) against FP64 after that many steps from the initial state.
    bubble: the paper's rising bubble (case 1) on n x 2n quads instead."""
    import torch
    from paper_2306_05002_gb300 import workloads as W
    if bubble:
        wl = W.rising_bubble(nx=n, ny=2 * n, p=4, case=1)
        desc = (f"2D rising bubble (the paper's case 1: R=0.25 at (0,0.5) in [-0.5,0.5]x[0,2], density and "
                f"viscosity ratio 10, Re=35, Eo=10) on {n}x{2 * n} quads p=4, slip sides, no-slip bottom, "
                "Riemann-invariant pressure top")
    elif paper:
        wl = W.rayleigh_taylor_paper(nx=n, ny=4 * n, p=4)
        desc = (f"2D viscous Rayleigh-Taylor, the paper's domain [0,1]x[0,4] on {n}x{4 * n} quads p=4, slip sides, "
                "no-slip bottom, Riemann-invariant pressure top, g=-9.81, density ratio 3, Re=3000")
    else:
        wl = W.rayleigh_taylor(n=n, p=4, seed=3)
        desc = (f"2D viscous Rayleigh-Taylor {n}x{n} quads p=4, no-slip walls, g=-9.81, sigma=0.07, "
                "density ratio 3, seeded 8-mode interface")
    out = {"workload": desc, "nodes": wl.N, "steps": steps}
    states = {}
    for prec in ("fp32bulk", "fp64"):
        s = dg.Solver(wl, precision=prec)
        w = torch.from_numpy(wl.w.copy()).cuda()
        s.dg_step(w, wl.dt, 2)
        w.copy_(torch.from_numpy(wl.w.copy()))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.dg_step(w, wl.dt, steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[prec] = {"ms_per_step": ms, "value": 21 * wl.N / (ms * 1e-3), "unit": UNIT,
                     "device_status": s.dg_status_read()}
        names = NAMES[prec]
        f, b = s.dg_kernel_costs()
        out[prec]["roofline"] = roofline(prec, names, s.dg_time_kernels(w, nrep=10), f, b, wl.N)
        states[prec] = w.cpu().numpy()
        s.close()
    out["accuracy_after_timed_steps"] = l2_errors(wl, states["fp32bulk"], states["fp64"])
    if acc_steps > 0:
        acc = {"steps": acc_steps}
        acc.update(l2_errors(wl, run_steps(dg, wl, "fp32bulk", acc_steps), run_steps(dg, wl, "fp64", acc_steps)))
        out["accuracy"] = acc
    out["speedup_fp32bulk_vs_fp64"] = out["fp64"]["ms_per_step"] / out["fp32bulk"]["ms_per_step"]
    if cpu:
        out["cpu_oracle"] = oracle_sample([wl], [wl], of="the full grid")
    return out


def kin_flops_per_node_stage(p):
    """Algorithmic FP64 flops per node and RK stage of the kinematic mode on rectangles (both fields,
    2 per multiply-add): the gradients of phi and psi and the weak-form term of -a_1 (six contractions
    of length p+1), n, a_1, the transport terms and the velocity (23); per face node the transport and
    SIP fluxes and the symmetric term (34, 4 (p+1) face nodes per (p+1)^2 nodes); the lifting, M^-1 and
    the RK4 update (20).  The neighbour's trace, which the stage kernel evaluates again from the
    neighbour's nodal values, is not counted twice."""
    P1 = p + 1
    return 12 * P1 + 23 + 34 * 4 * P1 // (P1 * P1) + 20


def reinit_flops_per_node_stage(p):
    """Algorithmic FP64 flops per node and SSP-RK3 stage of the level-set re-initialisation (one field,
    2 per multiply-add): the gradient and the weak-form diffusion term (four contractions of length
    p+1), the source S (1 - |grad psi|) (9); per face node the SIP flux and the symmetric term (11,
    4 (p+1) face nodes per (p+1)^2 nodes); the lifting, M^-1 and the stage update (14)."""
    P1 = p + 1
    return 8 * P1 + 9 + 11 * 4 * P1 // (P1 * P1) + 14


def reinit_block(dg, iters, n=64):
    """Level-set re-initialisation (end of Sec. 3) of the Rider-Kothe drop on n x n quads, p = 3, FP64:
    `iters` pseudo-time SSP-RK3 steps with the default nu and dtau in one dg_reinit call (the paper
    applies ~50 every 2000 steps); one sign kernel, then a volume and a surface kernel per stage."""
    import torch
    from paper_2306_05002_gb300 import workloads as W
    wl = W.rider_kothe(n=n, p=3)
    s = dg.KinematicSolver(wl)
    w = torch.from_numpy(wl.w.copy()).cuda()
    s.dg_reinit(w, 3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    s.dg_reinit(w, iters)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    status = s.dg_status_read()
    s.close()
    per_iter = ms / iters
    ach = reinit_flops_per_node_stage(wl.p) * wl.N * 3 / (per_iter * 1e-3) / 1e12
    return {"workload": f"level-set re-initialisation of the Rider-Kothe drop, {n}x{n} quads p=3, FP64, "
                        f"{iters} SSP-RK3 pseudo-time steps", "nodes": wl.N, "iterations": iters,
            "ms_per_iteration": per_iter, "ms_total": ms, "gpu_launches": 1 + 6 * iters,
            "device_status": status,
            "roofline": {"bound": "alu", "kernel": "k_ri_volume + k_ri_surface", "achieved": ach,
                         "peak": fp64_peak(), "unit": "TFLOP/s", "frac": ach / fp64_peak(),
                         "per_unit": f"{reinit_flops_per_node_stage(wl.p)} flops per node and stage x {wl.N} nodes",
                         "duration": "call time / iterations / 3 stages (gaps included)"}}


def kinematic_block(dg, steps, n=64):
    """Kinematic mode (Sec. 4.1), FP64, classical RK4: the Rider-Kothe vortex on n x n quads,
    p = 3, timed over `steps` steps (2 fields x 4 right-hand sides per step per node); and the
    full period T = 4 on 16 x 16, p = 3 (the paper's 64^2-DoF mesh): L1 error of phi against
    the initial drop and the relative phase-field mass error (paper, p = 3: L1 1.75e-2)."""
    import numpy as np
    import torch
    from paper_2306_05002_gb300 import workloads as W
    wl = W.rider_kothe(n=n, p=3)
    s = dg.KinematicSolver(wl)
    w = torch.from_numpy(wl.w.copy()).cuda()
    s.dg_kin_step(w, 0.0, wl.dt, 2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    s.dg_kin_step(w, 2 * wl.dt, wl.dt, steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    s.close()
    small = W.rider_kothe(n=16, p=3)
    s = dg.KinematicSolver(small)
    w = torch.from_numpy(small.w.copy()).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.dg_kin_step(w, 0.0, small.dt, small.nsteps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    wend = w.cpu().numpy()
    s.close()
    # GLL weights w_i = 2 / (p (p + 1) P_p(xi_i)^2)
    from numpy.polynomial import legendre
    xi = W.gll_points(3)
    wt = 2.0 / (3 * 4 * legendre.Legendre.basis(3)(xi) ** 2)
    M = np.tile(np.outer(wt, wt).ravel() * 0.25 * small.hx * small.hy, small.nx * small.ny)
    ach = kin_flops_per_node_stage(wl.p) * wl.N * 4 / (ms * 1e-3) / 1e12
    return {"workload": f"Rider-Kothe vortex {n}x{n} quads p=3, T=4, eps=0.75 h/(p+1), Gamma=1, FP64, classical RK4",
            "nodes": wl.N, "steps": steps, "ms_per_step": ms, "value": 2 * 4 * wl.N / (ms * 1e-3), "unit": UNIT,
            "gpu_launches_per_step": 4,
            "roofline": {"bound": "alu", "kernel": "k_kin_stage", "achieved": ach,
                         "peak": fp64_peak(), "unit": "TFLOP/s", "frac": ach / fp64_peak(),
                         "per_unit": f"{kin_flops_per_node_stage(wl.p)} flops per node and stage x {wl.N} nodes",
                         "duration": "step time / 4 (one kernel per stage in a graph; gaps included)"},
            "full_period_16x16p3": {"steps": small.nsteps, "wall_s": wall,
                                    "l1_phi": float(np.sum(M * np.abs(wend[0] - small.w[0]))),
                                    "mass_error": float(np.sum(M * (wend[0] - small.w[0])) / np.sum(M * small.w[0])),
                                    "paper_l1_p3_64sq_dof": 1.75e-2}}


def slab_block(dg, steps):
    """The 1D periodic water slab in air (100 elements, p = 3, eps = h, u = 1): `steps` SSP-RK3 steps
    in one dg_step call (CUDA graphs of 8 steps), FP64 (the configuration's precision) and
    FP32-bulk with its relative L2 errors (alpha, P, u) against FP64 after them.  Far too small for
    a roofline (400 nodes): the step latency is the number to read."""
    import torch
    from paper_2306_05002_gb300 import workloads as W
    wl = W.slab_1d(nx=100, p=3)
    out = {"workload": "1D periodic water slab in air, 100 elements p=3, eps=h, u=1, SSP-RK3", "nodes": wl.N,
           "steps": steps}
    states = {}
    for prec in ("fp64", "fp32bulk"):
        s = dg.Solver(wl, precision=prec)
        w = torch.from_numpy(wl.w.copy()).cuda()
        s.dg_step(w, wl.dt, 9)
        w.copy_(torch.from_numpy(wl.w.copy()))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.dg_step(w, wl.dt, steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[prec] = {"us_per_step": 1e3 * ms, "value": 21 * wl.N / (ms * 1e-3), "unit": UNIT,
                     "device_status": s.dg_status_read()}
        states[prec] = w.cpu().numpy()
        s.close()
    out["accuracy"] = l2_errors(wl, states["fp32bulk"], states["fp64"])
    return out


def tri_flops_per_stage(p):
    """Algorithmic FP64 flops of one triangle and one RK stage (both fields), 2 per multiply-add:
    phi and its r-, s-derivatives and psi's at the (p+2)^2 volume points (5 dot products of length
    Np); on both sides of the 3 (p+2) edge points phi, psi and psi's tangential derivative from the
    p+1 edge nodes and the normal derivatives of phi and psi from all Np; the weak-form sums at
    every node (4 basis terms per volume point, the lifted symmetric term at every edge point, the
    edge fluxes of phi and psi on the edges through the node); M^-1 R for two fields."""
    P1, Np, nq1 = p + 1, (p + 1) * (p + 2) // 2, p + 2
    nqv, nqe = nq1 * nq1, 3 * nq1
    return (10 * Np * nqv + 2 * nqe * (3 * P1 + 2 * Np) * 2 + 8 * Np * nqv + 2 * Np * nqe
            + 12 * P1 * nq1 + 4 * Np * Np)


def triangle_block(dg, steps, n=64):
    """Kinematic mode on triangles (the paper's mesh (b)), FP64, classical RK4: the Rider-Kothe
    vortex on n x n cells split into 2 n^2 triangles, p = 3, timed over `steps` steps (one fused
    kernel per stage, four per step); and the full period T = 4 on 16 x 16 cells (the paper's mesh
    (b) 64^2-DoF row): L1 error of phi and the relative mass error (paper, p = 3: L1 1.58e-2)."""
    import numpy as np
    import torch
    from paper_2306_05002_gb300 import workloads as W
    wl = W.rider_kothe(n=n, p=3, elem="tri")
    s = dg.KinematicSolver(wl)
    w = torch.from_numpy(wl.w.copy()).cuda()
    s.dg_kin_step(w, 0.0, wl.dt, 8)
    s.dg_kin_step(w, 8 * wl.dt, wl.dt, 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    s.dg_kin_step(w, 9 * wl.dt, wl.dt, steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    s.close()
    flops = tri_flops_per_stage(wl.p) * wl.E
    stage_ms = ms / 4
    ach = flops / (stage_ms * 1e-3) / 1e12
    small = W.rider_kothe(n=16, p=3, elem="tri")
    s = dg.KinematicSolver(small)
    w = torch.from_numpy(small.w.copy()).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.dg_kin_step(w, 0.0, small.dt, small.nsteps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    wend = w.cpu().numpy()
    s.close()
    # int f = sum over triangles of sum_n f_n int l_n, with int l_n of the cubic equispaced basis
    # (the triangle's Newton-Cotes weights): 1/30 at the vertices, 3/40 on the edges, 9/20 at the
    # centroid, times the area
    wn = np.array([1 / 30, 3 / 40, 3 / 40, 1 / 30, 3 / 40, 9 / 20, 3 / 40, 3 / 40, 3 / 40, 1 / 30])
    M = np.tile(wn * 0.5 * small.hx * small.hy, small.E)
    l1 = float(np.sum(M * np.abs(wend[0] - small.w[0])))
    mass = float(np.sum(M * (wend[0] - small.w[0])) / np.sum(M * small.w[0]))
    return {"workload": f"Rider-Kothe vortex {n}x{n} cells split into {wl.E} triangles, p=3, T=4, eps=0.75 h/(p+1), "
                        f"Gamma=1, FP64, classical RK4",
            "nodes": wl.N, "steps": steps, "ms_per_step": ms, "value": 2 * 4 * wl.N / (ms * 1e-3), "unit": UNIT,
            "gpu_launches_per_step": 4,
            "roofline": {"bound": "alu", "kernel": "k_tri_stage", "achieved": ach, "peak": fp64_peak(),
                         "unit": "TFLOP/s", "frac": ach / fp64_peak(),
                         "per_unit": f"{tri_flops_per_stage(wl.p)} flops per triangle and stage x {wl.E} triangles",
                         "duration": "step time / 4 (graph of back-to-back stage kernels; gaps included)"},
            "full_period_16x16p3": {"steps": small.nsteps, "wall_s": wall, "l1_phi": l1,
                                    "mass_error": mass, "paper_l1_p3_64sq_dof_mesh_b": 1.58e-2}}


def adjoint_block(dg, steps, every=20, n=128):
    """Gradient of J = 1/2 int (alpha_N - alpha*)^2 with respect to the initial state of the
    128 x 128, p = 3 drop (level set with 16 seeded Fourier coefficients, seed 5/50/51),
    FP64, checkpoints every 20 steps.  adjoint/forward = backward sweep (segment replay +
    adjoint steps) / forward sweep (with checkpoint copies)."""
    import numpy as np
    import torch
    from paper_2306_05002_gb300 import adjoint as A
    from paper_2306_05002_gb300 import workloads as W
    wl = W.adjoint_drop(n=n, p=3, nsteps=steps)
    tgt = W.adjoint_drop(n=n, p=3, nsteps=steps, theta=np.random.default_rng(51).normal(0, 0.01, 16))
    s = dg.Solver(wl)
    x = torch.from_numpy(tgt.w.copy()).cuda()
    s.dg_step(x, wl.dt, steps)
    target = x[0].clone()
    w0 = torch.from_numpy(wl.w.copy()).cuda()
    # warm-up: the same forward and backward sweeps once, untimed, with the same operations as the
    # timed ones (graph capture, allocator, and the first use of every torch kernel: a torch
    # kernel's first launch in a process loads its module, which has taken 0.6 s on a fresh box)
    wW, ckW = A.forward(s, w0, wl.dt, steps, every)
    lamW = torch.zeros_like(wW)
    lamW[0] = wW[0] - target
    A.backward(s, ckW, lamW, wl.dt, steps, every)
    del wW, ckW, lamW
    torch.cuda.synchronize()
    # Three timed repetitions, the median reported.  Each checkpoint segment of the backward sweep
    # is one captured graph (dg_adjoint_segment), reused by every sweep: the warm-up captured it.
    tfs, tbs = [], []
    for _ in range(3):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        wN, ckpt = A.forward(s, w0, wl.dt, steps, every)
        e[1].record()
        lam = torch.zeros_like(wN)
        lam[0] = wN[0] - target  # J's gradient up to the (positive) quadrature weights
        lam0 = A.backward(s, ckpt, lam, wl.dt, steps, every)
        e[2].record()
        torch.cuda.synchronize()
        tfs.append(e[0].elapsed_time(e[1]))
        tbs.append(e[1].elapsed_time(e[2]))
        del wN, ckpt
    tf, tb = float(np.median(tfs)), float(np.median(tbs))
    ok = bool(torch.isfinite(lam0).all())
    s.close()
    return {"workload": f"2D drop {n}x{n} quads p=3, FP64, 16 level-set Fourier parameters (seeds 5, 50, 51)",
            "steps": steps, "checkpoint_every": every, "forward_ms": tf, "backward_ms": tb,
            "adjoint_over_forward": tb / tf, "repetitions_ms": {"forward": tfs, "backward": tbs}, "finite": ok}


def summary(line):
    """A short digest of the line, one entry per configuration (3 significant digits): the figures
    a reader of the line's last few hundred characters needs."""
    r3 = lambda x: float(f"{x:.3g}") if isinstance(x, (int, float)) and x == x else x
    acc3 = lambda a: None if not a else [r3(a.get(k, a.get("max_" + k))) for k in ("l2_rel_alpha", "l2_rel_p", "l2_rel_u")]
    out = {"acc_order": "l2_rel alpha, P, u vs the FP64 path",
           "config2": {"us_per_step": r3(1e3 * line["ms_per_step"]), "value": r3(line["value"]),
                       "frac": r3(line["roofline"]["frac"]), "e2e": r3(line["e2e"]["value"]),
                       "acc_500": acc3(line.get("accuracy"))}}
    if line.get("accuracy") and "one_call" in line["accuracy"]:
        out["config2"]["us_per_step_500_in_one_call"] = r3(line["accuracy"]["one_call"]["us_per_step"])
    if "fp64" in line:
        out["config2"]["fp64_us_per_step"] = r3(1e3 * line["fp64"]["ms_per_step"])
    if "slab_1d" in line:
        sl = line["slab_1d"]
        out["config1"] = {"fp64_us_per_step": r3(sl["fp64"]["us_per_step"]),
                          "fp32bulk_us_per_step": r3(sl["fp32bulk"]["us_per_step"]), "acc_1000": acc3(sl["accuracy"])}
    if "rayleigh_taylor" in line:
        rt = line["rayleigh_taylor"]
        out["config3"] = {"ms_per_step": r3(rt["fp32bulk"]["ms_per_step"]), "value": r3(rt["fp32bulk"]["value"]),
                          "frac": r3(rt["fp32bulk"]["roofline"]["frac"]),
                          "fp64_ms_per_step": r3(rt["fp64"]["ms_per_step"]), "acc_2000": acc3(rt.get("accuracy"))}
    if "batched" in line:
        b = line["batched"]
        out["config4"] = {"ms_per_step": r3(b["ms_per_step"]), "value": r3(b["value"]),
                          "frac": r3(b["roofline"]["frac"]) if "roofline" in b else None,
                          "speedup_vs_fp64": r3(b["speedup_vs_fp64"]), "acc_200_max": acc3(b.get("accuracy"))}
    if "rising_bubble" in line:
        rb = line["rising_bubble"]
        out["rising_bubble"] = {"ms_per_step": r3(rb["fp32bulk"]["ms_per_step"]),
                                "fp64_ms_per_step": r3(rb["fp64"]["ms_per_step"]), "acc": acc3(rb.get("accuracy"))}
    if "adjoint" in line:
        a = line["adjoint"]
        out["config5"] = {"adjoint_over_forward": r3(a["adjoint_over_forward"]), "forward_ms": r3(a["forward_ms"]),
                          "backward_ms": r3(a["backward_ms"])}
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2306_05002_gb300 as dg

    torch.cuda.set_device(local_rank)
    dist = world > 1
    if dist:
        import torch.distributed as tdist

    def barrier():
        if dist:
            tdist.barrier()
        torch.cuda.synchronize()

    wl = workload(2 + rank)
    measure_pipes(dg)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    other = "fp64" if args.precision == "fp32bulk" else None

    barrier()
    main = time_path(dg, wl, args.precision, args.steps, args.warmup, flush, stream, local_rank, True)
    barrier()
    ref = time_path(dg, wl, other, args.steps, args.warmup, flush, stream, local_rank, False) if other else None

    # roofline of the dominant kernel of the timed path
    names = NAMES[args.precision]
    kms, flops, bytes_ = main["kms"], main["flops"], main["bytes"]
    roof = roofline(args.precision, names, kms, flops, bytes_, wl.N)
    roof["traffic"] = profiled_traffic(roof["kernel"], wl.name, args.precision)

    # end to end through the public API with a pinned host state: H2D, step, D2H
    solver = main["solver"]
    host = torch.from_numpy(wl.w.copy()).pin_memory()
    for _ in range(2):
        solver.dg_step(host, wl.dt, 1)
    torch.cuda.synchronize()
    e2e_steps = max(5, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.dg_step(host, wl.dt, 1)
    torch.cuda.synchronize()
    e2e_t = time.perf_counter() - t0

    acc = (accuracy(dg, wl, args.accuracy_steps)
           if (args.precision == "fp32bulk" and args.accuracy_steps > 0 and rank == 0) else None)
    batched = (batched_block(dg, args.batch_steps, args.batch_problems, args.batch_accuracy_steps)
               if (args.batch_steps > 0 and rank == 0) else None)
    adjoint = (adjoint_block(dg, args.adjoint_steps, n=args.adjoint_n)
               if (args.adjoint_steps > 0 and rank == 0) else None)
    rt = (rt_block(dg, args.rt_steps, cpu=True, acc_steps=args.rt_accuracy_steps)
          if (args.rt_steps > 0 and rank == 0) else None)
    slab = slab_block(dg, args.slab_steps) if (args.slab_steps > 0 and rank == 0) else None
    kin = kinematic_block(dg, args.kin_steps) if (args.kin_steps > 0 and rank == 0) else None
    tri = triangle_block(dg, args.tri_steps, args.tri_n) if (args.tri_steps > 0 and rank == 0) else None
    ri = reinit_block(dg, args.reinit_iters) if (args.reinit_iters > 0 and rank == 0) else None
    rtp = rt_block(dg, args.rt_paper_steps, n=64, paper=True) if (args.rt_paper_steps > 0 and rank == 0) else None
    rb = (rt_block(dg, args.rb_steps, n=20, bubble=True, acc_steps=1000)
          if (args.rb_steps > 0 and rank == 0) else None)

    ms_max, e2e_max, ref_ms = reduce_max([main["ms"], e2e_t, ref["ms"] if ref else 0.0], "cuda")

    if rank == 0:
        units = 7 * wl.N * 3
        value = weak_scaling_value(units, args.steps, world, ms_max)
        launches = main["solver"].dg_step_launches(1)  # kernels of one single-step dg_step call
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
                "data": "synthetic",
                "config": config_of(wl, {"parallelism": f"replicas x{world}", "precision": args.precision,
                                         "wall_s_timed_region": main["wall"],
                                         "host_enqueue_s": main["enqueue_s"]}),
                "gpu_launches": launches * args.steps,
                "roofline": roof,
                "e2e": {"value": units * e2e_steps * world / e2e_max, "unit": UNIT,
                        "h2d_bytes_per_step": 8 * 7 * wl.N, "d2h_bytes_per_step": 8 * 7 * wl.N},
                "clocks": main["clocks"], "device_status": main["status"],
                "pipe_peaks": dict(MEASURED_PIPES, fp64_derived_tflops=FP64_PEAK_DERIVED)}
        if ref:
            line["fp64"] = {"value": units * args.steps * world / (ref_ms * 1e-3), "unit": UNIT,
                            "ms_per_step": ref_ms / args.steps, "kernel_ms": dict(zip(["k_volume", "k_surface"],
                                                                                        ref["kms"])),
                            "device_status": ref["status"]}
            line["speedup_vs_fp64"] = ref_ms / ms_max
        if acc:
            line["accuracy"] = acc
        if batched:
            line["batched"] = batched
        if adjoint:
            line["adjoint"] = adjoint
        if rt:
            line["rayleigh_taylor"] = rt
        if slab:
            line["slab_1d"] = slab
        if kin:
            line["kinematic"] = kin
        if tri:
            line["kinematic_triangles"] = tri
        if ri:
            line["reinit"] = ri
        if rtp:
            line["rayleigh_taylor_paper_domain"] = rtp
        if rb:
            line["rising_bubble"] = rb
        if world == 1:
            line["cpu_baseline"] = cpu_baseline(wl, args.cpu_sample_steps)
        line["summary"] = summary(line)  # last key: a short digest of every block
        print(json.dumps(line), flush=True)
    main["solver"].close()
    if ref:
        ref["solver"].close()


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as tdist
            tdist.destroy_process_group()


if __name__ == "__main__":
    main()
