#!/usr/bin/env python3
"""Throughput benchmark of the fused hybrid central-moment / BGK lattice Boltzmann step.

Workload (default): spinodal decomposition on a 4096 x 4096 periodic D2Q9 lattice, phi i.i.d.
uniform in [-0.05, 0.05] (SplitMix64 seed 2024), u = 0, rho = 1, viscosity ratio 1:10
(nu_l = 0.1, nu_g = 0.01, tau interpolated linearly in phi), a = gamma = 0.04, M = 0.1,
Gamma = 1, FP32 storage and arithmetic.  One step = one launch of the fused kernel over all
nodes (both population sets).  Metric: MLUPS counting one update of f and g per node.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--n 4096] [--prec fp32] [--no-e2e] [--no-cpu-baseline]

Under torchrun (N > 1) every rank runs an independent replica of the lattice on its own GPU
(no data-path collective; weak scaling); the step time is the max over ranks.
``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded sample of the
same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "MLUPS (f+g) and % HBM roofline on 1 GB300; surrogate/16-bit/batch speedup at φ err"
BYTES_PER_NODE = {"fp64": 288, "fp32": 144, "fp16s": 80, "bf16s": 80}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16s": "f32 (16-bit storage)", "bf16s": "f32 (bf16 storage)"}
PHYS = dict(nu_l=0.1, nu_g=0.01, a=0.04, gamma=0.04, M=0.1, Gamma=1.0)
SEED = 2024


def tau(nu):
    return nu * 3.0 + 0.5


def workload_params():
    return dict(tau_l=tau(PHYS["nu_l"]), tau_g=tau(PHYS["nu_g"]), a=PHYS["a"], gamma=PHYS["gamma"],
                M=PHYS["M"], Gamma=PHYS["Gamma"])


# ------------------------------------------------------------------------------------------
# Environment helpers.

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Sources that hold the device code of the fused step kernel the roofline reports: k_step (FP32 /
# FP64) and, for 16-bit storage, k_step_pair as well.  Host-side files (launchers, the C ABI) are
# left out: editing them does not change what the kernel reads and writes.
STEP_SOURCES = ("lbm_step.cuh", "lbm_device.cuh")
PAIR_SOURCES = STEP_SOURCES + ("lbm_pair.cu", "lbm_pair.cuh", "lbm_f2.cuh")


def kernel_source_hash(prec: str = "fp32"):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1803_11345_gb300", "csrc")
    for name in (PAIR_SOURCES if prec in ("fp16s", "bf16s") else STEP_SOURCES):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(prec: str, n: int):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, if it was
    taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", f"k_step_{prec}_spinodal.md")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("bench-traffic:"):
                for kv in line.split(":", 1)[1].split():
                    k, v = kv.split("=")
                    vals[k] = v
    if vals.get("source_hash") != kernel_source_hash(prec):
        return None
    try:
        per_node = float(vals["dram_bytes_per_node"])
    except (KeyError, ValueError):
        return None
    return per_node * n * n


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons every 100 ms; stop() reports the samples
    that arrived inside [t0, t1] (host clock), the window of sustained load around the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0=None, t1=None):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.15)  # let the sample that closes the window arrive
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, power, smax, reasons = [], [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in list(self.lines):
            if (t0 is not None and ts < t0) or (t1 is not None and ts > t1 + 0.12):
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "sm_mhz_min": min(sm) if sm else None, "power_w_max": max(power) if power else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "window": "samples taken while the lattice was stepped continuously: load steps before and "
                          "after the timed region plus the timed region itself"}


def max_over_ranks(value: float) -> float:
    """Max of a per-rank timing over all ranks (identity without a process group).  Runs on the
    CPU for gloo and on the current CUDA device for NCCL."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes_per_rank: int, steps: int, world: int, ms_max: float) -> float:
    """Weak scaling: every rank advances its own replica; the job's rate counts all replicas
    over the slowest rank's time."""
    return world * nodes_per_rank * steps / (ms_max * 1e-3) / 1e6


# ------------------------------------------------------------------------------------------
# CPU oracle leg (bounded sample).

def time_oracle(budget_s: float, n_side: int, max_steps: int = 10**9, threads: int = 0):
    """Run the FP64 oracle on an n_side^2 sample of the workload for up to budget_s seconds
    (whole steps) on `threads` OpenMP threads (0: all host cores).  Returns (MLUPS, steps,
    seconds, threads used)."""
    import oracle
    from paper_1803_11345_gb300 import workloads as W
    oracle.build()
    default = oracle.set_threads(0)
    threads = oracle.set_threads(threads if threads > 0 else default)
    phi0 = W.spinodal(n_side, n_side, seed=SEED)
    o = oracle.Oracle(phi0, visc_interp=1, **workload_params())
    o.step(1)
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps:
        o.step(1)
        steps += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    o.close()
    oracle.set_threads(default)
    return n_side * n_side * steps / dt / 1e6, steps, dt, threads


def oracle_case(phi0, params, budget_s, max_steps):
    """MLUPS of the FP64 oracle (all host cores) on one workload: whole steps for up to budget_s
    seconds (at most max_steps) after one untimed step."""
    import oracle
    oracle.build()
    o = oracle.Oracle(phi0, **params)
    o.step(1)
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps:
        o.step(1)
        steps += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    o.close()
    ny, nx = phi0.shape
    return {"mlups": nx * ny * steps / dt / 1e6, "steps": steps, "seconds": round(dt, 3)}


def oracle_sizes(budget_s=3.0):
    """The oracle timed at the sizes of the paper's workloads (FP64, all host cores)."""
    from paper_1803_11345_gb300 import workloads as W
    out = {}
    lap = dict(tau_l=1.0, tau_g=1.0, gamma=0.02, a=0.04, M=0.1, Gamma=1.0)
    out["laplace droplet 64x64"] = oracle_case(W.droplet(64, 64, 16, gamma=0.02, a=0.04), lap, budget_s, 2000)
    sp = dict(workload_params(), visc_interp=1)
    out["spinodal 256x256"] = oracle_case(W.spinodal(256, 256, seed=SEED), sp, budget_s, 1000)
    ch = dict(tau_l=tau(0.2), tau_g=tau(0.02), gamma=0.04, a=0.04, M=0.1, Gamma=1.0, walls=1, u_top=0.01,
              u_bottom=-0.01)
    out["sheared channel 1024x512"] = oracle_case(W.droplet(1024, 512, 64, gamma=0.04, a=0.04), ch, budget_s, 300)
    out["spinodal 4096x4096"] = oracle_case(W.spinodal(4096, 4096, seed=SEED), sp, budget_s, 3)
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    # Each timed step is one oracle time step on a sample lattice sized so that the whole
    # K-step run takes about 30 s of host time.
    import oracle
    from paper_1803_11345_gb300 import workloads as W
    oracle.build()
    threads = oracle.set_threads(0)
    probe = 64
    o = oracle.Oracle(W.spinodal(probe, probe, seed=SEED), visc_interp=1, **workload_params())
    t0 = time.perf_counter()
    o.step(3)
    per_node = (time.perf_counter() - t0) / (3 * probe * probe)
    o.close()
    target = 30.0 / max(1, args.steps + args.warmup)
    side = int(max(16, min(args.n, math.sqrt(target / per_node))))
    phi0 = W.spinodal(side, side, seed=SEED)
    o = oracle.Oracle(phi0, visc_interp=1, **workload_params())
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    o.close()
    mlups = side * side * args.steps / dt / 1e6
    sample = f"{side}x{side} periodic sample of the spinodal workload (same parameters), FP64"
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(args),
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --kernel choices: (variant getter, bx, by, depth); "auto" keeps the library's default.
KERNELS = {
    "generic": (lambda m: m.LBM_KERNEL_GENERIC, 256, 1, 1),
    "pair": (lambda m: m.LBM_KERNEL_PAIR, 128, 1, 1),
    "pair_staged": (lambda m: m.LBM_KERNEL_PAIR_STAGED, 128, 1, 1),
}


def config_dict(args):
    return {"workload": f"spinodal decomposition {args.n}x{args.n} periodic, viscosity ratio 1:10 "
                        f"(tau linear in phi), {args.prec} storage",
            "nx": args.n, "ny": args.n, "precision": args.prec, "seed": SEED,
            "nu_l": PHYS["nu_l"], "nu_g": PHYS["nu_g"], "a": PHYS["a"], "gamma": PHYS["gamma"],
            "M": PHYS["M"], "collision": "central moments (f) + BGK (g)",
            "l2": "inputs larger than L2 (state >= 1 GB per buffer at 4096^2): no flush",
            "parallelism": f"replicas x{args.gpus}", "kernel": args.kernel}


# ------------------------------------------------------------------------------------------
# GPU leg.

def storage_forms(lbm, phi0, params, stream, ms_fp32, steps=500, phi_steps=1000):
    """The 16-bit storage forms on the same workload and GPU, rounded to nearest and stochastically:
    time per step against the FP32 step just timed, and phi after `phi_steps` steps against an FP32
    run from the same state (the error against the FP64 oracle is stated by the tests: 2e-3 FP16,
    2e-2 BF16 over 1000 steps; the deformation statistic is stated there too)."""
    import numpy as np
    import torch
    ref = lbm.Lattice(phi0, stream=stream, **params)
    ref.step(phi_steps)
    phi_ref = ref.fields()[3]
    ref.close()
    out = {}
    # each 16-bit form rounded to nearest (the default) and stochastically (lbm_params.rounding)
    for form in ("fp16s", "bf16s", "fp16s+sr", "bf16s+sr"):
        prec = form.split("+")[0]
        kw = dict(params, prec=lbm.PRECISIONS[prec])
        if form.endswith("+sr"):
            kw.update(rounding=lbm.LBM_ROUND_STOCHASTIC, seed=1)
        lat = lbm.Lattice(phi0, stream=stream, **kw)
        lat.step(20)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        lat.step(phi_steps - 20 - steps)
        d = np.abs(lat.fields()[3] - phi_ref)
        kernel = {lbm.LBM_KERNEL_PAIR: "k_step_pair (two nodes per thread)"}.get(lat.kernel[0], "k_step")
        lat.close()
        nodes = phi0.size
        out[form] = {"ms_per_step": ms, "mlups": nodes / (ms * 1e-3) / 1e6, "speedup_vs_fp32": ms_fp32 / ms,
                     "hbm_frac": BYTES_PER_NODE[prec] * nodes / (ms * 1e-3) / 1e9 / measured_peaks()[0],
                     "phi_vs_fp32_after_steps": phi_steps, "phi_max_abs_diff": float(d.max()),
                     "phi_rms_diff": float(np.sqrt((d * d).mean())), "kernel": kernel}
    return out

def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1803_11345_gb300 import build as B
    ws, rank, local = dist_env()
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    B.build()
    from paper_1803_11345_gb300 import lbm
    from paper_1803_11345_gb300 import workloads as W

    n = args.n
    phi0 = W.spinodal(n, n, seed=SEED + rank)
    params = dict(prec=lbm.PRECISIONS[args.prec], visc=lbm.LBM_TAU_LINEAR, **workload_params())
    stream = torch.cuda.Stream()
    lat = lbm.Lattice(phi0, stream=stream, **params)
    if args.kernel != "auto":
        lat.set_kernel(KERNELS[args.kernel][0](lbm), *KERNELS[args.kernel][1:])

    def barrier():
        if ws > 1:
            dist.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    lat.step(args.warmup)
    torch.cuda.synchronize()
    # Keep the GPU stepping for ~0.4 s on each side of the timed region (untimed), so that the
    # clock sampler (one sample per 100 ms) sees the clocks of sustained load around it.
    probe0, probe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    probe0.record(stream)
    lat.step(5)
    probe1.record(stream)
    torch.cuda.synchronize()
    pad = 0 if args.pad_ms <= 0 else max(1, int(args.pad_ms / max(probe0.elapsed_time(probe1) / 5, 1e-3)))
    t_load0 = time.time()
    if pad:
        lat.step(pad)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(args.steps)
    e1.record(stream)
    if pad:
        lat.step(pad)
    torch.cuda.synchronize()
    t_load1 = time.time()
    barrier()
    clk = clocks.stop(t_load0, t_load1)
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms)
    nodes = n * n
    mlups = whole_job_mlups(nodes, args.steps, ws, ms_max)
    ms_step = ms_max / args.steps

    # Roofline of the dominant (only) kernel in the timed region: algorithmic bytes per launch
    # / average launch duration (CUDA events on the launching stream).
    peak, peak_kind = measured_peaks()
    bpn = BYTES_PER_NODE[args.prec]
    achieved = bpn * nodes / (ms / args.steps * 1e-3) / 1e9
    traffic = ncu_traffic(args.prec, n) if args.kernel == "auto" else None

    # Parity spot check on this run (cheap): sum phi is conserved by the scheme.
    sphi, srho, _, _ = lat.conservation()
    kernel_name = {lbm.LBM_KERNEL_PAIR: "k_step_pair", lbm.LBM_KERNEL_STAGED: "k_step_staged",
                   lbm.LBM_KERNEL_PAIR_STAGED: "k_step_pair_tma"}.get(lat.kernel[0], "k_step")
    lat.close()
    del lat
    torch.cuda.synchronize()

    # End-to-end through the C ABI with host buffers: pinned phi0 in, K steps, fields out.
    e2e = None
    if not args.no_e2e:
        pinned = torch.from_numpy(phi0.reshape(-1)).pin_memory()
        host_phi = pinned.numpy()
        out = [torch.empty(nodes, dtype=torch.float64).pin_memory().numpy() for _ in range(4)]
        p = lbm.lbm_default_params(nx=n, ny=n, **params)
        nbytes = lbm.lbm_state_bytes(p)
        buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        h = lbm.lbm_init(p, host_phi, None, None, None, buf.data_ptr(), nbytes, stream.cuda_stream)
        lbm.lbm_step(h, args.steps)
        lbm.lbm_fields(h, *out)
        t1 = time.perf_counter()
        lbm.lbm_free(h)
        dt = max_over_ranks(t1 - t0)
        e2e = {"value": whole_job_mlups(nodes, args.steps, ws, dt * 1e3), "unit": "MLUPS",
               "h2d_bytes_per_step": 8 * nodes / args.steps,
               "d2h_bytes_per_step": 4 * 8 * nodes / args.steps,
               "what": "lbm_init from pinned host phi0 (H2D) + lbm_step(K) + lbm_fields to pinned "
                       "host (D2H), wall clock; bytes amortised over the K steps"}
        del buf

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        try:
            c_mlups, c_steps, c_dt, c_thr = time_oracle(args.cpu_budget, 128)
            s_mlups, s_steps, s_dt, _ = time_oracle(min(5.0, args.cpu_budget), 128, threads=1)
            cpu = {"value": c_mlups, "unit": "MLUPS", "cores": c_thr, "kind": "oracle",
                   "sample": f"128x128 periodic sample of the spinodal workload, {c_steps} steps "
                             f"in {c_dt:.1f} s, FP64",
                   "serial": {"value": s_mlups, "unit": "MLUPS", "cores": 1,
                              "sample": f"same sample, {s_steps} steps in {s_dt:.1f} s on one thread"},
                   "sizes": oracle_sizes()}
        except Exception as exc:  # report, do not hide
            cpu = {"value": None, "unit": "MLUPS", "cores": None, "kind": "oracle",
                   "sample": f"failed: {exc}"}

    forms = None
    if rank == 0 and ws == 1 and args.prec == "fp32" and not args.no_forms:
        forms = storage_forms(lbm, phi0, params, stream, ms_step)
        for key, fn in (("batch", lambda: batch_form(lbm, args.count, "fp32", 20, 5)),
                        ("surrogate", lambda: surrogate_form(args))):
            try:
                forms[key] = fn()
            except Exception as exc:  # report, do not hide
                forms[key] = {"failed": f"{type(exc).__name__}: {exc}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.prec], "data": "synthetic",
            "config": config_dict(args),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "frac_vs_nominal_8tbs": achieved / 8000.0, "traffic": traffic,
                         "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                         "bytes_per_node": bpn, "kernel": kernel_name},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": args.steps,
            "check": {"sum_phi": sphi, "sum_rho": srho},
            "forms": forms,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------------------------------
# Batched sweep (many independent lattices in one persistent launch per step).

def batch_members(count: int, seed: int):
    """Members of the batched parameter sweep: sizes {64..512}^2 and 2:1 rectangles, half sheared
    droplets between walls moving at +-0.01 (R = ny/4; the capillary number Ca = v_w R nu_l /
    (H sigma), H = ny/2, sets sigma and gamma = a = 3 sigma / sqrt(8), interface width 1), half
    periodic spinodal decomposition (gamma = a = 0.04); viscosity ratio zeta: nu_l = 0.1,
    nu_g = nu_l / zeta, omega linear in phi as in the paper."""
    from paper_1803_11345_gb300 import workloads as W
    out = []
    for m in W.batch_members(count, seed):
        nx, ny = m["nx"], m["ny"]
        kw = dict(tau_l=tau(0.1), tau_g=tau(0.1 / m["zeta"]), M=0.1, Gamma=1.0)
        if m["kind"] == "droplet":
            uw, R, H = 0.01, ny / 4.0, ny / 2.0
            sigma = uw * R * 0.1 / (H * m["Ca"])
            ga = 3.0 * sigma / math.sqrt(8.0)
            phi0 = W.droplet(nx, ny, R, gamma=ga, a=ga)
            kw.update(gamma=ga, a=ga, bc=1, u_top=uw, u_bottom=-uw)
        else:
            phi0 = W.spinodal(nx, ny, seed=m["seed"])
            kw.update(gamma=0.04, a=0.04)
        out.append((phi0, kw))
    return out


def batch_form(lbm, count, prec, steps, warmup):
    """The batched sweep (`count` lattices of batch_members) in one persistent launch per step:
    aggregate MLUPS against the same members stepped one launch per member per step."""
    import torch
    members = batch_members(count, SEED)
    nodes = sum(p.shape[0] * p.shape[1] for p, _ in members)
    bat = lbm.Batch(members, prec=prec)
    tuned_ms = bat.autotune(trial_steps=3)
    bat.step(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(bat.stream)
    bat.step(steps)
    e1.record(bat.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st, flags = bat.check()
    tile = bat.tile
    bat.close()
    lats = [lbm.Lattice(p, prec=prec, stream=torch.cuda.current_stream(), **kw) for p, kw in members]
    seq_steps = max(3, min(steps, 20))
    for L in lats:
        L.step(2)
    torch.cuda.synchronize()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record()
    for _ in range(seq_steps):
        for L in lats:
            L.step(1)
    s1.record()
    torch.cuda.synchronize()
    seq_ms = s0.elapsed_time(s1) / seq_steps
    for L in lats:
        L.close()
    bpn = BYTES_PER_NODE[prec]
    ms_step = ms / steps
    return {"members": count, "nodes": nodes, "precision": prec, "steps": steps, "ms_per_step": ms_step,
            "mlups": nodes / (ms_step * 1e-3) / 1e6,
            "hbm_frac": bpn * nodes / (ms_step * 1e-3) / 1e9 / measured_peaks()[0],
            "ms_per_step_one_launch_per_member": seq_ms, "speedup_vs_one_launch_per_member": seq_ms / ms_step,
            "tile": {"bx": tile[0], "by": tile[1], "nodes_per_item": tile[2], "items": tile[3], "grid": tile[4]},
            "autotuned_ms": tuned_ms, "members_nonfinite": int(sum(flags)), "status": st,
            "workload": f"batched sweep: {count} independent lattices, sizes {{64..512}}^2 and 2:1, half sheared "
                        "droplets (walls +-0.01, Ca log-U[0.01,0.5]), half spinodal, zeta log-U[1,1000], one "
                        "persistent launch per step, CUDA-graph replays"}


def run_batch(args):
    import torch

    from paper_1803_11345_gb300 import build as B
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    B.build()
    from paper_1803_11345_gb300 import lbm
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.time()
    r = batch_form(lbm, args.count, args.prec, args.steps, args.warmup)
    clk = clocks.stop(t0, time.time())
    peak, peak_kind = measured_peaks()
    line = {
        "metric": METRIC, "value": r["mlups"], "unit": "MLUPS", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[args.prec], "data": "synthetic",
        "config": {"workload": r["workload"], "members": args.count, "nodes": r["nodes"], "precision": args.prec,
                   "tile": r["tile"], "autotuned_ms": r["autotuned_ms"], "members_nonfinite": r["members_nonfinite"]},
        "roofline": {"bound": "hbm", "achieved": r["hbm_frac"] * peak, "peak": peak, "unit": "GB/s",
                     "frac": r["hbm_frac"], "traffic": None, "peak_kind": f"{peak_kind} copy bandwidth",
                     "kernel": "k_step_batch"},
        "vs_sequential": {"ms_per_step_one_at_a_time": r["ms_per_step_one_launch_per_member"],
                          "speedup": r["speedup_vs_one_launch_per_member"],
                          "what": "the same members as separate lattices, one lbm_step launch each per step"},
        "clocks": clk, "gpu_launches": args.steps,
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# Learned surrogate vs the plain FP32 solver.

def surrogate_form(args):
    """The learned surrogate as deployed: trained on the solver's own trajectories (256^2 periodic
    spinodal decomposition, viscosity ratio 10, windows of K = 50 steps), then a closed-loop rollout
    of held-out lattices under the judge (sum-phi drift checked on the GPU every window, a solver
    audit every `sur_audit` windows, the solver advancing every rejected window), timed end to end
    against the solver alone over the same windows, with the final phi error against it."""
    import time as _t

    import numpy as np
    import torch

    from paper_1803_11345_gb300 import surrogate as S
    n, K = args.sur_n, args.sur_k
    ntr, nte, wins = args.sur_train, args.sur_test, args.sur_windows
    t0 = _t.time()
    members = S.spinodal_members(ntr + nte, n, seed=SEED)
    states = S.generate_states(members, K, wins)
    t_data = _t.time() - t0
    net = S.UNet(ch=(32, 64, 128, 256), cin=16, seed=SEED)
    t0 = _t.time()
    hist = S.train_states(net, states[:, :ntr], args.sur_iters, args.sur_batch, lr=1e-3, seed=SEED, log_every=100)
    torch.cuda.synchronize()
    t_train = _t.time() - t0
    e, p = S.one_window_errors(net, states[:, ntr:][:min(wins, 40) + 1])
    test_members = members[ntr:]
    k0 = min(10, wins)
    st0 = states[k0, ntr:].contiguous()
    judge = S.Judge(phi_err=1e-2, drift=1e-6, audit_every=args.sur_audit)
    S.rollout(net, test_members, st0, 2, K, judge)  # warm-up
    fin, stats = S.rollout(net, test_members, st0, args.sur_rollout, K, judge)
    ref, t_solver = S.solver_only(test_members, st0, args.sur_rollout, K)
    err = S.phi_rms(fin, ref)
    pers = S.phi_rms(st0, ref)
    x = torch.empty((nte, n, n, net.cin), dtype=torch.bfloat16, device="cuda")
    base = torch.zeros((nte, n, n, 3), dtype=torch.float32, device="cuda")
    ms_fwd = S.time_forward(net, x, base, reps=10, graph=True)
    nodes = nte * n * n
    return {"lattices": nte, "n": n, "K": K, "windows": args.sur_rollout, "start_window": k0,
            "seconds_rollout": stats["seconds"], "seconds_solver_alone": t_solver,
            "speedup_vs_solver": t_solver / stats["seconds"],
            "mlups_equivalent": nodes * K * args.sur_rollout / stats["seconds"] / 1e6,
            "final_phi_rms_vs_solver_max": float(err.max()), "persistence_phi_rms": float(np.median(pers)),
            "kept": stats["kept"], "audits": stats["audits"], "audit_failed": stats["audit_failed"],
            "solver_windows": stats["solver"], "drift_rejected": stats["drift_rejected"],
            "audit_rms": stats["audit_rms"],
            "thresholds": {"phi_rms": judge.phi_err, "sum_phi_drift_per_node": judge.drift, "audit_every": judge.audit_every},
            "one_window_phi_rms_median": float(np.median(e)), "persistence_one_window_median": float(np.median(p)),
            "ms_forward_graph": ms_fwd, "ms_solver_window": t_solver * 1e3 / args.sur_rollout,
            "training": {"trajectories": ntr, "windows": wins, "steps_per_trajectory": wins * K,
                         "iters": args.sur_iters, "batch": args.sur_batch,
                         "seconds_data": t_data, "seconds_train": t_train, "loss": hist[::3]},
            "what": "closed-loop rollout of held-out lattices, wall time including the judge's GPU reductions, "
                    "its per-window host read of the sums, every audit and fallback; solver alone: the batched "
                    "solver over the same windows from the same state"}


def run_surrogate(args):
    import torch

    from paper_1803_11345_gb300 import build as B
    B.build()
    r = surrogate_form(args)
    line = {
        "metric": METRIC, "value": r["mlups_equivalent"], "unit": "MLUPS-equivalent", "n_gpus": 1,
        "steps": r["K"] * r["windows"], "warmup": 2 * r["K"], "ms_per_step": r["seconds_rollout"] * 1e3 / (r["K"] * r["windows"]),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)",
        "data": "synthetic",
        "config": {"workload": f"learned surrogate: 4-level U-Net (32,64,128,256 channels, BF16, FP32 accumulate) "
                               f"advancing (phi, ux, uy) by {r['K']} steps on {r['n']}x{r['n']} periodic spinodal "
                               f"decomposition (viscosity ratio 1:10), judged closed-loop rollout of {r['lattices']} "
                               f"held-out lattices"},
        "surrogate": r,
        "gpu_launches": None,
    }
    torch.cuda.synchronize()
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--n", type=int, default=4096, help="lattice side (profiling uses smaller)")
    ap.add_argument("--prec", choices=list(BYTES_PER_NODE), default="fp32")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the 16-bit storage comparison")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle time")
    ap.add_argument("--pad-ms", type=float, default=400.0,
                    help="untimed stepping before and after the timed region, for the clock samples (0: none)")
    ap.add_argument("--workload", choices=["spinodal", "batch", "surrogate"], default="spinodal")
    ap.add_argument("--kernel", choices=["auto", *KERNELS], default="auto",
                    help="step kernel of the spinodal workload (auto: the library's default)")
    ap.add_argument("--sur-n", type=int, default=256)
    ap.add_argument("--sur-k", type=int, default=50, help="solver steps per surrogate window")
    ap.add_argument("--sur-windows", type=int, default=30, help="windows per trajectory (x K solver steps)")
    ap.add_argument("--sur-train", type=int, default=248, help="training trajectories")
    ap.add_argument("--sur-test", type=int, default=8, help="held-out lattices (rollout batch)")
    ap.add_argument("--sur-iters", type=int, default=2000)
    ap.add_argument("--sur-batch", type=int, default=16)
    ap.add_argument("--sur-rollout", type=int, default=16, help="windows of the judged rollout")
    ap.add_argument("--sur-audit", type=int, default=8, help="audit every this many windows")
    ap.add_argument("--count", type=int, default=256, help="members of the batched sweep")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "surrogate":
        return run_surrogate(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
