"""Benchmark of the calibration hot path on GB300; prints one JSON line.

Workload (default, the single-window FP32 configuration): 60-day window, transmission rate
piecewise constant over 4 segments (7 parameters with gamma, mu, I0), log-uniform PSO box,
4096 particles, 1000 PSO iterations, Euler at dt = 0.1 day, FP32 trajectories with a Kahan
loss, FP64 re-evaluation of the 32 best personal bests.  One step = one full calibration
(initialisation, 1000 fused PSO iterations, top-k, FP64 re-evaluation) on synthetic deaths
(Poisson-noised Euler curve at ground-truth rates, N = 38e6).

Metric: particle-day ODE steps per second = particles x days x PSO iterations / second
(the initial evaluation and the FP64 re-evaluation are extra work, not counted).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload c2|c1|c5]

With --gpus N > 1 (one process per GPU under torchrun) every rank calibrates its own
independent replica (its own Philox stream word, as in repeated calibrations of one
window); there is no data-path collective, and value = all ranks' particle-days / the
slowest rank's time (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2204_12346_gb300 import configs, synth  # noqa: E402

METRIC = "particle-day ODE steps/sec"
UNIT = "particle-days/s"

# FP32 peak from unit counts: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2070 MHz max SM clock.
SMS, FP32_LANES, MAX_SM_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = SMS * FP32_LANES * 2 * MAX_SM_MHZ * 1e6 / 1e12


# DRAM bytes per launch of the dominant kernel from the committed ncu capture
# (profiles/pso_f32_persistent_c2.md), valid only for the kernel sources it was taken on.
PROFILED_KERNEL_FILES = ["pso_persistent.cu", "sird_model.cuh", "device_common.cuh", "kernels.h"]
PROFILED = {"sha": "ea40821fd8e456d2", "traffic_bytes": 727296, "profile": "profiles/pso_f32_persistent_c2.md"}


def kernel_sources_sha() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in PROFILED_KERNEL_FILES:
        with open(os.path.join(ROOT, "paper_2204_12346_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def algorithmic_flops_per_particle_day(spd: int) -> int:
    """8 flops per Euler step (S = N - C, inf = cb*S*I, C += inf, I += inf - a*I, D += dm*I with
    FMA counted as 2) times steps per day, plus 3 for the day's error and its square-sum."""
    return 8 * spd + 3


def workload(name: str):
    c = dict(configs.CONFIGS[name])
    ser = synth.load_series(c["series"])
    days = c["days"]
    y = ser["yD"][: days + 1]
    lb, ub = configs.bounds(c["K"], c["log"])
    return c, ser, y, lb, ub


def describe(c) -> str:
    if c["series"] == "c2":
        return ("single window FP32 + Kahan loss: 60 days, beta piecewise constant over 4 segments (7 params), "
                "log-uniform PSO box, 4096 particles, 1000 iterations, dt=0.1, FP64 re-evaluation of the 32 best")
    if c["series"] == "c1":
        return "plain method FP64: constant beta, gamma, mu + I0, 30 days, 64 particles, 200 iterations, dt=0.1"
    return f"{c['name']}: K={c['K']}, {c['days']} days, {c['M']} particles, {c['iters']} iterations, spd={c['spd']}"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        if self.proc is None or self.f is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ our arm

def flush_l2(buf):
    buf.add_(1.0)  # 256 MiB write, larger than the 129 MB L2


def run_ours(args, rank: int, world: int) -> dict | None:
    import torch

    from paper_2204_12346_gb300 import sird

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    c, ser, y, lb, ub = workload(args.workload)
    log = [1] * len(lb) if c["log"] else None
    stream = torch.cuda.Stream()
    kw = dict(K=c["K"], spd=c["spd"], particles=c["M"], iters=c["iters"], lb=lb, ub=ub, log_scale=log,
              precision=c["precision"], seed=c["seed"], stream_id=rank, reeval_topk=c.get("reeval_topk", 0))
    with torch.cuda.stream(stream):
        cal = sird.Calibrator(y, ser["N"], stream=stream, **kw)
        ev_it0, ev_it1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev_it0.record(stream)  # torch only reads events it has seen recorded once; the graph re-records them
        ev_it1.record(stream)
        cal.set_timing(ev_it0, ev_it1)
        flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
        for _ in range(args.warmup):
            res = cal.calibrate()
        L = c["days"]
        units_per_step = c["M"] * L * c["iters"]
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        iter_ms = []
        _barrier(world)
        torch.cuda.synchronize()
        with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clk:
            for i in range(args.steps):
                flush_l2(flush)
                starts[i].record(stream)
                res = cal.calibrate()
                ends[i].record(stream)
                torch.cuda.synchronize()
                iter_ms.append(ev_it0.elapsed_time(ev_it1))
        torch.cuda.synchronize()
        _barrier(world)
        step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        total_ms = _max_over_ranks(sum(step_ms), world)

        # end to end through the public API with host buffers: upload this step's observations
        # from host memory, calibrate, read the result back (the result struct is the output)
        e2e_ms = []
        y_host = np.asarray(y, dtype=np.float64)
        for i in range(args.steps):
            flush_l2(flush)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cal.set_observations(y_host)
            r2 = cal.calibrate()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        e2e_total = _max_over_ranks(sum(e2e_ms), world)
        assert r2["loss"] == res["loss"]

    if rank != 0:
        return None
    value = units_per_step * args.steps * world / (total_ms / 1e3)
    e2e_value = units_per_step * args.steps * world / (e2e_total / 1e3)
    spd = c["spd"]
    flops_per_launch = c["M"] * L * algorithmic_flops_per_particle_day(spd)
    avg_iter_ms = statistics.mean(iter_ms) / c["iters"]
    achieved_tflops = flops_per_launch / (avg_iter_ms / 1e3) / 1e12
    n_obs = L + 1
    h2d = n_obs * (4 + 4 + 8)
    d2h = 8 * 32 + 8 * 3 + 8  # ResultDev
    topk_passes = 1 if c.get("reeval_topk", 0) else 0
    persistent = cal.launch_mode == sird.LAUNCH_PERSISTENT
    iter_launches = 1 if persistent else c["iters"]
    launches = args.steps * (1 + iter_launches + topk_passes + 1)
    kernel = ("pso_f32_persistent (all iterations in one cooperative launch)" if persistent
              else "pso_f32_kernel (one fused PSO iteration per launch)")
    launch_us = statistics.mean(iter_ms) * 1e3 / iter_launches
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if c["precision"] == 32 else "f64", "data": "synthetic",
        "config": {"workload": describe(c), "name": c["name"], "particles": c["M"], "days": L,
                   "iterations": c["iters"], "steps_per_day": spd, "params": len(lb),
                   "l2": "flushed between timed steps (256 MiB write); the 1000 iterations inside one "
                         "calibration keep the swarm resident in L2 by design",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved_tflops / FP32_PEAK_TFLOPS,
                     "traffic": (PROFILED["traffic_bytes"] if persistent and args.workload == "c2"
                                 and kernel_sources_sha() == PROFILED["sha"] else None),
                     "traffic_source": PROFILED["profile"],
                     "kernel": kernel, "avg_launch_us": launch_us, "us_per_iteration": avg_iter_ms * 1e3,
                     "flops_per_launch": flops_per_launch * c["iters"] / iter_launches,
                     "peak_basis": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_total / args.steps},
        "gpu_launches": launches,
        "result": {"loss_fp64": res["loss"], "loss_search": res["loss_search"], "r2_D": res["r2_D"],
                   "theta": [float(v) for v in res["theta"]]},
    }
    out["clocks"] = clk.summary()
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, budget_s=args.cpu_budget)
    return out


def _barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def _max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ oracle on the host cores

def cpu_baseline(name: str, budget_s: float = 15.0, iters_cap: int | None = None) -> dict:
    """The FP64 oracle as it stands, single-threaded, on a bounded sample of the workload:
    the same swarm (all particles) for as many PSO iterations as fit in about budget_s."""
    import oracle as O

    c, ser, y, lb, ub = workload(name)
    K = c["K"]
    logd = [1] * len(lb) if c["log"] else [0] * len(lb)
    zlb = np.log(lb) if c["log"] else np.array(lb, float)
    zub = np.log(ub) if c["log"] else np.array(ub, float)
    pb = O.Problem(yD=y, N=ser["N"], K=K, spd=c["spd"])
    pso = O.PSO(pb, c["M"], zlb, zub, logdim=logd, seed=c["seed"], store_f32=c["precision"] == 32)
    t0 = time.perf_counter()
    pso.init()
    its = 0
    while time.perf_counter() - t0 < budget_s and (iters_cap is None or its < iters_cap):
        pso.step(1)
        its += 1
    dt = time.perf_counter() - t0
    units = c["M"] * c["days"] * (its + 1)
    return {"value": units / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{c['M']} particles x {c['days']} days, init + {its} PSO iterations "
                      f"({dt:.1f} s, single thread, FP64)"}


def run_reference(args, rank: int, world: int) -> dict | None:
    if rank != 0:
        return None
    c, ser, y, lb, ub = workload(args.workload)
    per_step = []
    import oracle as O

    O.build()
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(args.workload, budget_s=0.0, iters_cap=args.ref_iters)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            per_step.append((cb, dt))
    units = sum(c["M"] * c["days"] * (args.ref_iters + 1) for _ in per_step)
    secs = sum(dt for _, dt in per_step)
    value = units / secs
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / len(per_step) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": describe(c), "name": c["name"],
                   "sample": f"each step: init + {args.ref_iters} PSO iterations of the full swarm"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{c['M']} particles x {c['days']} days x (init + {args.ref_iters} iterations) "
                                   f"per step, single thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["c1", "c2", "c5"], default="c2")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-iters", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    try:
        out = run_ours(args, rank, world) if args.impl == "ours" else run_reference(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
