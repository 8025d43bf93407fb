"""Benchmark of the calibration hot path on GB300; prints one JSON line.

Default workload (the batched FP32 configuration): 512 rolling windows cut from a 450-day
synthetic series, window lengths uniform in 21..90 days, swarms of 256..2048 particles,
transmission rate piecewise constant over 6 segments (9 parameters with gamma, mu, I0),
log-uniform PSO box, 100 PSO iterations, Euler at dt = 0.1 day, FP32 trajectories with a Kahan
loss, one persistent launch captured in a CUDA graph with autotuned block shape, FP64
re-evaluation of every window's global best.  One step = one such batched calibration.

Metric: particle-day ODE steps per second = sum over windows of particles x days, times PSO
iterations, per second (the initial evaluation and the FP64 re-evaluation are extra work, not
counted).  The metric's second part, seconds to calibrate at fixed loss, is measured on the
single 60-day window: the plain FP64 swarm (4096 particles, 1000 iterations) sets the loss
L_ref; the FP32 swarm followed by the L-BFGS polish (FP32 trials and adjoint gradient, FP64
re-scoring of the result) must reach (1 + 1e-6) L_ref.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload batch512|window60|plain64|gradient90|swarm2p20|paper|paper_ird|stability]

With --gpus N > 1 every rank (one process per GPU; started here through torch.distributed.run
unless an outer launcher already set WORLD_SIZE, which must then equal N) calibrates its own batch
of windows (its own Philox stream words); there is no data-path collective, and value = all
ranks' particle-days / the slowest rank's time (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
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

# DRAM bytes per launch of the dominant kernel from committed ncu captures, valid only for the
# kernel sources they were taken on (sha256[:16] of the files listed).
PROFILED = {
    "batch512": {"files": ["batched.cu", "traj_f32.cuh", "sird_model.cuh", "device_common.cuh", "kernels.h"],
           "sha": "e82eef7ec000d386", "traffic_bytes": 12888576, "fma_pipe": 0.6128,
           "profile": "profiles/pso_batch_f32_batch512.md"},
    "window60": {"files": ["pso_persistent.cu", "traj_f32.cuh", "sird_model.cuh", "device_common.cuh", "kernels.h"],
           "sha": "dc2f1813dbce77c6", "traffic_bytes": 478464, "fma_pipe": 0.3180,
           "profile": "profiles/pso_f32_persistent_window60.md"},
    "gradient90": {"files": ["adjoint_f32.cu", "traj_f32.cuh", "sird_model.cuh", "device_common.cuh", "kernels.h"],
           "sha": "69a9d7c0c61d445b", "traffic_bytes": 182784, "fma_pipe": 0.0751,
           "profile": "profiles/loss_grad_f32_gradient90.md"},
    "paper": {"files": ["batched.cu", "traj_f32.cuh", "sird_model.cuh", "device_common.cuh", "kernels.h"],
           "sha": "e82eef7ec000d386", "traffic_bytes": 15183807000, "fma_pipe": 0.5143,
           "profile": "profiles/pso_batch_f32_paper.md"},
    "paper_ird": {"files": ["batched.cu", "traj_f32.cuh", "sird_model.cuh", "device_common.cuh", "kernels.h"],
           "sha": "e82eef7ec000d386", "traffic_bytes": 15357156000, "fma_pipe": 0.5173,
           "profile": "profiles/pso_batch_f32_paper_ird.md"},
    "stability": {"files": ["batched.cu", "traj_f32.cuh", "sird_model.cuh", "device_common.cuh", "kernels.h"],
           "sha": "e82eef7ec000d386", "traffic_bytes": 300685507328, "fma_pipe": 0.5305,
           "profile": "profiles/pso_batch_f32_stability.md"},
    "swarm2p20": {"files": ["pso_kernels.cu", "traj_f32.cuh", "sird_model.cuh", "device_common.cuh", "kernels.h"],
           "sha": "4c27a2f29190ec1e", "traffic_bytes": 275710720, "fma_pipe": 0.7650,
           "profile": "profiles/pso_f32_kernel_swarm2p20.md"},
}


def kernel_sources_sha(files) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2204_12346_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, key: str = "traffic_bytes"):
    """A figure of the committed ncu capture of the workload's dominant kernel (DRAM bytes per
    launch, or the FMA pipe's active fraction), or None once the kernel sources have changed."""
    p = PROFILED.get(workload)
    if not p or p["sha"] is None or kernel_sources_sha(p["files"]) != p["sha"]:
        return None
    return p[key]


def algorithmic_flops_per_particle_day(spd: int, ramp: bool = False, ird: bool = False) -> int:
    """8 flops per Euler step (S = N - C, inf = cb*S*I, C += inf, I += inf - a*I, D += dm*I with
    FMA counted as 2) times steps per day, plus 3 for the day's error and its square-sum; the
    ramp form of eq. (beta) adds 5 per step (t = k dt, beta on the ramp, cb = beta dt/N), the
    F_IRD objective 2 per step (R += dr*I) and the I and R errors each day."""
    per_step = 8 + (5 if ramp else 0) + (2 if ird else 0)
    return per_step * spd + (9 if ird else 3)


# Bytes of one window's result record copied back by a batched calibration.
BATCH_OUT_BYTES = 408

# Gradient: 8 flops forward, 8 to recompute the stretch from its checkpoint, 20 in the
# reverse step (lambda_S, lambda_I and the three parameter sums, FMA counted as 2).
GRAD_FLOPS_PER_STEP = 36


def single_window(name: str):
    c = dict(configs.CONFIGS[name])
    ser = synth.load_series(c["series"])
    y = ser["yD"][: c["days"] + 1]
    lb, ub = configs.bounds(c["K"], c["log"])
    return c, ser, y, lb, ub


BATCHED = ("batch512", "paper", "paper_ird")

# The paper's own timing (context only: other hardware, real data, time per PSO iteration of one
# window with 10000 particles on F_IRD^MXSE): 2.176 s on a TITAN V, 55.655 s on a Xeon E5-2650 v4.
PAPER_GPU_S_PER_ITERATION = 2.176


def batch_windows(name: str, seed_offset: int = 0):
    """(config, windows, lb, ub, model keywords) of a batched workload; rank r's windows use the
    Philox stream words r*W .. r*W + W - 1."""
    c = dict(configs.CONFIGS[name])
    ser = synth.load_series(c["series"])
    fit_I0 = c.get("fit_I0", True)
    ird = c.get("objective") == "ird"
    if ird or not fit_I0:  # reported I and R: observed series, or the windows' initial state
        ser = synth.reported_IR(ser, c["seed"])
    lay = synth.rolling_windows(W=c["W"], L_min=c["L_min"], L_max=c["L_max"], M_min=c["M_min"], M_max=c["M_max"],
                                delta=c["delta"], seed=c["seed"])
    wins = synth.rolling_window_problems(ser, lay)
    for i, w in enumerate(wins):
        w["seed"] = c["seed"]
        w["stream_id"] = seed_offset * c["W"] + i
        if not ird:  # F_D fits deaths only
            w.pop("yI", None)
            w.pop("yR", None)
    if c.get("beta_form") == "ramp":
        lb, ub = configs.bounds_ramp(fit_I0=fit_I0)
        model = dict(K=1, beta_form=1, log_scale=None)
    else:
        lb, ub = configs.bounds(c["K"], c["log"])
        model = dict(K=c["K"], beta_form=0, log_scale=[1] * len(lb) if c["log"] else None)
    model["fit_I0"] = fit_I0
    model["objective"] = 1 if ird else 0
    model["cost"] = {"mse": 0, "mxse": 1, "mae": 2, "mape": 3}[c.get("cost", "mse")]
    return c, wins, lb, ub, model


def describe(name: str) -> str:
    return {
        "batch512": ("batched FP32: 512 rolling windows of 21..90 days cut from a 450-day series, 256..2048 particles "
               "per window, beta piecewise constant over 6 segments (9 params), log-uniform PSO box, 100 iterations, "
               "dt=0.1, one persistent launch in a CUDA graph, autotuned block shape, FP64 re-evaluation per window"),
        "window60": ("single window FP32 + Kahan loss: 60 days, beta piecewise constant over 4 segments (7 params), "
               "log-uniform PSO box, 4096 particles, 1000 iterations, dt=0.1, FP64 re-evaluation of the 32 best"),
        "plain64": "plain method FP64: constant beta, gamma, mu + I0, 30 days, 64 particles, 200 iterations, dt=0.1",
        "paper": ("the paper's setting, batched FP32: ramp beta(t) (beta1, beta2, t1, t2, gamma, mu; initial state from "
                  "the reported I, R, D of the window's first day), 139 "
                  "rolling windows of 35 days shifted by 3 days over a 450-day series, 10000 particles per window, "
                  "linear PSO box, 100 iterations, dt=0.1, one persistent launch, FP64 re-evaluation per window"),
        "paper_ird": ("the paper's setting on its representative objective F_IRD^MXSE, batched FP32: ramp beta(t), "
                      "139 rolling 35-day windows shifted by 3 days, reported I, R, D (the initial state from their first "
                      "day), 10000 particles per window, "
                      "linear PSO box, 100 iterations, dt=0.1, one persistent launch, FP64 re-evaluation per window"),
        "stability": ("the paper's stability test (Sec. 4.2): 2 windows of 35 days each calibrated 1000 times "
                      "(independent Philox streams, 10000 particles, ramp beta(t), F_IRD^MXSE, 100 iterations) in "
                      "one batched launch, then per day the median and 95/90/50% bands of beta, R0, S, I, R, D over "
                      "the window and a 21-day extension (FP64 ensemble integration, on-device sort)"),
        "gradient90": ("gradient FP32: loss + exact gradient (discrete adjoint of the compensated FP32 trajectory, "
               "day-start checkpoints) of the 4096 personal bests of a calibrated swarm, 90 days, 4 beta segments "
               "(7 params), dt=0.05"),
        "swarm2p20": ("large FP32: 2^20 particles, 10 segments (13 params), 120 days, dt=0.05, 100 iterations, FP64 "
               "re-evaluation of the 32 best, 20 FP32 L-BFGS iterations (adjoint gradient) on the 32 best, then the "
               "1024 best personal bests forecast 14 held-out days (FP64)"),
    }[name]


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


def flush_l2(buf):
    buf.add_(1.0)  # 256 MiB write, larger than the 129 MB L2


def _barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def _max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def timed_steps(args, world, stream, step_fn, kernel_events=None):
    """Runs args.steps steps with an L2 flush before each, timed by CUDA events on `stream`.
    Returns (total ms max over ranks, per-step kernel ms from kernel_events -- the step's own
    events when None --, clocks, last result)."""
    import torch

    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kern_ms = []
    res = None
    _barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush_l2(flush)
            starts[i].record(stream)
            res = step_fn()
            ends[i].record(stream)
            torch.cuda.synchronize()
            kev = kernel_events or (starts[i], ends[i])
            kern_ms.append(kev[0].elapsed_time(kev[1]))
    torch.cuda.synchronize()
    _barrier(world)
    total = _max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), world)
    return total, kern_ms, clk.summary(), res


# ------------------------------------------------------------------ seconds to calibrate

def s_to_calibrate() -> dict:
    """Single 60-day window: wall seconds of the plain FP64 swarm (1000 iterations; its final loss
    is L_ref) vs the FP32 swarm plus the FP32 L-BFGS polish of its 32 best until the FP64 loss is
    <= (1 + 1e-6) L_ref.  The FP32 swarm runs 100, 200, 500 or 1000 iterations; for each, the
    polish iterations grow until the target is reached; the line reports the fastest setting that
    reaches it (every trial is listed)."""
    import torch

    from paper_2204_12346_gb300 import sird

    c, ser, y, lb, ub = single_window("window60")
    kw = dict(K=c["K"], spd=c["spd"], particles=c["M"], lb=lb, ub=ub, log_scale=[1] * len(lb), seed=c["seed"])
    c64 = sird.Calibrator(y, ser["N"], precision=64, iters=c["iters"], **kw)
    c64.calibrate()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r64 = c64.calibrate()
    t64 = time.perf_counter() - t0
    target = r64["loss"] * (1 + 1e-6)
    out = {"window": "60 days, 4 segments, 4096 particles, 1000 FP64 PSO iterations, dt=0.1", "L_ref": r64["loss"],
           "target": "(1 + 1e-6) L_ref", "fp64_pso_s": t64, "trials": []}
    best = None
    for iters in (100, 200, 500, c["iters"]):
        c32 = sird.Calibrator(y, ser["N"], precision=32, iters=iters, reeval_topk=32, **kw)
        c32.calibrate()
        c32.polish(k=32, iters=5, first_step=1e-2, precision=32)  # warm-up: the first polish sets up its buffers
        for n in (0, 5, 10, 15, 20, 30, 40, 50, 75, 100, 150, 200, 300):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r32 = c32.calibrate()
            loss = r32["loss"]
            if n > 0:
                rp = c32.polish(k=32, iters=n, first_step=1e-2, precision=32)
                loss = min(loss, rp["loss"])
            dt = time.perf_counter() - t0
            ok = loss <= target
            out["trials"].append({"swarm_iters": iters, "polish_iters": n, "s": dt, "loss_over_L_ref": loss / r64["loss"],
                                  "reached": ok})
            if ok:
                if best is None or dt < best["s"]:
                    best = {"s": dt, "swarm_iters": iters, "polish_iters": n, "loss": loss}
                break
    if best is None:
        out.update({"reached": False})
        return out
    out.update({"fp32_plus_polish_s": best["s"], "swarm_iters": best["swarm_iters"], "polish_iters": best["polish_iters"],
                "loss_reached": best["loss"], "speedup": t64 / best["s"], "reached": True})
    return out


def s_to_calibrate_batch(batch, c, wins, lb, ub, model, stride=32) -> dict:
    """A batch of windows (the 512-window batch, or the paper's 139 windows on F_IRD^MXSE): on every
    stride-th window (a subsample spanning the batch) the plain FP64 swarm -- the window's own
    particles and Philox stream, 10x the batch's PSO iterations -- sets L_ref; then the wall
    seconds of the batched FP32 swarm followed by the batched L-BFGS polish of every window's k
    best personal bests (FP32 trials and adjoint, FP64 re-scoring) until every subsampled window's
    FP64 loss is <= (1 + 1e-6) L_ref; the schedule tries 32 candidates per window first, then 128,
    then the FP32 swarm with the reference's iteration count and 2x and 4x that (with and without the
    polish)."""
    import torch

    from paper_2204_12346_gb300 import sird

    sub = list(range(0, len(wins), stride))
    it64 = 10 * c["iters"]
    t64, ref = 0.0, {}
    for i in sub:
        w = wins[i]
        ird = model["objective"] == 1
        cal = sird.Calibrator(w["yD"], w["N"], R0=w["R0"], I0=w.get("I0", 0.0), particles=w["particles"], iters=it64,
                              precision=64, seed=w["seed"], stream_id=w["stream_id"], spd=c["spd"], lb=lb, ub=ub,
                              K=model["K"], beta_form=model["beta_form"], log_scale=model["log_scale"],
                              fit_I0=model["fit_I0"], cost=model["cost"], objective=model["objective"],
                              yI=w["yI"] if ird else None, yR=w["yR"] if ird else None)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ref[i] = cal.calibrate()["loss"]
        torch.cuda.synchronize()
        t64 += time.perf_counter() - t0
    pd = {i: wins[i]["particles"] * wins[i]["L"] for i in range(len(wins))}
    scale = sum(pd.values()) / sum(pd[i] for i in sub)  # FP64 seconds scale with particle-days
    out = {"windows": f"every {stride}th of {len(wins)} ({len(sub)} windows, {min(wins[i]['L'] for i in sub)}.."
                      f"{max(wins[i]['L'] for i in sub)} days)",
           "L_ref": f"plain FP64 swarm, {it64} iterations, the window's own particles and stream",
           "target": "(1 + 1e-6) L_ref on every subsampled window",
           "fp64_pso_s_subsample": t64, "fp64_pso_s_all_windows_est": t64 * scale, "trials": []}
    # the batch's own iterations with the polish first; then (for objectives whose kinks stall the
    # polish, such as F_IRD^MXSE) the FP32 batched swarm run for the FP64 reference's iterations
    long_batches = {}
    # (swarm iterations / the batch's, polish candidates, polish iterations, polish first step)
    schedule = [(1, 32, 0, 1e-2), (1, 32, 10, 1e-2), (1, 32, 20, 1e-2), (1, 32, 40, 1e-2), (1, 128, 20, 1e-2),
                (1, 128, 40, 1e-2), (1, 128, 80, 1e-2), (1, 128, 160, 1e-2), (1, 128, 80, 1e-3), (1, 128, 80, 1e-4),
                (10, 32, 0, 1e-2), (10, 32, 20, 1e-2), (10, 128, 40, 1e-2), (10, 128, 80, 1e-3), (10, 128, 80, 1e-4),
                (20, 32, 0, 1e-2), (20, 128, 40, 1e-2), (40, 32, 0, 1e-2), (40, 128, 40, 1e-2)]
    for mult, k, n, fs in schedule:
        b = batch
        if mult != 1:
            if mult not in long_batches:
                long_batches.clear()  # one longer batch at a time
                long_batches[mult] = sird.Batch(wins, spd=c["spd"], iters=mult * c["iters"], lb=lb, ub=ub,
                                                stream=torch.cuda.current_stream(), **model)
                long_batches[mult].calibrate()  # warm-up (the autotuner runs at creation)
            b = long_batches[mult]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = b.calibrate()
        t_swarm = time.perf_counter() - t0
        pol = b.polish(k=k, iters=n, first_step=fs) if n else res
        dt = time.perf_counter() - t0
        got = {i: min(res[i]["loss"], pol[i]["loss"]) for i in sub}
        ok = [got[i] <= ref[i] * (1 + 1e-6) for i in sub]
        frac = sum(ok) / len(sub)
        out["trials"].append({"swarm_iters": mult * c["iters"], "polish_k": k, "polish_iters": n, "first_step": fs,
                              "s": dt, "swarm_s": t_swarm, "fraction_reached": frac,
                              "median_loss_over_L_ref": float(np.median([got[i] / ref[i] for i in sub]))})
        if frac == 1.0:
            out.update({"fp32_batch_plus_polish_s": dt, "swarm_iters": mult * c["iters"], "polish_k": k,
                        "polish_iters": n, "first_step": fs, "reached": True,
                        "speedup_vs_fp64_all_windows_est": t64 * scale / dt})
            return out
    # not reached: the trial that reached the most windows (the fastest among equals)
    top = min(out["trials"], key=lambda t: (-t["fraction_reached"], t["s"]))
    out.update({"reached": False, "fraction_reached": top["fraction_reached"], "fp32_batch_plus_polish_s": top["s"],
                "best_trial": top})
    return out


# ------------------------------------------------------------------ our arm

def run_batched(args, rank, world):
    import torch

    from paper_2204_12346_gb300 import sird

    name = args.workload
    c, wins, lb, ub, model = batch_windows(name, rank)
    ramp = model["beta_form"] == 1
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch = sird.Batch(wins, spd=c["spd"], iters=c["iters"], lb=lb, ub=ub, block_size=args.block, stream=stream,
                           **model)
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record(stream)  # torch reads only events it has seen recorded; the graph re-records them
        ev[1].record(stream)
        batch.set_timing(*ev)
        for _ in range(args.warmup):
            batch.calibrate()
    total_ms, kern_ms, clocks, res = timed_steps(args, world, stream, batch.calibrate, ev)

    # end to end through the public API with host buffers: every step uploads all windows'
    # observations (and the windows' settings that depend on them) from host memory, calibrates
    # and copies every window's result back (the daily re-calibration of a serving loop)
    y_host = np.concatenate([np.concatenate([w["yD"], w["yI"], w["yR"]]) if model["objective"] == 1
                             else np.asarray(w["yD"], dtype=np.float64) for w in wins])
    e2e, h2d = [], 0
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2d = batch.set_observations(y_host)
        batch.calibrate()
        e2e.append((time.perf_counter() - t0) * 1e3)
    e2e_total = _max_over_ranks(sum(e2e), world)
    if rank != 0:
        return None
    pdays = sum(w["particles"] * w["L"] for w in wins)
    units = pdays * c["iters"]
    flops = pdays * algorithmic_flops_per_particle_day(c["spd"], ramp, model["objective"] == 1) * (c["iters"] + 1)
    kms = statistics.mean(kern_ms)
    achieved = flops / (kms / 1e3) / 1e12
    d2h = len(wins) * BATCH_OUT_BYTES
    out = {
        "metric": METRIC, "value": units * args.steps * world / (total_ms / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": describe(name), "name": c["name"], "windows": len(wins),
                   "particle_days_per_iteration": pdays, "iterations": c["iters"], "steps_per_day": c["spd"],
                   "params": len(lb), "block": f"{batch.block_size} threads x {batch.blocks_per_sm} per SM, "
                                               + ("flat" if batch.launch_mode == sird.LAUNCH_FLAT
                                                  else "one window per block")
                                               + (" (autotuned)" if args.block == 0 else " (given)"),
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"independent batches x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": profiled_traffic(name),
                     "traffic_source": PROFILED.get(name, {}).get("profile"),
                     "kernel": "pso_flat_f32" if batch.launch_mode == sird.LAUNCH_FLAT else "pso_batch_f32",
                     "ncu_fma_pipe_active": profiled_traffic(name, "fma_pipe"),
                     "avg_launch_us": kms * 1e3, "flops_per_launch": flops,
                     "peak_basis": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"},
        "e2e": {"value": units * args.steps * world / (e2e_total / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_total / args.steps},
        "gpu_launches": args.steps * 2,
        "clocks": clocks,
        "result": {"windows": len(res), "median_r2_D": float(np.median([r["r2_D"] for r in res])),
                   "min_r2_D": float(np.min([r["r2_D"] for r in res])),
                   "window0_loss_fp64": res[0]["loss"]},
    }
    if name.startswith("paper"):
        per_it = (total_ms / args.steps / 1e3) / (len(wins) * (c["iters"] + 1))
        out["result"]["paper_context"] = {
            "s_per_pso_iteration_per_window": per_it,
            "paper_gpu_s_per_pso_iteration": PAPER_GPU_S_PER_ITERATION,
            "note": "the paper's figure is one window's PSO iteration (10000 particles, F_IRD^MXSE, real data) on a "
                    "TITAN V with the cost on the CPU; ours is the batch's wall time spread over its window-iterations"}
    if not args.no_s2c and name == "batch512":
        out["s_to_calibrate"] = s_to_calibrate()
        with torch.cuda.stream(stream):
            out["s_to_calibrate_batch"] = s_to_calibrate_batch(batch, c, wins, lb, ub, model)
    if not args.no_s2c and name == "paper_ird":  # the paper's setting on its representative objective
        with torch.cuda.stream(stream):
            out["s_to_calibrate_batch"] = s_to_calibrate_batch(batch, c, wins, lb, ub, model, stride=17)
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(name, budget_s=args.cpu_budget)
        out["cpu_baseline_all_cores"] = cpu_baseline_all_cores(name)
    return out


def stability_windows(rank: int = 0):
    """The stability configuration: reps copies of each chosen window (Philox stream words
    distinct per copy and per rank), with reported I and R."""
    c = dict(configs.CONFIGS["stability"])
    ser = synth.reported_IR(synth.load_series(c["series"]), c["seed"])
    T = np.repeat(np.asarray(c["windows_T"]), c["reps"])
    lay = {"L": np.full(T.size, c["L"]), "M": np.full(T.size, c["M"]), "T": T}
    wins = synth.rolling_window_problems(ser, lay)
    for i, w in enumerate(wins):
        w["seed"] = c["seed"]
        w["stream_id"] = rank * len(wins) + i
    return c, ser, wins


def run_stability(args, rank, world):
    import torch

    from paper_2204_12346_gb300 import sird

    c, ser, wins = stability_windows(rank)
    fit_I0 = c.get("fit_I0", True)
    lb, ub = configs.bounds_ramp(fit_I0=fit_I0)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch = sird.Batch(wins, K=1, beta_form=sird.BETA_RAMP, spd=c["spd"], iters=c["iters"], lb=lb, ub=ub,
                           fit_I0=fit_I0, cost=sird.COST_MXSE, objective=sird.FIT_IRD, block_size=args.block,
                           stream=stream)
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record(stream)
        ev[1].record(stream)
        batch.set_timing(*ev)
    reps = c["reps"]

    def step():
        res = batch.calibrate()
        bands, pbands = [], []
        for t in range(len(c["windows_T"])):
            th = np.array([r["theta"] for r in res[t * reps:(t + 1) * reps]])
            w = wins[t * reps]
            kw = dict(K=1, beta_form=sird.BETA_RAMP, R0=w["R0"], I0=w["I0"], fit_I0=fit_I0, spd=c["spd"], stream=stream)
            bands.append(sird.ensemble_bands(w["yD"], w["N"], th, c["horizon"], c["fractions"], **kw))
            pbands.append(sird.parameter_bands(w["yD"], w["N"], th, c["fractions"], **kw))
        return res, bands, pbands

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    total_ms, kern_ms, clocks, (res, bands, pbands) = timed_steps(args, world, stream, step, ev)
    # end to end: every step also uploads all windows' D, I, R series from host memory
    y_host = np.concatenate([np.concatenate([w["yD"], w["yI"], w["yR"]]) for w in wins])
    e2e, h2d = [], 0
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2d = batch.set_observations(y_host)
        step()
        e2e.append((time.perf_counter() - t0) * 1e3)
    e2e_total = _max_over_ranks(sum(e2e), world)
    if rank != 0:
        return None
    pdays = sum(w["particles"] * w["L"] for w in wins)
    units = pdays * c["iters"]
    kms = statistics.mean(kern_ms)
    flops = pdays * algorithmic_flops_per_particle_day(c["spd"], True, True) * (c["iters"] + 1)
    achieved = flops / (kms / 1e3) / 1e12
    held = {}
    for t, T in enumerate(c["windows_T"]):
        L, h = c["L"], c["horizon"]
        days = slice(L + 1, L + 1 + h)
        cover = {}
        for q, key in (("I", "yI"), ("R", "yR"), ("D", "yD")):
            rep_ = np.asarray(ser[key][T + L + 1:T + L + 1 + h])
            b = bands[t][q][days]
            cover[q] = {"inside_95": float(np.mean((b[:, 1] <= rep_) & (rep_ <= b[:, 2]))),
                        "median_max_rel_err": float(np.max(np.abs(b[:, 0] - rep_) / np.abs(rep_)))}
        names = ["beta1", "beta2", "t1", "t2", "gamma", "mu"] + ([] if not fit_I0 else ["I0"])
        cols = ["median"] + [f"{e}_{int(round(100 * f))}" for f in c["fractions"] for e in ("low", "high")]
        held[f"window_day_{T}"] = {"extension_vs_reported": cover,
                                   "parameter_bands": {n: dict(zip(cols, map(float, pbands[t][i])))
                                                       for i, n in enumerate(names)},
                                   "beta_R0_last_day_median": [float(bands[t]["beta"][L, 0]),
                                                               float(bands[t]["R0"][L, 0])]}
    return {
        "metric": METRIC, "value": units * args.steps * world / (total_ms / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": describe("stability"), "name": c["name"], "windows": len(wins),
                   "repetitions_per_window": reps, "particles": c["M"], "days": c["L"], "iterations": c["iters"],
                   "block": f"{batch.block_size} threads x {batch.blocks_per_sm} per SM",
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"independent batches x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": profiled_traffic("stability"),
                     "traffic_source": PROFILED.get("stability", {}).get("profile"),
                     "kernel": "pso_flat_f32" if batch.launch_mode == sird.LAUNCH_FLAT else "pso_batch_f32",
                     "avg_launch_us": kms * 1e3, "flops_per_launch": flops,
                     "peak_basis": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"},
        "e2e": {"value": units * args.steps * world / (e2e_total / 1e3), "unit": UNIT,
                # per window: theta ([reps][P] doubles) for each of the two band calls, the bands back
                "h2d_bytes_per_step": h2d + len(c["windows_T"]) * 2 * reps * len(lb) * 8,
                "d2h_bytes_per_step": len(wins) * BATCH_OUT_BYTES + len(c["windows_T"]) * (
                    6 * (c["L"] + 1 + c["horizon"]) + len(lb)) * (1 + 2 * len(c["fractions"])) * 8,
                "ms_per_step": e2e_total / args.steps},
        # the batch and its re-evaluation; per window two kernels of the ensemble bands and two of
        # the parameter bands (the ramp's change times ordered, then the sort)
        "gpu_launches": args.steps * (2 + len(c["windows_T"]) * 4),
        "clocks": clocks,
        "result": held,
        **({} if args.no_cpu_baseline else {"cpu_baseline": cpu_baseline("stability", budget_s=args.cpu_budget)}),
    }


def topk_launches(M: int, k: int, chunk: int = 4096) -> int:
    """Launches of the selection kernel for the k best of M (chunks of 4096, then the k best of
    every chunk, until one chunk is left)."""
    n, launches = M, 0
    while True:
        blocks = (n + chunk - 1) // chunk
        launches += 1
        if blocks == 1:
            return launches
        n = blocks * k


def run_single(args, rank, world):
    import torch

    from paper_2204_12346_gb300 import sird

    c, ser, y, lb, ub = single_window(args.workload)
    stream = torch.cuda.Stream()
    kw = dict(K=c["K"], spd=c["spd"], particles=c["M"], iters=c["iters"], lb=lb, ub=ub,
              log_scale=[1] * len(lb) if c["log"] else None, precision=c["precision"], seed=c["seed"],
              stream_id=rank, reeval_topk=c.get("reeval_topk", 0))
    horizon, fk = c.get("horizon", 0), c.get("forecast_topk", 0)

    with torch.cuda.stream(stream):
        cal = sird.Calibrator(y, ser["N"], stream=stream, **kw)
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record(stream)
        ev[1].record(stream)
        cal.set_timing(*ev)

    polish = c.get("polish_iters", 0)

    def step():
        r = cal.calibrate()
        if polish:  # FP32 L-BFGS polish of the best personal bests (adjoint gradient)
            r = dict(r, polished=cal.polish(k=c["polish_topk"], iters=polish, first_step=1e-2, precision=32))
        if not horizon:
            return r, None
        # the forecast leg (Sec. 4.2): the fk best personal bests continued `horizon` days
        th, _ = cal.topk(fk)
        return r, sird.forecast(y, ser["N"], th, horizon, K=c["K"], spd=c["spd"], precision=64, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    total_ms, kern_ms, clocks, (res, fc) = timed_steps(args, world, stream, step, ev)
    e2e = []
    y_host = np.asarray(y, dtype=np.float64)
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cal.set_observations(y_host)
        step()
        e2e.append((time.perf_counter() - t0) * 1e3)
    e2e_total = _max_over_ranks(sum(e2e), world)
    if rank != 0:
        return None
    L, spd, P = c["days"], c["spd"], len(lb)
    units = c["M"] * L * c["iters"]
    persistent = cal.launch_mode in (sird.LAUNCH_PERSISTENT, sird.LAUNCH_CLUSTER)
    iter_launches = 1 if persistent else c["iters"]
    kms = statistics.mean(kern_ms)
    flops = c["M"] * L * algorithmic_flops_per_particle_day(spd) * c["iters"]
    achieved = flops / (kms / 1e3) / 1e12
    fp64 = c["precision"] == 64
    peak = 1.25 if fp64 else FP32_PEAK_TFLOPS
    rk = c.get("reeval_topk", 0)
    launches = 1 + iter_launches + (topk_launches(c["M"], rk) + 1 if rk else 1)
    h2d, d2h = (L + 1) * 16, 288
    if polish:  # selection, init + gradient + accept, 6 per iteration, the final FP64 pick
        launches += topk_launches(c["M"], c["polish_topk"]) + 3 + 6 * polish + 1
    if horizon:
        launches += topk_launches(c["M"], fk) + 1 + 1
        h2d += fk * P * 8 + (L + 1) * 16
        d2h += fk * (P + 1) * 8 + fk * horizon * 8
    out = {
        "metric": METRIC, "value": units * args.steps * world / (total_ms / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if fp64 else "f32", "data": "synthetic",
        "config": {"workload": describe(args.workload), "name": c["name"], "particles": c["M"], "days": L,
                   "iterations": c["iters"], "steps_per_day": spd, "params": P,
                   "l2": "flushed between timed steps (256 MiB write)" + (
                       "; swarm state larger than L2" if c["M"] * P * 16 > 129e6 else ""),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": profiled_traffic(args.workload),
                     "traffic_source": PROFILED.get(args.workload, {}).get("profile"),
                     "ncu_fma_pipe_active": profiled_traffic(args.workload, "fma_pipe"),
                     "kernel": "pso_f32_persistent" if persistent else ("pso_f64_kernel" if fp64 else "pso_f32_kernel"),
                     "avg_launch_us": kms * 1e3 / iter_launches, "us_per_iteration": kms * 1e3 / c["iters"],
                     "peak_basis": ("nominal FP64 1.25 TFLOP/s" if fp64
                                    else "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz")},
        "e2e": {"value": units * args.steps * world / (e2e_total / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_total / args.steps},
        "gpu_launches": args.steps * launches,
        "clocks": clocks,
        "result": {"loss_fp64": res["loss"], "loss_search": res["loss_search"], "r2_D": res["r2_D"]},
    }
    if polish:
        out["result"].update({"polish": f"top {c['polish_topk']}, {polish} FP32 L-BFGS iterations",
                              "loss_fp64_polished": res["polished"]["loss"]})
    if horizon:
        held = np.asarray(ser["yD"][L + 1:L + 1 + horizon])
        rel = np.abs(fc - held[None, :]) / held[None, :]
        inside = (fc.min(axis=0) <= held) & (held <= fc.max(axis=0))
        out["result"].update({"forecast_days": f"{L + 1}..{L + horizon} (held out)", "forecast_topk": fk,
                              "forecast_best_max_rel_err": float(rel[0].max()),
                              "forecast_median_max_rel_err": float(np.median(rel.max(axis=1))),
                              "held_out_inside_topk_range": float(inside.mean())})
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, budget_s=args.cpu_budget)
    return out


def run_gradient(args, rank, world):
    """Gradient workload: loss and exact gradient (discrete adjoint, FP32 compensated trajectory,
    day-start checkpoints) of every personal best of a calibrated 4096-particle FP32 swarm on the
    90-day window at dt = 0.05 day.  One step = one gradient launch over all particles.  The FP64
    adjoint (checkpoints every 16 steps) of the same points is timed beside it."""
    import torch

    from paper_2204_12346_gb300 import sird

    c, ser, y, lb, ub = single_window("gradient90")
    stream = torch.cuda.Stream()
    P = len(lb)
    with torch.cuda.stream(stream):
        cal = sird.Calibrator(y, ser["N"], K=c["K"], spd=c["spd"], particles=c["M"], iters=c["iters"], lb=lb, ub=ub,
                              log_scale=[1] * P, precision=32, seed=c["seed"], stream_id=rank,
                              reeval_topk=c["reeval_topk"], stream=stream)
        cal.calibrate()
        st = cal.get_state()
        theta64 = torch.from_numpy(np.exp(st["pbest"].astype(np.float64))).to("cuda").contiguous()
        theta = theta64.float().contiguous()
        for _ in range(args.warmup):
            cal.loss_grad(theta)
            cal.loss_grad(theta64, ckpt_every=c["ckpt"])
    total_ms, kern_ms, clocks, (loss, grad) = timed_steps(args, world, stream, lambda: cal.loss_grad(theta))
    f64_ms = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cal.loss_grad(theta64, ckpt_every=c["ckpt"])
        e1.record(stream)
        torch.cuda.synchronize()
        f64_ms.append(e0.elapsed_time(e1))
    e2e = []
    th_host = torch.empty_like(theta, device="cpu").pin_memory()
    th_host.copy_(theta)
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            th_dev = th_host.to("cuda", non_blocking=True)
            lo, gr = cal.loss_grad(th_dev)
            lo_h, gr_h = lo.cpu(), gr.cpu()
        e2e.append((time.perf_counter() - t0) * 1e3)
    e2e_total = _max_over_ranks(sum(e2e), world)
    pol = cal.polish(k=c["polish_topk"], iters=50, first_step=1e-2, precision=32)
    if rank != 0:
        return None
    L, spd, M = c["days"], c["spd"], c["M"]
    units = M * L
    kms = statistics.mean(kern_ms)
    flops = M * L * spd * GRAD_FLOPS_PER_STEP
    achieved = flops / (kms / 1e3) / 1e12
    out = {
        "metric": METRIC, "value": units * args.steps * world / (total_ms / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": describe("gradient90"), "name": c["name"], "particles": M, "days": L, "steps_per_day": spd,
                   "params": P, "checkpoints": "every day start", "units": "particle-days of loss + gradient",
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": profiled_traffic("gradient90"),
                     "traffic_source": PROFILED["gradient90"]["profile"],
                     "ncu_fma_pipe_active": profiled_traffic("gradient90", "fma_pipe"),
                     "kernel": "loss_grad_f32_ws_kernel", "avg_launch_us": kms * 1e3, "flops_per_launch": flops,
                     "peak_basis": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"},
        "e2e": {"value": units * args.steps * world / (e2e_total / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": M * P * 4, "d2h_bytes_per_step": M * (P + 1) * 4,
                "ms_per_step": e2e_total / args.steps},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "result": {"finite_fraction": float(torch.isfinite(grad).all(dim=0).double().mean()),
                   "median_loss": float(loss.median()), "fp64_adjoint_ms": statistics.mean(f64_ms),
                   "fp64_adjoint_particle_days_per_s": units / (statistics.mean(f64_ms) / 1e3),
                   "polish_fp32_50_iters_loss_fp64": pol["loss"]},
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline("gradient90", budget_s=args.cpu_budget)
    return out


# ------------------------------------------------------------------ oracle on the host cores

def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


_WORKER_WINDOWS = {}


def _oracle_windows_worker(args):
    """One worker of the all-cores baseline: the oracle's initialisation and one PSO iteration on
    the given windows of the batched workload; returns particle-days processed."""
    name, idx = args
    import oracle as O

    if name not in _WORKER_WINDOWS:  # built once per worker, before the timed call
        _WORKER_WINDOWS[name] = batch_windows(name, 0)
    c, wins, lb, ub, model = _WORKER_WINDOWS[name]
    logd = [1] * len(lb) if model["log_scale"] else [0] * len(lb)
    zlb = np.where(logd, np.log(np.maximum(lb, 1e-300)), lb)
    zub = np.where(logd, np.log(np.maximum(ub, 1e-300)), ub)
    units = 0
    for i in idx:
        w = wins[i]
        pb = O.Problem(yD=w["yD"], N=w["N"], R0=w["R0"], K=model["K"], spd=c["spd"],
                       beta_form=O.BETA_RAMP if model["beta_form"] == 1 else O.BETA_PWC, cost=model["cost"],
                       objective=model["objective"], yI=w.get("yI"), yR=w.get("yR"), fit_I0=model["fit_I0"],
                       I0=w.get("I0", 0.0))
        O.PSO(pb, w["particles"], zlb, zub, logdim=logd, seed=w["seed"], stream=w["stream_id"],
              store_f32=True).init().step(1)
        units += w["particles"] * w["L"] * 2
    return units


def cpu_baseline_all_cores(name: str, windows_per_core: int = 16) -> dict:
    """The same oracle on every host core: one process per core (spawned, not forked, since the
    parent has used the GPU), each running whole windows of the batched workload."""
    import multiprocessing as mp

    import oracle as O

    O.build()
    cores = os.cpu_count() or 1
    c, wins, _, _, _ = batch_windows(name, 0)
    n = min(len(wins), cores * windows_per_core)
    jobs = [(name, list(range(r, n, cores))) for r in range(cores)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_windows_worker, [(name, [0])] * cores)  # start-up and imports, not timed
        t0 = time.perf_counter()
        units = sum(pool.map(_oracle_windows_worker, jobs))
        dt = time.perf_counter() - t0
    return {"value": units / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"{n} windows x (init + 1 PSO iteration), one process per core, FP64 ({dt:.3g} s)"}


def cpu_baseline(name: str, budget_s: float = 15.0, iters_cap: int | None = None) -> dict:
    """The FP64 oracle as it stands, single-threaded, on a bounded sample of the workload."""
    import oracle as O

    O.build()
    t0 = time.perf_counter()
    units = 0
    if name in BATCHED:
        c, wins, lb, ub, model = batch_windows(name, 0)
        logd = [1] * len(lb) if model["log_scale"] else [0] * len(lb)
        zlb = np.where(logd, np.log(np.maximum(lb, 1e-300)), lb)
        zub = np.where(logd, np.log(np.maximum(ub, 1e-300)), ub)
        done = 0
        for w in wins:
            if time.perf_counter() - t0 >= budget_s or (iters_cap is not None and done >= iters_cap):
                break
            pb = O.Problem(yD=w["yD"], N=w["N"], R0=w["R0"], K=model["K"], spd=c["spd"],
                           beta_form=O.BETA_RAMP if model["beta_form"] == 1 else O.BETA_PWC, cost=model["cost"],
                           objective=model["objective"], yI=w.get("yI"), yR=w.get("yR"), fit_I0=model["fit_I0"],
                           I0=w.get("I0", 0.0))
            O.PSO(pb, w["particles"], zlb, zub, logdim=logd, seed=w["seed"], stream=w["stream_id"],
                  store_f32=True).init().step(1)
            units += w["particles"] * w["L"] * 2
            done += 1
        sample = f"{done} windows x (init + 1 PSO iteration), full swarms"
    elif name == "stability":
        c, ser, wins = stability_windows(0)
        fit_I0 = c.get("fit_I0", True)
        lb, ub = configs.bounds_ramp(fit_I0=fit_I0)
        done = 0
        for w in wins:
            if time.perf_counter() - t0 >= budget_s or (iters_cap is not None and done >= iters_cap):
                break
            pb = O.Problem(yD=w["yD"], N=w["N"], R0=w["R0"], beta_form=O.BETA_RAMP, spd=c["spd"], cost=O.MXSE,
                           objective=O.FIT_IRD, yI=w["yI"], yR=w["yR"], fit_I0=fit_I0, I0=w["I0"])
            O.PSO(pb, w["particles"], lb, ub, logdim=[0] * len(lb), seed=w["seed"], stream=w["stream_id"],
                  store_f32=True).init().step(1)
            units += w["particles"] * w["L"] * 2
            done += 1
        sample = f"{done} repetitions x (init + 1 PSO iteration), 10000 particles each"
    elif name == "gradient90":
        c, ser, y, lb, ub = single_window(name)
        pb = O.Problem(yD=y, N=ser["N"], K=c["K"], spd=c["spd"])
        rng = np.random.default_rng(c["seed"])
        done = 0
        while time.perf_counter() - t0 < budget_s and (iters_cap is None or done < iters_cap * 64):
            for th in synth.box_sample(lb, ub, [1] * len(lb), 64, rng):
                O.loss_grad(pb, th)
            done += 64
        units = done * c["days"]
        sample = f"loss + gradient of {done} box-sampled parameter vectors (90 days, dt=0.05)"
    else:
        c, ser, y, lb, ub = single_window(name)
        logd = [1] * len(lb) if c["log"] else [0] * len(lb)
        M = min(c["M"], 4096)  # bounded sample of the 2^20-particle swarm
        zlb = np.log(lb) if c["log"] else np.array(lb, float)
        zub = np.log(ub) if c["log"] else np.array(ub, float)
        pso = O.PSO(O.Problem(yD=y, N=ser["N"], K=c["K"], spd=c["spd"]), M, zlb, zub, logdim=logd,
                    seed=c["seed"], store_f32=c["precision"] == 32).init()
        its = 0
        while time.perf_counter() - t0 < budget_s and (iters_cap is None or its < iters_cap):
            pso.step(1)
            its += 1
        units = M * c["days"] * (its + 1)
        sample = f"{M} particles x {c['days']} days, init + {its} PSO iterations"
    dt = time.perf_counter() - t0
    return {"value": units / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"{sample}, single thread, FP64 ({dt:.3g} s)"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    per_step = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(args.workload, budget_s=1e9, iters_cap=args.ref_units)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            per_step.append((cb, dt))
    value = statistics.mean(cb["value"] for cb, _ in per_step)
    ms = statistics.mean(dt for _, dt in per_step) * 1e3
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": describe(args.workload), "name": configs.CONFIGS[args.workload]["name"],
                   "sample": per_step[0][0]["sample"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": per_step[0][0]["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def _free_port() -> int:
    import socket

    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def relaunch_under_torchrun(n: int):
    """Replaces this process by `torch.distributed.run` starting n ranks of this script with the
    same arguments (rendezvous on 127.0.0.1); the ranks print as a launched job would."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", f"--master-port={_free_port()}", os.path.abspath(__file__)] + sys.argv[1:]
    sys.stdout.flush()
    os.execv(sys.executable, cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["batch512", "window60", "plain64", "gradient90", "swarm2p20", "paper", "paper_ird", "stability"],
                    default="batch512")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-units", type=int, default=2,
                    help="reference arm: windows (batched) or PSO iterations (single window) per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-s2c", action="store_true", help="skip the seconds-to-calibrate comparison")
    ap.add_argument("--block", type=int, default=0, help="batched: threads per block (0 = autotune)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.gpus < 1:
        ap.error("--gpus must be >= 1")
    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        # one process per GPU: start the ranks here rather than asking for an outer launcher
        relaunch_under_torchrun(args.gpus)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world != args.gpus:
        ap.error(f"--gpus {args.gpus} but WORLD_SIZE={world}: launch one rank per GPU")
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        if args.impl == "ours":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    try:
        if args.impl == "reference":
            out = run_reference(args, rank, world)
        elif args.workload in BATCHED:
            out = run_batched(args, rank, world)
        elif args.workload == "gradient90":
            out = run_gradient(args, rank, world)
        elif args.workload == "stability":
            out = run_stability(args, rank, world)
        else:
            out = run_single(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
