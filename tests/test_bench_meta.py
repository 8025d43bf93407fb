"""Consistency of the benchmark's bookkeeping (CPU): every workload it can run has a
description and a configuration, and every profiled kernel's summary under profiles/ exists and
names the source hash the bench compares against."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_every_workload_is_described_and_configured():
    import bench
    from paper_2204_12346_gb300 import configs

    for name in ("batch512", "window60", "plain64", "gradient90", "swarm2p20", "paper", "paper_ird", "stability"):
        assert name in configs.CONFIGS
        assert len(bench.describe(name)) > 40


def test_profile_summaries_name_their_source_hash():
    import bench

    for name, p in bench.PROFILED.items():
        path = os.path.join(ROOT, p["profile"])
        assert os.path.exists(path), path
        text = open(path).read()
        assert p["sha"] and f"`{p['sha']}`" in text, (name, p["sha"])
        assert p["traffic_bytes"] > 0 and 0.0 < p["fma_pipe"] < 1.0
        for f in p["files"]:
            assert os.path.exists(os.path.join(ROOT, "paper_2204_12346_gb300", "csrc", f)), f


def test_algorithmic_flop_counts():
    import bench

    # 8 flops per Euler step and 3 per day; the ramp adds 5 per step, F_IRD 2 per step and 6 per day
    assert bench.algorithmic_flops_per_particle_day(10) == 83
    assert bench.algorithmic_flops_per_particle_day(20) == 163
    assert bench.algorithmic_flops_per_particle_day(10, ramp=True) == 133
    assert bench.algorithmic_flops_per_particle_day(10, ramp=True, ird=True) == 159


def test_every_workload_fits_the_binding_checks():
    # the boxes, series and model settings each workload passes satisfy the binding's checks
    import bench
    from paper_2204_12346_gb300 import configs, sird

    for name in bench.BATCHED:
        c, wins, lb, ub, model = bench.batch_windows(name)
        P = sird.n_params(model["K"], model["beta_form"], model["fit_I0"])
        sird._check_box(P, lb, ub, model["log_scale"])
        assert len(lb) == P
        for w in wins:
            sird.make_problem(w["yD"], w["N"], yI=w.get("yI"), yR=w.get("yR"))
    for name in ("window60", "plain64", "gradient90", "swarm2p20"):
        c, ser, y, lb, ub = bench.single_window(name)
        P = sird.n_params(c["K"])
        sird._check_box(P, lb, ub, [1] * len(lb) if c["log"] else None)
        assert len(lb) == P
    c, ser, wins = bench.stability_windows()
    lb, ub = configs.bounds_ramp(fit_I0=c.get("fit_I0", True))
    assert len(lb) == sird.n_params(beta_form=sird.BETA_RAMP, fit_I0=c.get("fit_I0", True))


def test_reference_arm_line_has_the_contract_keys():
    import json
    import subprocess

    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3",
                        "--ref-units", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert k in out, k
    assert out["impl"] == "reference" and out["n_gpus"] == 1 and out["steps"] == 1 and out["warmup"] == 3
    assert out["value"] > 0 and out["higher_is_better"] is True and out["vs_baseline"] is None
    assert out["dtype"] == "f64" and out["data"] == "synthetic" and "512" in out["config"]["workload"]
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == out["value"] and cb["sample"]
    assert out["e2e"] == {"value": out["value"], "unit": out["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
