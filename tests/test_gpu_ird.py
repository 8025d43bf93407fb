"""The F_IRD^C objective (Sec. 3.1: the largest of the min-max-normalised costs of I, R and D)
on the GPU against the FP64 oracle (GPU only)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2204_12346_gb300 import configs, sird, synth
from util import assert_fp32_losses, box_thetas, f32, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    torch.cuda.set_device(0)
    O.build()


def ird_series(name, days=None, seed=1):
    s = synth.reported_IR(synth.load_series(name), seed)
    n = len(s["yD"]) if days is None else days + 1
    return s["yD"][:n], s["yI"][:n], s["yR"][:n], float(s["N"])


def ramp_thetas(M, seed, days):
    rng = np.random.default_rng(seed)
    return f32(np.column_stack([rng.uniform(0.05, 0.5, M), rng.uniform(0.05, 0.5, M), rng.uniform(0, days, M),
                                rng.uniform(0, days, M), rng.uniform(0.02, 0.3, M), rng.uniform(1e-4, 5e-3, M),
                                rng.uniform(1e3, 5e4, M)]))


def setup(cost, form, days=60, spd=10):
    yD, yI, yR, N = ird_series("60d", days)
    if form == "pwc":
        K, bf, th = 4, sird.BETA_PWC, np.concatenate([box_thetas(4, 96, 3), f32(synth.box_sample(
            [0.1] * 4 + [0.05, 1e-3, 5e3], [0.3] * 4 + [0.15, 3e-3, 2e4], [0] * 7, 64, np.random.default_rng(4)))])
    else:
        K, bf, th = 1, sird.BETA_RAMP, ramp_thetas(160, 5, days)
    common = dict(K=K, spd=spd, R0=float(yR[0]), beta_form=bf, cost=sird.COSTS[cost], objective=sird.FIT_IRD, yI=yI,
                  yR=yR, particles=32, iters=1, lb=[0.0] * th.shape[1], ub=[1e6] * th.shape[1])
    pb = O.Problem(yD=yD, yI=yI, yR=yR, N=N, R0=float(yR[0]), K=K, spd=spd, cost=O.COSTS[cost],
                   beta_form=O.BETA_RAMP if form == "ramp" else O.BETA_PWC, objective=O.FIT_IRD)
    return yD, N, th, common, pb


@pytest.mark.parametrize("form", ["pwc", "ramp"])
@pytest.mark.parametrize("cost", ["mse", "mxse", "mae", "mape"])
def test_ird_fp64_bit_exact(cost, form):
    yD, N, th, common, pb = setup(cost, form)
    cal = sird.Calibrator(yD, N, precision=64, **common)
    L = cal.eval(torch.from_numpy(np.ascontiguousarray(th.T)).cuda()).cpu().numpy()
    want = O.losses(pb, th)
    assert np.array_equal(L, want), np.max(rel_err(L, want))


@pytest.mark.parametrize("form", ["pwc", "ramp"])
@pytest.mark.parametrize("cost", ["mse", "mxse", "mae", "mape"])
def test_ird_fp32_within_tolerance(cost, form):
    yD, N, th, common, pb = setup(cost, form)
    cal = sird.Calibrator(yD, N, precision=32, **common)
    L = cal.eval(torch.from_numpy(np.ascontiguousarray(th.T).astype(np.float32)).cuda()).cpu().numpy()
    want = O.losses(pb, th)
    print("largest relative error", assert_fp32_losses(L, want, (cost, form)))


def test_ird_fp64_calibration_matches_the_oracle_swarm():
    # the plain method in FP64 on F_IRD^MXSE (the paper's representative objective)
    yD, yI, yR, N = ird_series("30d")
    lb, ub = configs.bounds(1, log=False)
    cal = sird.Calibrator(yD, N, R0=float(yR[0]), objective=sird.FIT_IRD, yI=yI, yR=yR, cost=sird.COST_MXSE,
                          particles=64, iters=30, lb=lb, ub=ub, precision=64, seed=3)
    r = cal.calibrate()
    st = cal.get_state()
    pb = O.Problem(yD=yD, yI=yI, yR=yR, N=N, R0=float(yR[0]), cost=O.MXSE, objective=O.FIT_IRD)
    pso = O.PSO(pb, 64, lb, ub, logdim=[0] * 4, seed=3, stream=0).init().step(30)
    assert np.array_equal(st["pbest"].T, pso.pbest) and np.array_equal(st["pbest_f"], pso.pbest_f)
    assert r["index"] == pso.gbest_idx and r["loss"] == pso.gbest_f


def test_ird_fp32_calibration_reports_its_fp64_loss_and_batches_agree():
    ser = synth.reported_IR(synth.load_series("450d"), 2)
    lay = {"L": np.array([30, 45, 21]), "M": np.array([300, 700, 90]), "T": np.array([10, 150, 300])}
    wins = synth.rolling_window_problems(ser, lay)
    lb, ub = configs.bounds(3, log=True)
    kw = dict(K=3, spd=10, lb=lb, ub=ub, log_scale=[1] * 6, seed=7, objective=sird.FIT_IRD, cost=sird.COST_MXSE)
    res = sird.Batch(wins, iters=6, block_size=128, **kw).calibrate()
    for i, w in enumerate(wins):
        cal = sird.Calibrator(w["yD"], w["N"], R0=w["R0"], yI=w["yI"], yR=w["yR"], particles=w["particles"], iters=6,
                              precision=32, stream_id=i, reeval_topk=0, **kw)
        r = cal.calibrate()
        assert res[i]["index"] == r["index"] and res[i]["loss"] == r["loss"], i
        pb = O.Problem(yD=w["yD"], yI=w["yI"], yR=w["yR"], N=w["N"], R0=w["R0"], K=3, spd=10, cost=O.MXSE,
                       objective=O.FIT_IRD)
        assert r["loss"] == O.loss(pb, r["theta"])


def test_ird_rejects_the_gradient_calls():
    yD, yI, yR, N = ird_series("60d", 30)
    lb, ub = configs.bounds(1, log=True)
    cal = sird.Calibrator(yD, N, R0=float(yR[0]), objective=sird.FIT_IRD, yI=yI, yR=yR, particles=64, iters=2,
                          lb=lb, ub=ub, log_scale=[1] * 4, precision=32)
    cal.calibrate()
    with pytest.raises(sird.SirdError):
        cal.loss_grad(torch.ones(4, 8, dtype=torch.float64, device="cuda"))


def test_ird_batch_set_observations_equals_a_fresh_batch():
    ser = synth.reported_IR(synth.load_series("450d"), 4)
    lay = {"L": np.array([25, 40]), "M": np.array([200, 450]), "T": np.array([30, 200])}
    wins = synth.rolling_window_problems(ser, lay)
    nxt = synth.rolling_window_problems(ser, dict(lay, T=lay["T"] + 2))
    lb, ub = configs.bounds(2, log=True)
    kw = dict(K=2, spd=10, lb=lb, ub=ub, log_scale=[1] * 5, seed=9, objective=sird.FIT_IRD, cost=sird.COST_MSE,
              block_size=128)
    batch = sird.Batch(wins, iters=4, **kw)
    batch.calibrate()
    batch.set_observations(np.concatenate([np.concatenate([w["yD"], w["yI"], w["yR"]]) for w in nxt]))
    got = batch.calibrate()
    fresh = sird.Batch([dict(w, R0=o["R0"]) for w, o in zip(nxt, wins)], iters=4, **kw).calibrate()
    for a, b in zip(got, fresh):
        assert a["index"] == b["index"] and a["loss"] == b["loss"] and np.array_equal(a["theta"], b["theta"])
