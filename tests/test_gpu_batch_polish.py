"""L-BFGS polish of a whole batch of windows against the one-window polish (GPU only).

Every window of a batch is polished in the same launches, with its own constants, observations
and personal bests (Sec. 3.1: rolling windows calibrated independently).  Each window's result
must equal the one-window polish of the same swarm bit for bit, and its reported loss must be the
oracle's FP64 loss at the reported parameters.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2204_12346_gb300 import configs, sird, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    torch.cuda.set_device(0)
    O.build()


def layout():
    # eight windows of uneven length (21..90 days) and swarm size, cut from the 450-day series
    return {"L": np.array([21, 34, 25, 40, 22, 30, 27, 90]), "M": np.array([64, 96, 150, 40, 300, 48, 200, 128]),
            "T": np.array([0, 57, 120, 201, 300, 333, 410, 350])}


def pwc(K, spd, cost):
    lb, ub = configs.bounds(K, log=True)
    return dict(K=K, spd=spd, cost=cost, lb=lb, ub=ub, log_scale=[1] * len(lb), seed=5)


def ramp(spd, cost):
    lb, ub = configs.bounds_ramp(t_max=20.0, fit_I0=True)
    return dict(beta_form=sird.BETA_RAMP, spd=spd, cost=cost, lb=lb, ub=ub, seed=7)


# the warp-specialised adjoint (PWC, 10 and 20 steps per day), the generic one (7 steps per day)
# and the ramp form's; all four costs
CASES = {
    "pwc-spd10-mse": pwc(6, 10, sird.COST_MSE),
    "pwc-spd20-mape": pwc(3, 20, sird.COST_MAPE),
    "pwc-spd7-mae": pwc(2, 7, sird.COST_MAE),
    "ramp-spd10-mxse": ramp(10, sird.COST_MXSE),
}


def oracle_problem(w, kw):
    return O.Problem(yD=w["yD"], N=w["N"], R0=w["R0"], K=kw.get("K", 1), spd=kw["spd"], cost=kw["cost"],
                     beta_form=kw.get("beta_form", sird.BETA_PWC))


@pytest.mark.parametrize("case", list(CASES))
def test_batch_polish_equals_one_window_polish(case):
    kw = CASES[case]
    wins = synth.rolling_window_problems(synth.load_series("450d"), layout())
    iters, k, piters = 12, 16, 6
    batch = sird.Batch(wins, iters=iters, **kw)
    cal_b = batch.calibrate()
    got = batch.polish(k=k, iters=piters, first_step=1e-2)
    assert len(got) == len(wins)
    for i, w in enumerate(wins):
        cal = sird.Calibrator(w["yD"], w["N"], R0=w["R0"], particles=w["particles"], iters=iters, precision=32,
                              stream_id=i, reeval_topk=0, **kw)
        cal.calibrate()
        want = cal.polish(k=k, iters=piters, first_step=1e-2, precision=32)
        assert got[i]["index"] == want["index"], (case, i)
        assert got[i]["loss"] == want["loss"], (case, i)
        assert got[i]["loss_search"] == want["loss_search"], (case, i)
        assert np.array_equal(got[i]["theta"], want["theta"]), (case, i)
        assert got[i]["r2_D"] == pytest.approx(want["r2_D"], rel=1e-12)
        # the reported loss is the FP64 loss of the reported parameters
        assert got[i]["loss"] == O.loss(oracle_problem(w, kw), got[i]["theta"]), (case, i)
        # the polish starts from the global best among others and keeps the best point it saw
        assert got[i]["loss"] <= cal_b[i]["loss"] * (1 + 2e-5), (case, i)


def test_batch_polish_repeats_and_leaves_the_swarms_alone():
    kw = CASES["pwc-spd10-mse"]
    wins = synth.rolling_window_problems(synth.load_series("450d"), layout())
    batch = sird.Batch(wins, iters=8, **kw)
    first = batch.calibrate()
    a = batch.polish(k=8, iters=4)
    b = batch.polish(k=24, iters=2)  # a larger scratch
    c = batch.polish(k=8, iters=4)
    for x, y in zip(a, c):
        assert x["loss"] == y["loss"] and np.array_equal(x["theta"], y["theta"]) and x["index"] == y["index"]
    assert all(np.isfinite(r["loss"]) for r in b)
    # a new calibration of the same batch reproduces the first (the polish did not touch the swarms)
    again = batch.calibrate()
    for x, y in zip(first, again):
        assert x["loss"] == y["loss"] and x["index"] == y["index"]


def test_batch_polish_refusals():
    kw = CASES["pwc-spd10-mse"]
    wins = synth.rolling_window_problems(synth.load_series("450d"), layout())
    batch = sird.Batch(wins, iters=4, **kw)
    with pytest.raises(sird.SirdError, match="STATE"):
        batch.polish(k=4, iters=1)  # before any calibration
    batch.calibrate()
    for bad in (dict(k=0), dict(k=41), dict(k=4, iters=-1), dict(k=4, first_step=0.0)):
        with pytest.raises(sird.SirdError, match="ARG"):
            batch.polish(**bad)  # 41 > the smallest swarm (40)
    batch.set_observations(np.concatenate([w["yD"] for w in wins]))
    with pytest.raises(sird.SirdError, match="STATE"):
        batch.polish(k=4, iters=1)  # the personal bests belong to the old observations
    ser = synth.reported_IR(synth.load_series("450d"), 0)  # reported I and R series for F_IRD
    ird = synth.rolling_window_problems(ser, layout())
    lb, ub = configs.bounds_ramp(fit_I0=False)
    bi = sird.Batch(ird, beta_form=sird.BETA_RAMP, objective=sird.FIT_IRD, cost=sird.COST_MXSE, fit_I0=False,
                    iters=2, lb=lb, ub=ub)
    bi.calibrate()
    assert len(bi.polish(k=4, iters=1)) == len(ird)  # F_IRD batches polish too (FP32 F_IRD adjoint)


def test_batch_polish_512_window_layout_sampled_windows():
    # the batched configuration's layout and iterations; the polish the benchmark runs on it
    c = configs.CONFIGS["batch512"]
    ser = synth.load_series("450d")
    lay = synth.rolling_windows(W=c["W"], L_min=c["L_min"], L_max=c["L_max"], M_min=c["M_min"], M_max=c["M_max"],
                                delta=c["delta"], seed=c["seed"])
    wins = synth.rolling_window_problems(ser, lay)
    lb, ub = configs.bounds(c["K"], True)
    kw = dict(K=c["K"], spd=c["spd"], lb=lb, ub=ub, log_scale=[1] * 9, seed=c["seed"])
    batch = sird.Batch(wins, iters=c["iters"], **kw)
    batch.calibrate()
    got = batch.polish(k=32, iters=10, first_step=1e-2)
    for i in np.random.default_rng(4).choice(len(wins), 4, replace=False):
        w = wins[i]
        cal = sird.Calibrator(w["yD"], w["N"], R0=w["R0"], particles=w["particles"], iters=c["iters"], precision=32,
                              stream_id=int(i), reeval_topk=0, **kw)
        cal.calibrate()
        want = cal.polish(k=32, iters=10, first_step=1e-2, precision=32)
        assert got[i]["loss"] == want["loss"] and got[i]["index"] == want["index"], i
        assert np.array_equal(got[i]["theta"], want["theta"]), i
        pb = O.Problem(yD=w["yD"], N=w["N"], R0=w["R0"], K=c["K"], spd=c["spd"])
        assert got[i]["loss"] == O.loss(pb, got[i]["theta"]), i
