"""Batched calibration of many rolling windows in one launch (GPU only)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2204_12346_gb300 import configs, sird, synth
from util import TOL32, f32, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    torch.cuda.set_device(0)
    O.build()


def small_layout():
    # seven windows of uneven length and ragged swarm sizes cut from the 450-day series
    return {"L": np.array([21, 34, 25, 40, 22, 30, 27]), "M": np.array([64, 96, 150, 33, 300, 1, 200]),
            "T": np.array([0, 57, 120, 201, 300, 333, 410])}


def shared(K=6):
    lb, ub = configs.bounds(K, log=True)
    return dict(K=K, spd=10, lb=lb, ub=ub, log_scale=[1] * len(lb), seed=11)


def test_batch_windows_match_single_window_calibrations():
    ser = synth.load_series("450d")
    wins = synth.rolling_window_problems(ser, small_layout())
    kw = shared()
    batch = sird.Batch(wins, iters=15, **kw)
    res = batch.calibrate()
    for i, w in enumerate(wins):
        cal = sird.Calibrator(w["yD"], w["N"], R0=w["R0"], particles=w["particles"], iters=15, precision=32,
                              stream_id=i, reeval_topk=0, **kw)
        r = cal.calibrate()
        assert res[i]["index"] == r["index"], i
        assert res[i]["loss_search"] == r["loss_search"], i
        assert res[i]["loss"] == r["loss"], i
        assert np.array_equal(res[i]["theta"], r["theta"]), i
        assert res[i]["r2_D"] == pytest.approx(r["r2_D"], rel=1e-12)


def test_batch_set_observations_equals_a_fresh_batch():
    # the next day's data on the same windows (each window shifted by one day, same lengths)
    ser = synth.load_series("450d")
    lay = small_layout()
    wins = synth.rolling_window_problems(ser, lay)
    nxt = synth.rolling_window_problems(ser, dict(lay, T=lay["T"] + 1))
    kw = shared()
    batch = sird.Batch(wins, iters=6, block_size=128, **kw)
    batch.calibrate()
    nb = batch.set_observations(np.concatenate([w["yD"] for w in nxt]))
    assert nb >= 16 * sum(len(w["yD"]) for w in nxt) + 128 * len(nxt)
    got = batch.calibrate()
    # R0 stays that of the first layout: the fresh batch gets the same R0
    fresh = sird.Batch([dict(w, R0=o["R0"]) for w, o in zip(nxt, wins)], iters=6, block_size=128, **kw).calibrate()
    for a, b in zip(got, fresh):
        assert a["index"] == b["index"] and a["loss"] == b["loss"] and a["loss_search"] == b["loss_search"]
        assert np.array_equal(a["theta"], b["theta"]) and a["r2_D"] == b["r2_D"]
    with pytest.raises(sird.SirdError):
        batch.set_observations(np.ones(3))


def test_batch_block_sizes_agree():
    ser = synth.load_series("450d")
    wins = synth.rolling_window_problems(ser, small_layout())
    out = [sird.Batch(wins, iters=8, block_size=b, **shared()).calibrate() for b in (64, 256)]
    for a, b in zip(*out):
        assert a["index"] == b["index"] and a["loss"] == b["loss"]
    auto = sird.Batch(wins, iters=8, **shared())
    assert auto.block_size in (128, 256, 384, 512, 640, 768, 1024) and auto.blocks_per_sm >= 1


def test_full_512_window_layout_against_the_oracle_at_initialisation():
    # the batched configuration's layout: 512 windows, 21..90 days, 256..2048 particles, 6 segments
    c = configs.CONFIGS["batch512"]
    ser = synth.load_series("450d")
    lay = synth.rolling_windows(W=c["W"], L_min=c["L_min"], L_max=c["L_max"], M_min=c["M_min"], M_max=c["M_max"],
                                delta=c["delta"], seed=c["seed"])
    wins = synth.rolling_window_problems(ser, lay)
    kw = shared(c["K"])
    res = sird.Batch(wins, iters=0, **kw).calibrate()
    assert len(res) == 512 and all(np.isfinite(r["loss"]) for r in res)
    lb, ub = configs.bounds(c["K"], log=True)
    zlb, zub = f32(np.log(lb)), f32(np.log(ub))
    for i in np.random.default_rng(0).choice(512, 6, replace=False):
        w = wins[i]
        pb = O.Problem(yD=w["yD"], N=w["N"], R0=w["R0"], K=c["K"], spd=10)
        pso = O.PSO(pb, w["particles"], zlb, zub, logdim=[1] * len(lb), seed=kw["seed"], stream=int(i),
                    store_f32=True).init()
        assert rel_err(res[i]["loss_search"], pso.gbest_f) <= 1e-5
        s = np.sort(pso.pbest_f)
        if s[1] - s[0] > 3e-5 * s[0]:
            assert res[i]["index"] == pso.gbest_idx


def ramp_shared():
    lb, ub = configs.bounds_ramp()
    return dict(K=1, spd=10, beta_form=sird.BETA_RAMP, lb=lb, ub=ub, log_scale=None, seed=5)


def test_batch_ramp_windows_match_single_window_calibrations():
    # the paper's ramp form on a linear box; swarms beyond 2 x block size (several passes per
    # thread, packed pairs and single particles)
    ser = synth.load_series("450d")
    lay = {"L": np.array([35, 35, 20, 35]), "M": np.array([3000, 700, 129, 2500]), "T": np.array([0, 90, 200, 414])}
    wins = synth.rolling_window_problems(ser, lay)
    kw = ramp_shared()
    res = sird.Batch(wins, iters=5, block_size=256, **kw).calibrate()
    for i, w in enumerate(wins):
        cal = sird.Calibrator(w["yD"], w["N"], R0=w["R0"], particles=w["particles"], iters=5, precision=32,
                              stream_id=i, reeval_topk=0, **kw)
        r = cal.calibrate()
        assert res[i]["index"] == r["index"], i
        assert res[i]["loss_search"] == r["loss_search"], i
        assert res[i]["loss"] == r["loss"], i
        assert np.array_equal(res[i]["theta"], r["theta"]), i


def test_paper_layout_against_the_oracle_at_initialisation():
    # the paper's setting: 139 windows of 35 days shifted by 3 days, 10000 particles, ramp beta(t),
    # each window's initial state from the reported I, R, D of its first day (theta: 6 rates)
    c = configs.CONFIGS["paper"]
    assert c["fit_I0"] is False
    ser = synth.reported_IR(synth.load_series(c["series"]), c["seed"])
    lay = synth.rolling_windows(W=c["W"], L_min=c["L_min"], L_max=c["L_max"], M_min=c["M_min"], M_max=c["M_max"],
                                delta=c["delta"], seed=c["seed"])
    wins = synth.rolling_window_problems(ser, lay)
    for w in wins:  # F_D: deaths only
        w.pop("yI")
        w.pop("yR")
    assert len(wins) == 139 and all(w["particles"] == 10000 and w["L"] == 35 for w in wins)
    assert [w["T"] for w in wins[:3]] == [0, 3, 6] and wins[-1]["T"] == 414
    lb, ub = configs.bounds_ramp(fit_I0=False)
    kw = dict(K=1, spd=10, beta_form=sird.BETA_RAMP, lb=lb, ub=ub, log_scale=None, seed=5, fit_I0=False)
    res = sird.Batch(wins, iters=0, **kw).calibrate()
    assert len(res) == 139 and all(np.isfinite(r["loss"]) for r in res)
    zlb, zub = f32(lb), f32(ub)
    for i in (0, 70, 138):
        w = wins[i]
        pb = O.Problem(yD=w["yD"], N=w["N"], R0=w["R0"], I0=w["I0"], fit_I0=False, beta_form=O.BETA_RAMP, spd=10)
        pso = O.PSO(pb, w["particles"], zlb, zub, logdim=[0] * 6, seed=kw["seed"], stream=i, store_f32=True).init()
        # the best of 10000 is a good fit; its FP32 loss is the oracle's within the contract
        assert rel_err(res[i]["loss_search"], pso.gbest_f) <= TOL32, i
        s = np.sort(pso.pbest_f)
        if s[1] - s[0] > 2 * TOL32 * s[0]:
            assert res[i]["index"] == pso.gbest_idx
        # the reported loss is the FP64 loss of the reported theta, bit for bit
        assert res[i]["loss"] == O.loss(pb, res[i]["theta"])


@pytest.mark.parametrize("block", [128, 256, 512])
def test_flat_form_equals_one_window_per_block(block):
    # every window's swarm spread over the grid (one grid barrier per iteration) gives the same
    # swarms as one window per block: same Philox counters and arithmetic per particle
    ser = synth.load_series("450d")
    wins = synth.rolling_window_problems(ser, small_layout())
    kw = shared()
    a = sird.Batch(wins, iters=9, block_size=256, **kw).calibrate()
    fb = sird.Batch(wins, iters=9, block_size=block, launch_mode=sird.LAUNCH_FLAT, **kw)
    assert fb.launch_mode == sird.LAUNCH_FLAT
    b = fb.calibrate()
    b2 = fb.calibrate()  # replayed graph: the barrier and reduction words start fresh
    for x, y, z in zip(a, b, b2):
        assert x["index"] == y["index"] == z["index"] and x["loss_search"] == y["loss_search"] == z["loss_search"]
        assert x["loss"] == y["loss"] and np.array_equal(x["theta"], y["theta"])
    with pytest.raises(sird.SirdError, match="flat"):  # above the flat form's launch bound
        sird.Batch(wins, iters=2, block_size=768, launch_mode=sird.LAUNCH_FLAT, **kw)


def test_flat_form_ramp_ird_and_mape():
    ser = synth.reported_IR(synth.load_series("450d"), 3)
    lay = {"L": np.array([35, 35, 20, 35]), "M": np.array([3000, 700, 129, 2500]), "T": np.array([0, 90, 200, 414])}
    wins = synth.rolling_window_problems(ser, lay)
    lb, ub = configs.bounds_ramp()
    for obj, cost in ((sird.FIT_D, sird.COST_MAPE), (sird.FIT_IRD, sird.COST_MXSE)):
        kw = dict(K=1, spd=10, beta_form=sird.BETA_RAMP, lb=lb, ub=ub, seed=4, objective=obj, cost=cost)
        a = sird.Batch(wins, iters=4, block_size=256, **kw).calibrate()
        b = sird.Batch(wins, iters=4, block_size=384, launch_mode=sird.LAUNCH_FLAT, **kw).calibrate()
        for x, y in zip(a, b):
            assert x["index"] == y["index"] and x["loss"] == y["loss"] and x["loss_search"] == y["loss_search"]
