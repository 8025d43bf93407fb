"""The benchmark's own configurations at full size, checked on sampled outputs the oracle can
compute one by one (GPU only).

Each test runs the configuration the benchmark times (same sizes, iterations and launch form)
and then checks: the reported loss is the oracle's FP64 loss of the reported theta bit for bit;
sampled personal-best losses (FP32) are the oracle's within 1e-5 at their points; and the
remaining outputs (FP64 re-evaluation choice, gradients, forecasts) against the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2204_12346_gb300 import configs, sird, synth
from util import TOL32, assert_fp32_losses, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    torch.cuda.set_device(0)
    O.build()


def decode(z, logd):
    z = np.asarray(z, dtype=np.float64)
    return np.where(np.asarray(logd, dtype=bool), np.exp(np.where(logd, z, 0.0)), z)


def check_swarm(cal, pb, logd, n_sample, seed):
    """Sampled personal bests of an FP32 swarm: each stored loss is the FP32 evaluation's at the
    point the swarm decoded (theta = exp(z) in FP32 on the GPU, as the kernels decode it), and
    that evaluation is the oracle's FP64 loss at the same FP32 point within the contract's 1e-5."""
    st = cal.get_state()
    M = st["M"]
    idx = np.random.default_rng(seed).choice(M, min(n_sample, M), replace=False)
    z = torch.from_numpy(np.ascontiguousarray(st["pbest"][:, idx])).cuda()
    lg = torch.tensor(np.asarray(logd, dtype=bool)).cuda()[:, None]
    th = torch.where(lg, torch.exp(z), z).contiguous()
    got = cal.eval(th).cpu().numpy()
    assert np.array_equal(got, st["pbest_f"][idx])
    th64 = th.cpu().numpy().astype(np.float64)
    want = np.array([O.loss(pb, th64[:, i]) for i in range(len(idx))])
    print("largest relative error of the sampled personal bests", assert_fp32_losses(got, want, "personal bests"))
    return st


def test_single_window_4096_particles_1000_iterations():
    c = configs.CONFIGS["window60"]
    s = synth.load_series("60d")
    y = s["yD"][: c["days"] + 1]
    lb, ub = configs.bounds(c["K"], True)
    cal = sird.Calibrator(y, s["N"], K=c["K"], spd=c["spd"], particles=c["M"], iters=c["iters"], lb=lb, ub=ub,
                          log_scale=[1] * 7, precision=32, seed=c["seed"], reeval_topk=c["reeval_topk"])
    r = cal.calibrate()
    pb = O.Problem(yD=y, N=s["N"], K=c["K"], spd=c["spd"])
    assert r["loss"] == O.loss(pb, r["theta"])
    st = check_swarm(cal, pb, [1] * 7, 150, 1)
    # the reported point is the FP64 best of the 32 best FP32 personal bests
    order = np.lexsort((np.arange(c["M"]), st["pbest_f"]))[: c["reeval_topk"]]
    f64 = [O.loss(pb, decode(st["pbest"][:, j], [1] * 7)) for j in order]  # decoded in FP64, as re-evaluated
    assert r["index"] == order[int(np.argmin(f64))]


def test_batched_512_windows_100_iterations():
    c = configs.CONFIGS["batch512"]
    ser = synth.load_series("450d")
    lay = synth.rolling_windows(W=c["W"], L_min=c["L_min"], L_max=c["L_max"], M_min=c["M_min"], M_max=c["M_max"],
                                delta=c["delta"], seed=c["seed"])
    wins = synth.rolling_window_problems(ser, lay)
    lb, ub = configs.bounds(c["K"], True)
    batch = sird.Batch(wins, K=c["K"], spd=c["spd"], iters=c["iters"], lb=lb, ub=ub, log_scale=[1] * 9,
                       seed=c["seed"])
    res = batch.calibrate()
    for i in np.random.default_rng(2).choice(len(wins), 8, replace=False):
        w = wins[i]
        pb = O.Problem(yD=w["yD"], N=w["N"], R0=w["R0"], K=c["K"], spd=c["spd"])
        assert res[i]["loss"] == O.loss(pb, res[i]["theta"])
        # the FP32 search loss of the reported point against the oracle at that FP32 point
        th32 = np.asarray(res[i]["theta"], dtype=np.float32).astype(np.float64)
        assert rel_err(res[i]["loss_search"], O.loss(pb, th32)) <= TOL32, i


def test_gradient_4096_personal_bests():
    c = configs.CONFIGS["gradient90"]
    s = synth.load_series("90d")
    y = s["yD"][: c["days"] + 1]
    lb, ub = configs.bounds(c["K"], True)
    cal = sird.Calibrator(y, s["N"], K=c["K"], spd=c["spd"], particles=c["M"], iters=c["iters"], lb=lb, ub=ub,
                          log_scale=[1] * 7, precision=32, seed=c["seed"], reeval_topk=c["reeval_topk"])
    cal.calibrate()
    th = np.exp(cal.get_state()["pbest"].astype(np.float64)).astype(np.float32)
    L, G = cal.loss_grad(torch.from_numpy(np.ascontiguousarray(th)).cuda())
    L, G = L.cpu().numpy(), G.cpu().numpy().astype(np.float64)
    E = cal.eval(torch.from_numpy(np.ascontiguousarray(th)).cuda()).cpu().numpy()
    assert np.array_equal(L, E)
    from test_gpu_adjoint import residual_bound

    pb = O.Problem(yD=y, N=s["N"], K=c["K"], spd=c["spd"])
    for j in np.random.default_rng(3).choice(c["M"], 24, replace=False):
        t = th[:, j].astype(np.float64)
        Lo, Go, _ = O.loss_grad(pb, t)
        tol = 1e-5 * (np.abs(t * Go).max() + abs(Lo)) + residual_bound(pb, t, "mse")
        assert np.all(np.abs(t * (G[:, j] - Go)) <= tol), j


def test_large_swarm_and_forecast():
    c = configs.CONFIGS["swarm2p20"]
    s = synth.load_series("134d")
    y = s["yD"][: c["days"] + 1]
    lb, ub = configs.bounds(c["K"], True)
    cal = sird.Calibrator(y, s["N"], K=c["K"], spd=c["spd"], particles=c["M"], iters=c["iters"], lb=lb, ub=ub,
                          log_scale=[1] * 13, precision=32, seed=c["seed"], reeval_topk=c["reeval_topk"])
    r = cal.calibrate()
    pb = O.Problem(yD=y, N=s["N"], K=c["K"], spd=c["spd"])
    assert r["loss"] == O.loss(pb, r["theta"])
    check_swarm(cal, pb, [1] * 13, 100, 4)
    th, lo = cal.topk(c["forecast_topk"])
    assert np.all(np.diff(lo) >= 0)
    fc = sird.forecast(y, s["N"], th, c["horizon"], K=c["K"], spd=c["spd"], precision=64)
    for j in np.random.default_rng(5).choice(c["forecast_topk"], 12, replace=False):
        assert np.array_equal(fc[j], O.forecast(pb, th[j], c["horizon"])), j
