"""Edge cases of the CUDA path against the FP64 oracle (GPU only): the largest parameter vector
(K = 29 segments, 32 parameters), the longest window (4096 observations), and degenerate
parameters (no transmission, no removal, no infected)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2204_12346_gb300 import configs, sird, synth
from test_gpu_adjoint import check_f32_gradient, f32_loss_grad, gpu_loss_grad
from util import assert_fp32_losses, box_thetas, f32, rel_err, window

pytestmark = pytest.mark.gpu

K_MAX = 29  # SIRD_MAX_PARAMS - 3: beta segments plus gamma, mu, I0
N_OBS_MAX = 4096  # SIRD_MAX_OBS


@pytest.fixture(scope="module", autouse=True)
def _dev():
    torch.cuda.set_device(0)
    O.build()


def gpu_eval(cal, thetas, precision):
    dt = torch.float32 if precision == 32 else torch.float64
    th = torch.from_numpy(np.ascontiguousarray(np.asarray(thetas).T)).to(dt).cuda()
    out = cal.eval(th, precision=precision)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def calibrator(y, N, K, spd, precision, cost=sird.COST_MSE, M=32, iters=1, **kw):
    P = K + 3
    kw.setdefault("lb", [0.0] * P)
    kw.setdefault("ub", [1e6] * P)
    return sird.Calibrator(y, N, K=K, spd=spd, particles=M, iters=iters, precision=precision, cost=cost, **kw)


# ------------------------------------------------------------------ the largest parameter vector

@pytest.mark.parametrize("cost", ["mse", "mxse", "mae", "mape"])
def test_max_segments_eval(cost):
    # 29 segments over 600 steps: every segment starts inside a day
    y, N, _, _ = window("60d")
    th = box_thetas(K_MAX, 256, 31)
    pb = O.Problem(yD=y, N=N, K=K_MAX, spd=10, cost=O.COSTS[cost])
    want = O.losses(pb, th)
    got64 = gpu_eval(calibrator(y, N, K_MAX, 10, 64, sird.COSTS[cost]), th, 64)
    assert np.array_equal(got64, want), rel_err(got64, want).max()
    got32 = gpu_eval(calibrator(y, N, K_MAX, 10, 32, sird.COSTS[cost]), th, 32)
    assert rel_err(got32, want).max() <= 1e-5


def test_max_segments_gradient():
    y, N, _, _ = window("60d")
    th = box_thetas(K_MAX, 40, 32)
    pb = O.Problem(yD=y, N=N, K=K_MAX, spd=10)
    L, G, GU = gpu_loss_grad(calibrator(y, N, K_MAX, 10, 64), th, 7)
    for j in range(th.shape[0]):
        Lo, Go, GUo = O.loss_grad(pb, th[j])
        assert L[j] == Lo and np.array_equal(G[j], Go) and np.array_equal(GU[j], GUo), j
    L, G, _, E = f32_loss_grad(calibrator(y, N, K_MAX, 10, 32), th)
    check_f32_gradient(pb, th, L, G, E)


def test_max_segments_calibration_matches_the_oracle_swarm():
    # the plain FP64 method on linear bounds (a log box decodes through exp, which the two sides
    # need not round alike)
    y, N, _, _ = window("60d", 30)
    lb, ub = configs.bounds(K_MAX, log=False)
    cal = sird.Calibrator(y, N, K=K_MAX, spd=10, particles=96, iters=4, lb=lb, ub=ub, precision=64, seed=5)
    r = cal.calibrate()
    pso = O.PSO(O.Problem(yD=y, N=N, K=K_MAX, spd=10), 96, lb, ub, logdim=[0] * (K_MAX + 3), seed=5).init().step(4)
    st = cal.get_state()
    assert np.array_equal(st["pbest_f"], pso.pbest_f)
    assert r["index"] == pso.gbest_idx and r["loss"] == pso.gbest_f


# ------------------------------------------------------------------ the longest window

def long_window(spd):
    """4096 daily observations (4095 days) of an epidemic held near its threshold: 8 transmission
    segments set to (gamma + mu) N / S at each segment start, +-0.3% (I between 1.3e3 and 2.2e3
    throughout, D reaching 1.4e4), Poisson death counts (seeded)."""
    beta = [0.102311, 0.101996, 0.102887, 0.10253, 0.103391, 0.103001, 0.103833, 0.103406]
    theta = np.array(beta + [0.1, 0.002, 2e3])
    pb = O.Problem(yD=np.zeros(N_OBS_MAX), N=38e6, K=8, spd=spd)
    y = synth.poisson_cumulative(O.simulate(pb, theta)["D"], np.random.default_rng(17))
    return y, 38e6, theta


def test_max_observations_eval():
    y, N, truth = long_window(10)
    rng = np.random.default_rng(18)
    th = f32(truth * np.exp(rng.normal(0.0, 0.02, (24, truth.size))))
    pb = O.Problem(yD=y, N=N, K=8, spd=10)
    want = O.losses(pb, th)
    got64 = gpu_eval(calibrator(y, N, 8, 10, 64), th, 64)
    assert np.array_equal(got64, want), rel_err(got64, want).max()
    got32 = gpu_eval(calibrator(y, N, 8, 10, 32), th, 32)
    # 40950 steps: the long-window mode of the FP32 trajectory keeps the contract's 1e-5
    print("largest relative error", assert_fp32_losses(got32, want, "4096 observations"))


def test_max_observations_batch_equals_single_windows():
    y, N, truth = long_window(10)
    lb, ub = configs.bounds(8, log=True)
    wins = [{"yD": y, "N": N, "R0": 0.0, "particles": 70}, {"yD": y[100:131], "N": N, "R0": 0.0, "particles": 300}]
    kw = dict(K=8, spd=10, lb=lb, ub=ub, log_scale=[1] * 11, seed=4)
    res = sird.Batch(wins, iters=2, **kw).calibrate()
    for i, w in enumerate(wins):
        cal = sird.Calibrator(w["yD"], N, particles=w["particles"], iters=2, precision=32, stream_id=i, reeval_topk=0,
                              **kw)
        r = cal.calibrate()
        assert res[i]["index"] == r["index"] and res[i]["loss"] == r["loss"], i
        assert r["loss"] == O.loss(O.Problem(yD=w["yD"], N=N, K=8, spd=10), r["theta"])


# ------------------------------------------------------------------ degenerate parameters

def degenerate_thetas(K):
    base = np.array([0.2] * K + [0.1, 0.002, 1e4])
    rows = []
    for mod in ({"beta": 0.0}, {"gamma": 0.0, "mu": 0.0}, {"I0": 0.0}, {"beta": 0.0, "gamma": 0.0, "mu": 0.0},
                {"mu": 0.0}, {"beta": 2.0, "I0": 1e6}):
        t = base.copy()
        if "beta" in mod:
            t[:K] = mod["beta"]
        if "gamma" in mod:
            t[K] = mod["gamma"]
        if "mu" in mod:
            t[K + 1] = mod["mu"]
        if "I0" in mod:
            t[K + 2] = mod["I0"]
        rows.append(t)
    return f32(np.array(rows))


@pytest.mark.parametrize("cost", ["mse", "mxse", "mae", "mape"])
def test_degenerate_parameters(cost):
    y, N, _, _ = window("60d", 40)
    K = 3
    th = degenerate_thetas(K)
    pb = O.Problem(yD=y, N=N, K=K, spd=10, cost=O.COSTS[cost])
    want = O.losses(pb, th)
    got64 = gpu_eval(calibrator(y, N, K, 10, 64, sird.COSTS[cost]), th, 64)
    assert np.array_equal(got64, want), rel_err(got64, want).max()
    got32 = gpu_eval(calibrator(y, N, K, 10, 32, sird.COSTS[cost]), th, 32)
    assert_fp32_losses(got32, want, cost)
    # no removal (gamma = mu = 0) or no infected (I0 = 0): D stays at D0 = y_0, so the cost is
    # that of the constant y_0
    e = np.asarray(y, dtype=np.float64) - y[0]
    const = {"mse": np.mean(e * e), "mxse": np.max(e * e), "mae": np.mean(np.abs(e)),
             "mape": 100.0 * np.mean(np.abs(e[y != 0] / y[y != 0]))}[cost]
    for j in (1, 2, 3):
        assert rel_err(want[j], const) <= 1e-14, (j, want[j], const)
        assert got64[j] == want[j]


def zero_beta_thetas(K, seed):
    """Segments with beta = 0 before, between and after ones with beta > 0, next to rows without
    any: the FP32 trajectory recovers Q from G = cb Q - a where a segment starts, which says
    nothing about Q after a segment with cb = 0 (Q is then carried through that segment)."""
    patterns = [[0, .2, .2, .2], [.2, 0, .2, .2], [.2, .2, 0, .25], [0, .3, 0, .2], [.2, .2, .2, 0], [0, 0, .3, .2],
                [.25, 0, 0, .2], [0, 0, 0, .3]]
    rng = np.random.default_rng(seed)
    rows = []
    for p in patterns:
        for _ in range(3):
            rows.append(list(np.array(p) * rng.uniform(0.8, 1.2)) + [rng.uniform(0.05, 0.15), 0.002, 1e4])
            rows.append(list(rng.uniform(0.1, 0.3, K)) + [0.1, 0.002, rng.uniform(5e3, 2e4)])
    return f32(np.array(rows))


@pytest.mark.parametrize("cost", ["mse", "mape"])
def test_zero_beta_segments(cost):
    y, N, _, _ = window("60d", 40)
    K = 4
    th = zero_beta_thetas(K, 3)
    pb = O.Problem(yD=y, N=N, K=K, spd=10, cost=O.COSTS[cost])
    want = O.losses(pb, th)
    assert np.array_equal(gpu_eval(calibrator(y, N, K, 10, 64, sird.COSTS[cost]), th, 64), want)
    cal = calibrator(y, N, K, 10, 32, sird.COSTS[cost])
    got = gpu_eval(cal, th, 32)
    print("largest relative error", assert_fp32_losses(got, want, cost))
    # each lane of a packed pair on its own: other partners give the same bits
    perm = np.random.default_rng(4).permutation(len(th))
    assert np.array_equal(gpu_eval(cal, th[perm], 32), got[perm])
    # the adjoint's forward pass carries Q every day (its checkpoints read it); its loss is still
    # the evaluation's bit for bit
    L, _, _, E = f32_loss_grad(cal, th)
    assert np.array_equal(L, E) and np.array_equal(E.astype(np.float64), got)


def test_swarm_with_a_segment_held_at_beta_zero():
    # a linear box whose second segment is held at beta = 0 (lb = ub = 0) and whose first may
    # reach it: every particle's trajectory carries Q through the segment without transmission;
    # the FP32 losses of positions and personal bests are the oracle's within 1e-5 and the batch
    # form agrees with the single window bit for bit
    y, N, _, _ = window("60d", 40)
    K = 4
    lb, ub = [0.0, 0.0, 0.0, 0.0, 0.02, 1e-4, 1e3], [0.02, 0.0, 0.5, 0.5, 0.3, 0.01, 5e4]
    kw = dict(K=K, spd=10, lb=lb, ub=ub, seed=9)
    cal = sird.Calibrator(y, N, particles=512, iters=6, precision=32, **kw)
    r = cal.calibrate()
    st = cal.get_state()
    x = f32(st["x"].T)
    assert np.all(x[:, 1] == 0.0)
    pb = O.Problem(yD=y, N=N, K=K, spd=10)
    print("largest relative error", assert_fp32_losses(gpu_eval(cal, x, 32), O.losses(pb, x), "positions"))
    pbest = f32(st["pbest"].T)
    print("largest relative error", assert_fp32_losses(st["pbest_f"], O.losses(pb, pbest), "personal bests"))
    res = sird.Batch([{"yD": y, "N": N, "particles": 512}], iters=6, **kw).calibrate()
    assert res[0]["index"] == r["index"] and res[0]["loss"] == r["loss"]


# ------------------------------------------------------------------ the shortest window, a batch of one

@pytest.mark.parametrize("cost", ["mse", "mxse", "mae", "mape"])
@pytest.mark.parametrize("spd", [10, 1])
def test_one_day_window(cost, spd):
    # two observations (days 0 and 1): FP64 losses, a plain FP64 calibration and the FP64 adjoint
    # identical to the oracle's; FP32 losses within 1e-5 and the FP32 loss of the adjoint equal to
    # the FP32 evaluation's
    y, N, _, _ = window("60d", 1)
    assert len(y) == 2
    th = box_thetas(2, 64, 41)
    pb = O.Problem(yD=y, N=N, K=2, spd=spd, cost=O.COSTS[cost])
    want = O.losses(pb, th)
    c64 = calibrator(y, N, 2, spd, 64, sird.COSTS[cost])
    assert np.array_equal(gpu_eval(c64, th, 64), want)
    got32 = gpu_eval(calibrator(y, N, 2, spd, 32, sird.COSTS[cost]), th, 32)
    assert_fp32_losses(got32, want, ("one day", cost, spd))
    L, G, GU = gpu_loss_grad(c64, th, 3)
    for j in range(th.shape[0]):
        Lo, Go, GUo = O.loss_grad(pb, th[j])
        assert L[j] == Lo and np.array_equal(G[j], Go) and np.array_equal(GU[j], GUo), j
    lb, ub = configs.bounds(2, log=False)
    res = calibrator(y, N, 2, spd, 64, sird.COSTS[cost], M=48, iters=6, lb=lb, ub=ub, seed=4).calibrate()
    pso = O.PSO(pb, 48, lb, ub, seed=4).init().step(6)
    assert res["index"] == pso.gbest_idx and res["loss"] == pso.gbest_f
    assert np.array_equal(res["theta"], pso.gbest)
    c32 = calibrator(y, N, 2, spd, 32, sird.COSTS[cost])
    L32, _, _, E32 = f32_loss_grad(c32, f32(th))
    assert np.array_equal(L32, E32)


def test_batch_of_one_window():
    # a batch holding a single window (one block at work, the rest of the grid idle) equals the
    # window's own calibration bit for bit, in both launch forms
    ser = synth.load_series("450d")
    wins = synth.rolling_window_problems(ser, {"L": np.array([37]), "M": np.array([700]), "T": np.array([90])})
    lb, ub = configs.bounds(3, log=True)
    kw = dict(K=3, spd=10, lb=lb, ub=ub, log_scale=[1] * 6, seed=8)
    w = wins[0]
    cal = sird.Calibrator(w["yD"], w["N"], R0=w["R0"], particles=w["particles"], iters=9, precision=32, stream_id=0,
                          reeval_topk=0, **kw)
    one = cal.calibrate()
    for mode in (sird.LAUNCH_WINDOW_PER_BLOCK, sird.LAUNCH_FLAT):
        got = sird.Batch(wins, iters=9, launch_mode=mode, **kw).calibrate()
        assert len(got) == 1
        assert got[0]["index"] == one["index"] and got[0]["loss"] == one["loss"], (mode, got[0], one)
        assert got[0]["loss_search"] == one["loss_search"] and np.array_equal(got[0]["theta"], one["theta"]), mode
