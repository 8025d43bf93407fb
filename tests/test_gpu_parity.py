"""CUDA path vs the FP64 oracle, element by element, through the C ABI (GPU only).

Tolerances: FP32 fitness within 1e-5 relative of the oracle, FP64
within 1e-12; the FP64 path is written in the paper's operation order without FMA
contraction, so it is expected to match the oracle bit for bit.  Parameter vectors are
drawn from the PSO search box and rounded to FP32 before both sides see them.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2204_12346_gb300 import configs, sird, synth
from util import box_thetas, f32, log_box, rel_err, window

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _dev():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    O.build()


def cal_for(y, N, K, spd, precision=32, cost=sird.COST_MSE, beta_form=sird.BETA_PWC, M=32, **kw):
    P = (6 if beta_form == sird.BETA_RAMP else K + 2) + 1
    lb, ub = kw.pop("lb", None), kw.pop("ub", None)
    if lb is None:
        lb, ub = [1e-3] * P, [1e6] * P
    return sird.Calibrator(y, N, K=K, spd=spd, particles=M, iters=1, lb=lb, ub=ub, precision=precision, cost=cost,
                           beta_form=beta_form, **kw)


def gpu_eval(cal, thetas, precision):
    dt = torch.float32 if precision == 32 else torch.float64
    th = torch.from_numpy(np.ascontiguousarray(np.asarray(thetas).T)).to(dt).cuda()
    out = cal.eval(th, precision=precision)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def orc_problem(y, N, K, spd, cost=O.MSE, beta_form=O.BETA_PWC):
    return O.Problem(yD=y, N=N, K=K, spd=spd, cost=cost, beta_form=beta_form)


CASES = [
    # series, days, K, spd
    ("60d", None, 4, 10),     # 60 days, 4 segments, unrolled 10-step days
    ("90d", None, 4, 20),     # 90 days at dt = 0.05
    ("134d", 120, 10, 20),     # 120 days, 10 segments
    ("60d", 22, 6, 10),       # ragged: segment starts inside a day
    ("60d", 17, 5, 7),        # steps per day not specialised
    ("30d", 3, 6, 1),         # segments shorter than a day, one step per day
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("cost", ["mse", "mxse", "mae", "mape"])
def test_eval_f32_box_samples(case, cost):
    name, days, K, spd = case
    y, N, _, _ = window(name, days)
    thetas = box_thetas(K, 1000 - 13, seed=100 * K + spd)
    cal = cal_for(y, N, K, spd, 32, sird.COSTS[cost])
    got = gpu_eval(cal, thetas, 32)
    want = O.losses(orc_problem(y, N, K, spd, O.COSTS[cost]), thetas)
    err = rel_err(got, want)
    assert np.all(np.isfinite(got))
    assert err.max() <= TOL32, (err.max(), int(err.argmax()))


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("cost", ["mse", "mxse", "mae", "mape"])
def test_eval_f64_bit_exact(case, cost):
    name, days, K, spd = case
    y, N, _, _ = window(name, days)
    rng = np.random.default_rng(7)
    lb, ub = log_box(K)
    thetas = synth.box_sample(lb, ub, [1] * len(lb), 300, rng)
    cal = cal_for(y, N, K, spd, 64, sird.COSTS[cost])
    got = gpu_eval(cal, thetas, 64)
    want = O.losses(orc_problem(y, N, K, spd, O.COSTS[cost]), thetas)
    assert np.array_equal(got, want), rel_err(got, want).max()


def test_eval_ramp_form():
    y, N, _, _ = window("60d", 36)
    rng = np.random.default_rng(3)
    M = 500
    th = np.column_stack([rng.uniform(0.05, 0.6, M), rng.uniform(0.05, 0.6, M), rng.uniform(0, 36, M),
                          rng.uniform(0, 36, M), rng.uniform(0.02, 0.3, M), rng.uniform(1e-4, 0.01, M),
                          rng.uniform(1e3, 5e4, M)])
    th = f32(th)
    pb = orc_problem(y, N, 1, 10, beta_form=O.BETA_RAMP)
    want = O.losses(pb, th)
    cal32 = cal_for(y, N, 1, 10, 32, beta_form=sird.BETA_RAMP)
    assert rel_err(gpu_eval(cal32, th, 32), want).max() <= TOL32
    cal64 = cal_for(y, N, 1, 10, 64, beta_form=sird.BETA_RAMP)
    assert np.array_equal(gpu_eval(cal64, th, 64), want)


def test_eval_fixed_I0_and_nonzero_R0():
    y, N, _, _ = window("60d", 30)
    y = y + 500.0
    thetas = box_thetas(4, 300, 11)[:, :6]
    cal = sird.Calibrator(y, N, K=4, spd=10, R0=2.5e4, I0=7.7e3, fit_I0=False, particles=32, iters=1,
                          lb=[1e-3] * 6, ub=[2] * 6, precision=32)
    got = gpu_eval(cal, thetas, 32)
    want = O.losses(O.Problem(yD=y, N=N, K=4, spd=10, R0=2.5e4, I0=7.7e3, fit_I0=False), thetas)
    assert rel_err(got, want).max() <= TOL32


def test_eval_f32_full_size_sampled():
    # the largest configuration: 2^20 parameter vectors, 120 days at dt = 0.05, K = 10
    y, N, _, _ = window("134d", 120)
    M = 1 << 20
    thetas = box_thetas(10, M, 5)
    cal = cal_for(y, N, 10, 20, 32)
    got = gpu_eval(cal, thetas, 32)
    assert np.all(np.isfinite(got))
    idx = np.random.default_rng(0).choice(M, 300, replace=False)
    want = O.losses(orc_problem(y, N, 10, 20), thetas[idx])
    assert rel_err(got[idx], want).max() <= TOL32


# ------------------------------------------------------------------ swarm

def plain64_setup(M=100):
    ser = synth.load_series("30d")
    lb, ub = configs.bounds(1, log=False)
    return ser["yD"], ser["N"], lb, ub


def test_pso_f64_bit_exact_with_oracle():
    y, N, lb, ub = plain64_setup()
    M = 100
    cal = sird.Calibrator(y, N, K=1, spd=10, particles=M, iters=5, lb=lb, ub=ub, precision=64, seed=3)
    pso = O.PSO(O.Problem(yD=y, N=N, K=1, spd=10), M, lb, ub, seed=3).init()
    cal.init()
    for t in range(6):
        st = cal.get_state()
        assert np.array_equal(st["x"], pso.x.T), t
        assert np.array_equal(st["v"], pso.v.T), t
        assert np.array_equal(st["pbest"], pso.pbest.T), t
        assert np.array_equal(st["pbest_f"], pso.pbest_f), t
        assert st["gbest_idx"] == pso.gbest_idx
        cal.step(1)
        pso.step(1)


def test_calibrate_f64_plain_method_matches_oracle():
    # the plain64 configuration: FP64, K = 1 plus I0, 30 days, 64 particles, 200 iterations, seed 0
    y, N, lb, ub = plain64_setup()
    c = configs.CONFIGS["plain64"]
    cal = sird.Calibrator(y, N, K=1, spd=10, particles=c["M"], iters=c["iters"], lb=lb, ub=ub, precision=64, seed=0)
    res = cal.calibrate()
    pso = O.PSO(O.Problem(yD=y, N=N, K=1, spd=10), c["M"], lb, ub, seed=0).init().step(c["iters"])
    assert res["index"] == pso.gbest_idx
    assert res["loss"] == pso.gbest_f
    assert np.array_equal(res["theta"], pso.gbest)
    assert res["iters_done"] == c["iters"]
    assert res["r2_D"] == pytest.approx(O.r2_D(O.Problem(yD=y, N=N, K=1, spd=10), pso.gbest), rel=1e-12)
    # a second call replays the captured graph and gives the same answer
    assert cal.calibrate()["loss"] == res["loss"]


def _f32_state_from_oracle(K, M, seed):
    y, N, _, _ = window("60d")
    lb, ub = log_box(K)
    zlb, zub = f32(np.log(lb)), f32(np.log(ub))
    pb = O.Problem(yD=y, N=N, K=K, spd=10)
    pso = O.PSO(pb, M, zlb, zub, logdim=[1] * len(lb), seed=seed, store_f32=True).init().step(3)
    return y, N, lb, ub, zlb, zub, pb, pso


def test_pso_f32_single_step_matches_oracle():
    K, M, seed = 4, 1000, 12
    y, N, lb, ub, zlb, zub, pb, pso = _f32_state_from_oracle(K, M, seed)
    cal = sird.Calibrator(y, N, K=K, spd=10, particles=M, iters=1, lb=lb, ub=ub, log_scale=[1] * 7,
                          precision=32, seed=seed)
    cal.set_state(pso.x.T, pso.v.T, pso.pbest.T, pso.pbest_f, pso.gbest_idx, pso.iter)
    old_pf = pso.pbest_f.copy()
    cal.step(1)
    pso.step(1)
    st = cal.get_state()
    rng_ = (zub - zlb)[:, None]
    assert np.all(np.abs(st["v"] - pso.v.T) <= TOL32 * (np.abs(pso.v.T) + rng_))
    assert np.all(np.abs(st["x"] - pso.x.T) <= TOL32 * (np.abs(pso.x.T) + rng_))
    f_new = np.array([pso.objective(pso.x[p]) for p in range(M)])
    margin = np.abs(f_new - old_pf) / np.abs(old_pf)
    decided = margin > 3 * TOL32
    gpu_improved = st["pbest_f"] < old_pf
    orc_improved = pso.pbest_f < old_pf
    assert np.array_equal(gpu_improved[decided], orc_improved[decided])
    both = gpu_improved & orc_improved
    assert rel_err(st["pbest_f"][both], pso.pbest_f[both]).max() <= TOL32
    assert np.array_equal(st["pbest_f"][~gpu_improved], old_pf[~gpu_improved])
    # global best: unique when the two smallest personal bests are further apart than the tolerance
    s = np.sort(pso.pbest_f)
    if (s[1] - s[0]) > 3 * TOL32 * s[0]:
        assert st["gbest_idx"] == pso.gbest_idx


def test_state_save_restore_is_bit_identical():
    y, N, _, _ = window("60d")
    lb, ub = log_box(4)
    kw = dict(K=4, spd=10, particles=300, iters=10, lb=lb, ub=ub, log_scale=[1] * 7, precision=32, seed=9)
    a = sird.Calibrator(y, N, **kw).init().step(8)
    sa = a.get_state()
    b = sird.Calibrator(y, N, **kw).init().step(4)
    sb = b.get_state()
    c = sird.Calibrator(y, N, **kw)
    c.set_state(sb["x"], sb["v"], sb["pbest"], sb["pbest_f"], sb["gbest_idx"], sb["iter"])
    c.step(4)
    sc = c.get_state()
    for k in ("x", "v", "pbest", "pbest_f", "gbest_idx", "iter"):
        assert np.array_equal(np.asarray(sa[k]), np.asarray(sc[k])), k


@pytest.mark.parametrize("k", [1, 32, 200])
def test_topk_reevaluation_matches_oracle(k):
    K, M, seed = 4, 1000, 21
    y, N, lb, ub, zlb, zub, pb, pso = _f32_state_from_oracle(K, M, seed)
    cal = sird.Calibrator(y, N, K=K, spd=10, particles=M, iters=1, lb=lb, ub=ub, log_scale=[1] * 7,
                          precision=32, seed=seed, reeval_topk=k)
    cal.set_state(pso.x.T, pso.v.T, pso.pbest.T, pso.pbest_f, pso.gbest_idx, pso.iter)
    res = cal.result()
    idx, f = pso.reeval_topk(k)
    assert res["index"] == idx
    assert rel_err(res["loss"], f) <= TOL64
    assert res["loss_search"] == pso.pbest_f[idx]


@pytest.mark.parametrize("M", [1, 31, 33, 129])
def test_small_and_ragged_swarms(M):
    y, N, lb, ub = plain64_setup()
    cal = sird.Calibrator(y, N, K=1, spd=10, particles=M, iters=7, lb=lb, ub=ub, precision=64, seed=M)
    res = cal.calibrate()
    pso = O.PSO(O.Problem(yD=y, N=N, K=1, spd=10), M, lb, ub, seed=M).init().step(7)
    assert res["index"] == pso.gbest_idx and res["loss"] == pso.gbest_f


def test_one_day_window():
    y = np.array([12.0, 20.0])
    th = f32([[0.3, 0.1, 0.002, 5e3], [1.9, 0.9, 0.09, 9e5]])
    cal = cal_for(y, 38e6, 1, 10, 32)
    want = O.losses(O.Problem(yD=y, N=38e6, K=1, spd=10), th)
    assert rel_err(gpu_eval(cal, th, 32), want).max() <= TOL32


@pytest.mark.parametrize("M,block", [(4096, 0), (4096, 256), (1000, 64), (77, 32), (16384, 0), (333, 0)])
def test_cluster_and_per_iteration_launches_agree_bit_for_bit(M, block):
    # all iterations in one thread-block cluster, the blocks' best exchanged in shared memory
    y, N, _, _ = window("60d")
    lb, ub = log_box(4)
    kw = dict(K=4, spd=10, particles=M, iters=25, lb=lb, ub=ub, log_scale=[1] * 7, precision=32, seed=5,
              reeval_topk=8, block_size=block)
    a = sird.Calibrator(y, N, launch_mode=sird.LAUNCH_PER_ITER, **kw)
    b = sird.Calibrator(y, N, launch_mode=sird.LAUNCH_CLUSTER, **kw)
    assert b.launch_mode == sird.LAUNCH_CLUSTER
    ra, rb = a.calibrate(), b.calibrate()
    assert ra["index"] == rb["index"] and ra["loss"] == rb["loss"] and ra["loss_search"] == rb["loss_search"]
    sa, sb = a.get_state(), b.get_state()
    for k in ("x", "v", "pbest", "pbest_f", "gbest_idx"):
        assert np.array_equal(np.asarray(sa[k]), np.asarray(sb[k])), k
    c = sird.Calibrator(y, N, launch_mode=sird.LAUNCH_CLUSTER, **kw).init()
    c.step(10)
    c.step(15)
    sc = c.get_state()
    for k in ("x", "v", "pbest", "pbest_f", "gbest_idx"):
        assert np.array_equal(np.asarray(sa[k]), np.asarray(sc[k])), k


def test_cluster_launch_refuses_a_swarm_beyond_one_cluster():
    y, N, _, _ = window("60d", 20)
    lb, ub = log_box(4)
    with pytest.raises(sird.SirdError) as e:
        sird.Calibrator(y, N, K=4, spd=10, particles=4096, iters=2, lb=lb, ub=ub, log_scale=[1] * 7, precision=32,
                        block_size=128, launch_mode=sird.LAUNCH_CLUSTER)  # 32 blocks
    assert e.value.status == 7


@pytest.mark.parametrize("M,block", [(4096, 128), (1000, 64), (77, 32)])
def test_persistent_and_per_iteration_launches_agree_bit_for_bit(M, block):
    y, N, _, _ = window("60d")
    lb, ub = log_box(4)
    kw = dict(K=4, spd=10, particles=M, iters=25, lb=lb, ub=ub, log_scale=[1] * 7, precision=32, seed=5,
              reeval_topk=8, block_size=block)
    a = sird.Calibrator(y, N, launch_mode=sird.LAUNCH_PER_ITER, **kw)
    b = sird.Calibrator(y, N, launch_mode=sird.LAUNCH_PERSISTENT, **kw)
    ra, rb = a.calibrate(), b.calibrate()
    assert ra["index"] == rb["index"] and ra["loss"] == rb["loss"] and ra["loss_search"] == rb["loss_search"]
    sa, sb = a.get_state(), b.get_state()
    for k in ("x", "v", "pbest", "pbest_f", "gbest_idx"):
        assert np.array_equal(np.asarray(sa[k]), np.asarray(sb[k])), k
    # stepping in pieces through the persistent kernel continues the same swarm
    c = sird.Calibrator(y, N, launch_mode=sird.LAUNCH_PERSISTENT, **kw).init()
    c.step(10)
    c.step(15)
    sc = c.get_state()
    for k in ("x", "v", "pbest", "pbest_f", "gbest_idx"):
        assert np.array_equal(np.asarray(sa[k]), np.asarray(sc[k])), k
