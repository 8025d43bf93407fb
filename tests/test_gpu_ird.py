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


def test_ird_fp32_at_fits_where_the_reported_R_passes_2_to_the_24():
    # Late windows of the paper's F_IRD^MXSE setting: the reported R is above 2^24 (float
    # integers are then even numbers only) and at a fit R's misfit on the last day is ~1e-3 of R
    # and sets the cost.  The FP32 path takes the series' day-to-day changes exactly (its copy of
    # D and R holds y - y_0), so the search loss stays within 1e-5 of the oracle at the fitted
    # points; rounding the levels themselves to float put four of these windows 6e-5 .. 3e-4 off.
    c = configs.CONFIGS["paper_ird"]
    ser = synth.reported_IR(synth.load_series(c["series"]), c["seed"])
    lay = synth.rolling_windows(W=c["W"], L_min=c["L_min"], L_max=c["L_max"], M_min=c["M_min"], M_max=c["M_max"],
                                delta=c["delta"], seed=c["seed"])
    every = synth.rolling_window_problems(ser, lay)
    wins = []
    for i in (92, 110, 116, 136):  # with their Philox streams in the full 139-window batch
        wins.append(dict(every[i], stream_id=i))
    assert all(w["yR"].max() > 2 ** 24 for w in wins)
    lb, ub = configs.bounds_ramp(fit_I0=False)
    kw = dict(K=1, spd=10, beta_form=sird.BETA_RAMP, lb=lb, ub=ub, log_scale=None, fit_I0=False, seed=0,
              objective=sird.FIT_IRD, cost=sird.COST_MXSE)
    res = sird.Batch(wins, iters=100, **kw).calibrate()
    got, want = [], []
    for w, r in zip(wins, res):
        pb = O.Problem(yD=w["yD"], yI=w["yI"], yR=w["yR"], N=w["N"], R0=w["R0"], I0=w["I0"], fit_I0=False,
                       beta_form=O.BETA_RAMP, spd=10, cost=O.MXSE, objective=O.FIT_IRD)
        got.append(r["loss_search"])
        want.append(O.loss(pb, f32(r["theta"])))
    print("largest relative error", assert_fp32_losses(got, want, "R above 2^24"))


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


# ---------------------------------------------------------------- F_IRD^C gradient (FP64 adjoint)

def dominated_problem(form, cost, dominant, fit_I0, days=35):
    """Reported series from a trajectory with 0.2% noise, one compartment moved 5-8% off it so that
    its normalised cost is the largest of the three (F_IRD^C, Sec. 3.1); returns the GPU keywords,
    the oracle problem and parameter vectors around the generating point."""
    s = synth.load_series("60d")
    R0 = 800.0
    if form == "pwc":
        ref, kw, gkw = [0.23, 0.19, 0.17, 0.13, 0.1, 0.002, 1.1e4], dict(K=4), dict(K=4, beta_form=sird.BETA_PWC)
    else:
        ref, kw, gkw = [0.25, 0.14, 9.5, 24.25, 0.1, 0.002, 1.1e4], dict(beta_form=O.BETA_RAMP), \
            dict(K=1, beta_form=sird.BETA_RAMP)
    th0 = np.array(ref) * (1 + 0.03 * np.sin(np.arange(len(ref)) + 1.0))
    tr = O.simulate(O.Problem(yD=np.zeros(days + 1), N=s["N"], R0=R0, spd=10, **kw), th0, days)
    rng = np.random.default_rng(11)
    wob = lambda v, a: v * (1 + a * rng.normal(size=v.size))
    yI, yR = wob(tr["I"], 2e-3), R0 + wob(tr["R"] - R0, 2e-3)
    yD = tr["D"][0] + wob(tr["D"] - tr["D"][0], 2e-3)
    t = np.linspace(0.0, 1.0, days + 1)
    if dominant == "I":
        yI = yI * (1 + 0.08 * t)
    elif dominant == "R":
        yR = R0 + (yR - R0) * (1 + 0.08 * t)
    else:
        yD = yD + 0.08 * t * (yD - yD[0])
    pb = O.Problem(yD=yD, yI=yI, yR=yR, N=s["N"], R0=R0, I0=float(yI[0]), fit_I0=fit_I0, spd=10,
                   objective=O.FIT_IRD, cost=O.COSTS[cost], **kw)
    th0 = th0 if fit_I0 else th0[:-1]
    th = th0 * np.exp(np.random.default_rng(12).normal(0.0, 0.01, (48, th0.size)))
    th[0] = th0
    P = th.shape[1]
    common = dict(spd=10, R0=R0, I0=float(yI[0]), fit_I0=fit_I0, cost=sird.COSTS[cost], objective=sird.FIT_IRD,
                  yI=yI, yR=yR, particles=32, iters=1, lb=[0.0] * P, ub=[1e6] * P, **gkw)
    return yD, float(s["N"]), pb, th, common


def compartment_costs(pb, th):
    tr = O.simulate(pb, th, len(pb.yD) - 1)
    out = []
    for y, yh in ((pb.yI, tr["I"]), (pb.yR, tr["R"]), (pb.yD, tr["D"])):
        if pb.cost == O.MAPE:
            m = y != 0
            out.append(100 * np.mean(np.abs((y[m] - yh[m]) / y[m])))
        else:
            e = (y - yh) / (y.max() - y.min())
            out.append({O.MSE: np.mean(e * e), O.MAE: np.mean(np.abs(e)), O.MXSE: np.max(e * e)}[pb.cost])
    return out


@pytest.mark.parametrize("form,cost,dominant,fit_I0", [
    ("pwc", "mse", "I", True), ("pwc", "mse", "R", True), ("pwc", "mse", "D", True),
    ("pwc", "mae", "R", True), ("pwc", "mape", "D", True), ("pwc", "mxse", "I", True), ("pwc", "mxse", "R", False),
    ("ramp", "mxse", "I", False), ("ramp", "mxse", "R", False), ("ramp", "mxse", "D", False),
    ("ramp", "mse", "D", False), ("ramp", "mape", "I", False), ("ramp", "mae", "D", True), ("ramp", "mape", "R", True)])
@pytest.mark.parametrize("ckpt", [1, 7, 16, 64])
def test_ird_adjoint_f64_bit_exact(form, cost, dominant, fit_I0, ckpt):
    # the FP64 adjoint of F_IRD^C against the oracle's discrete adjoint: loss, dL/dtheta and
    # dL/du0 identical, with the named compartment attaining the maximum at the generating point
    yD, N, pb, th, common = dominated_problem(form, cost, dominant, fit_I0)
    c = compartment_costs(pb, th[0])
    assert "IRD"[int(np.argmax(c))] == dominant, c
    cal = sird.Calibrator(yD, N, precision=64, **common)
    L, G, GU = cal.loss_grad(torch.from_numpy(np.ascontiguousarray(th.T)).cuda(), ckpt_every=ckpt, grad_u0=True)
    L, G, GU = L.cpu().numpy(), G.cpu().numpy().T, GU.cpu().numpy().T
    for j in range(th.shape[0]):
        Lo, Go, GUo = O.loss_grad(pb, th[j])
        assert L[j] == Lo, (j, L[j], Lo)
        assert np.array_equal(G[j], Go), (j, rel_err(G[j], Go))
        assert np.array_equal(GU[j], GUo), (j, GU[j], GUo)


@pytest.mark.parametrize("cost", ["mse", "mxse", "mae", "mape"])
def test_ird_adjoint_f64_box_samples_bit_exact(cost):
    # far from a fit too (random vectors, the dominant compartment varying between them)
    yD, N, th, common, pb = setup(cost, "pwc", days=30)
    cal = sird.Calibrator(yD, N, precision=64, **common)
    L, G = cal.loss_grad(torch.from_numpy(np.ascontiguousarray(th.T)).cuda(), ckpt_every=16)
    L, G = L.cpu().numpy(), G.cpu().numpy().T
    seen = set()
    for j in range(th.shape[0]):
        Lo, Go, _ = O.loss_grad(pb, th[j])
        assert L[j] == Lo and np.array_equal(G[j], Go), (j, rel_err(G[j], Go))
        seen.add(int(np.argmax(compartment_costs(pb, th[j]))))
    print("dominant compartments seen:", sorted("IRD"[i] for i in seen))


def test_ird_fp64_polish_never_worsens_and_reports_the_oracle_loss():
    # the FP64 polish on F_IRD^MXSE (the paper's representative objective, ramp beta)
    yD, yI, yR, N = ird_series("60d", 35)
    lb, ub = configs.bounds_ramp(fit_I0=False)
    cal = sird.Calibrator(yD, N, K=1, spd=10, R0=float(yR[0]), I0=float(yI[0]), fit_I0=False,
                          beta_form=sird.BETA_RAMP, cost=sird.COSTS["mxse"], objective=sird.FIT_IRD, yI=yI, yR=yR,
                          particles=1024, iters=30, lb=lb, ub=ub, precision=32, reeval_topk=8, seed=3)
    r0 = cal.calibrate()
    r1 = cal.polish(k=8, iters=10, first_step=1e-2, precision=64)
    assert r1["loss"] <= r0["loss"]
    assert all(lo <= t <= hi for t, lo, hi in zip(r1["theta"], lb, ub))
    pb = O.Problem(yD=yD, yI=yI, yR=yR, N=N, R0=float(yR[0]), I0=float(yI[0]), fit_I0=False, spd=10,
                   beta_form=O.BETA_RAMP, cost=O.MXSE, objective=O.FIT_IRD)
    assert r1["loss"] == O.loss(pb, r1["theta"])


# ---------------------------------------------------------------- F_IRD^C gradient (FP32 adjoint)

RHO_F32 = 4e-7  # relative accuracy assumed of the FP32 trajectory's I, R, D (as for the F_D gradient)


def ird_residual_bound(pb, th, cost, which, rho=RHO_F32):
    """|theta_j| times the change of dL/dtheta_j that relative errors rho of the dominant series'
    trajectory can cause through its scaled residuals e_i = (y_i - yhat_i) / range (MAPE: unscaled):
    MSE (2/n) sum_i ((rho yhat_i)/range^2) |dyhat_i/dlog theta_j|, MXSE the same at the largest e_i^2,
    MAE / MAPE the residuals within the error band, which may change sign.  Sensitivities by
    central differences of the oracle's trajectory."""
    key, y = ("I", pb.yI) if which == 0 else (("R", pb.yR) if which == 1 else ("D", pb.yD))
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    yh = O.simulate(pb, th, n - 1)[key]
    sc = 1.0 if pb.cost == O.MAPE else (y.max() - y.min())
    Sens = np.zeros((n, th.size))
    for j in range(th.size):
        tp, tm = th.copy(), th.copy()
        tp[j] *= 1 + 1e-5
        tm[j] *= 1 - 1e-5
        Sens[:, j] = (O.simulate(pb, tp, n - 1)[key] - O.simulate(pb, tm, n - 1)[key]) / 2e-5
    dY = rho * np.abs(yh)
    e = (y - yh) / sc
    if cost == "mse":
        return (2.0 / n) * ((dY / sc ** 2)[:, None] * np.abs(Sens)).sum(0)
    if cost == "mxse":
        i = int(np.argmax(e * e))
        near_tie = np.sort(e * e)[-2] > (1 - 1e-4) * e[i] ** 2
        return 2.0 * ((dY[i] / sc + (np.abs(e[i]) if near_tie else 0.0)) / sc) * np.abs(Sens[i])
    w = np.full(n, 1.0 / (n * sc)) if cost == "mae" else np.where(y != 0, 100.0 / np.maximum(np.abs(y), 1e-300)
                                                                  / max(int((y != 0).sum()), 1), 0.0)
    flip = np.abs(y - yh) <= dY
    return 2.0 * ((w * flip)[:, None] * np.abs(Sens)).sum(0)


@pytest.mark.parametrize("form,cost,dominant,fit_I0,days", [
    ("pwc", "mse", "I", True, 35), ("pwc", "mse", "R", True, 35), ("pwc", "mse", "D", True, 35),
    ("pwc", "mae", "R", True, 35), ("pwc", "mape", "D", True, 35), ("pwc", "mxse", "I", True, 35),
    ("ramp", "mxse", "R", False, 35), ("ramp", "mxse", "D", False, 35), ("ramp", "mse", "I", False, 35),
    ("ramp", "mape", "R", True, 35),
    # more than 1000 Euler steps: the trajectory's long-window mode in the forward pass
    ("pwc", "mse", "D", True, 110), ("ramp", "mxse", "I", False, 110)])
def test_ird_adjoint_f32_within_tolerance(form, cost, dominant, fit_I0, days):
    # the FP32 adjoint of F_IRD^C: its loss the FP32 evaluation's bit for bit, its gradient the
    # oracle's FP64 gradient at the same FP32-representable theta within
    #     |theta_j (g32_j - g64_j)| <= 1e-5 (|theta . g64|_inf + L) + ird_residual_bound_j,
    # on points where the dominant compartment is clear (top two costs more than 1e-4 apart)
    yD, N, pb, th, common = dominated_problem(form, cost, dominant, fit_I0, days)
    th = f32(th)
    cal = sird.Calibrator(yD, N, precision=32, **common)
    T = torch.from_numpy(np.ascontiguousarray(th.T).astype(np.float32)).cuda()
    L, G, GU = cal.loss_grad(T, grad_u0=True)
    E = cal.eval(T)
    L, G, GU, E = L.cpu().numpy(), G.cpu().numpy().T.astype(np.float64), GU.cpu().numpy().T, E.cpu().numpy()
    assert np.array_equal(L, E)
    worst, used, seen = 0.0, 0, set()
    for j in range(th.shape[0]):
        c = np.array(compartment_costs(pb, th[j]))
        top = np.sort(c)[::-1]
        if top[0] - top[1] <= 1e-4 * top[0]:
            continue
        which = int(np.argmax(c))
        seen.add(which)
        Lo, Go, GUo = O.loss_grad(pb, th[j])
        tol = 1e-5 * (np.abs(th[j] * Go).max() + abs(Lo)) + ird_residual_bound(pb, th[j], cost, which)
        worst = max(worst, (np.abs(th[j] * (G[j] - Go)) / tol).max())
        if which == 1:
            assert GU[j, 2] != 0.0  # lambda_R(0) carries R's misfit
        used += 1
    assert used >= 24, used
    print("worst gradient error / tolerance", worst, "dominant seen", sorted("IRD"[i] for i in seen))
    assert worst <= 1.0, worst


@pytest.mark.parametrize("form,cost", [("ramp", "mxse"), ("pwc", "mse"), ("pwc", "mape")])
def test_ird_fp32_polish_and_batch_polish(form, cost):
    # FP32 polish of F_IRD (F_IRD^MXSE with the ramp and the data's initial state: the paper's
    # representative setting): never worse than the swarm, reports the oracle's FP64 loss of its
    # point, and a batch of windows polished together gives each window's one-window polish bit
    # for bit
    ser = synth.reported_IR(synth.load_series("450d"), 2)
    lay = {"L": np.array([35, 35, 28]), "M": np.array([600, 900, 320]), "T": np.array([40, 160, 300])}
    wins = synth.rolling_window_problems(ser, lay)
    if form == "ramp":
        lb, ub = configs.bounds_ramp(fit_I0=False)
        kw = dict(K=1, beta_form=sird.BETA_RAMP)
        okw = dict(beta_form=O.BETA_RAMP)
    else:
        lb, ub = configs.bounds(3, log=True)
        lb, ub = lb[:-1], ub[:-1]  # the initial state from the data: no I0 dimension
        kw = dict(K=3, beta_form=sird.BETA_PWC, log_scale=[1] * len(lb))
        okw = dict(K=3)
    kw.update(spd=10, fit_I0=False, cost=sird.COSTS[cost], objective=sird.FIT_IRD, lb=lb, ub=ub, seed=5)
    batch = sird.Batch(wins, iters=20, **kw)
    r0 = batch.calibrate()
    rb = batch.polish(k=4, iters=8, first_step=1e-2)
    for i, w in enumerate(wins):
        pb = O.Problem(yD=w["yD"], yI=w["yI"], yR=w["yR"], N=w["N"], R0=w["R0"], I0=w["I0"], fit_I0=False, spd=10,
                       cost=O.COSTS[cost], objective=O.FIT_IRD, **okw)
        assert rb[i]["loss"] <= r0[i]["loss"]
        assert rb[i]["loss"] == O.loss(pb, rb[i]["theta"])
        cal = sird.Calibrator(w["yD"], w["N"], R0=w["R0"], I0=w["I0"], yI=w["yI"], yR=w["yR"], particles=w["particles"],
                              iters=20, precision=32, stream_id=i, **kw)
        cal.calibrate()
        r1 = cal.polish(k=4, iters=8, first_step=1e-2, precision=32)
        assert r1["loss"] == rb[i]["loss"] and np.array_equal(r1["theta"], rb[i]["theta"]), (i, r1, rb[i])
