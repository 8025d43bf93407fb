"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks the oracle against a closed form, an invariant, a published
known-answer vector, a library routine, or brute force, chosen so that a
dropped term, a wrong sign, a wrong index or a swapped operand fails one of them:

  Philox           published known-answer vectors (Salmon et al., SC'11)
  eq. (SIRD)       conservation of N; gamma (D - D0) = mu (R - R0) exactly under Euler;
                   the discrete beta = 0 closed form; the SIR final-size relation;
                   first-order convergence to a tight library ODE solution
  eq. (beta)       ramp with t1 = t2 equals a two-segment step; midpoint value;
                   swapped t1, t2; constant limits
  costs (Sec 3.1)  closed forms for constant and relative offsets; R^2 = 1 at the truth
  adjoint          central finite differences of the loss
  PSO (Sec 3.3)    sphere and Rosenbrock minima; box; monotone personal bests;
                   degenerate coefficient settings
  calibration      noise-free recovery; brute-force grid
"""
import math
import os

import numpy as np
import pytest

from paper_2204_12346_gb300 import synth

N = 38e6


def mkpb(O, days=30, K=1, spd=10, yD=None, **kw):
    if yD is None:
        yD = np.zeros(days + 1)
    return O.Problem(yD=np.asarray(yD, float), N=kw.pop("N", N), K=K, spd=spd, **kw)


# ------------------------------------------------------------------ Philox

def test_philox_known_answers(orc):
    path = os.path.join(os.path.dirname(__file__), "golden", "philox_kat.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = orc.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


def test_u01_conversion(orc):
    assert orc.u01(0) == 0.0
    assert orc.u01(0xFF) == 0.0
    assert orc.u01(0x100) == 2.0 ** -24
    assert orc.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    # uniformity of the stream over many counters
    u = np.array([orc.u01(orc.philox4x32_10([p, 0, 0, 0], [1, 2])[0]) for p in range(4000)])
    assert abs(u.mean() - 0.5) < 0.02 and abs(u.var() - 1 / 12) < 0.01


# ------------------------------------------------------------------ model

def test_conservation_of_N(orc):
    rng = np.random.default_rng(1)
    for form, K in [(orc.BETA_PWC, 4), (orc.BETA_RAMP, 0)]:
        pb = mkpb(orc, days=60, K=K, beta_form=form, R0=1234.0, yD=np.full(61, 77.0))
        for _ in range(5):
            if form == orc.BETA_PWC:
                th = list(rng.uniform(0.05, 0.6, K)) + [rng.uniform(0.02, 0.3), rng.uniform(1e-4, 0.02), 5e4]
            else:
                th = [0.4, 0.15, 12.3, 41.7, 0.1, 0.003, 5e4]
            tr = orc.simulate(pb, th)
            tot = tr["S"] + tr["I"] + tr["R"] + tr["D"]
            assert np.max(np.abs(tot - N)) <= 1e-12 * N


def test_recovered_to_deceased_identity(orc):
    # Both R and D grow by dt*(gamma or mu)*I_k, so gamma (D_k - D0) = mu (R_k - R0) for any beta(t).
    pb = mkpb(orc, days=45, K=3, R0=500.0, yD=np.full(46, 40.0))
    g, m = 0.13, 0.007
    tr = orc.simulate(pb, [0.5, 0.2, 0.35, g, m, 2e4])
    lhs = g * (tr["D"] - tr["D"][0])
    rhs = m * (tr["R"] - tr["R"][0])
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-9)
    assert tr["D"][0] == 40.0 and tr["R"][0] == 500.0


def test_beta_zero_closed_form(orc):
    # beta = 0: I_k = I0 (1 - dt (gamma + mu))^k, D = D0 + mu/(gamma+mu) (I0 - I), S constant.
    days, spd, g, m, I0, D0, R0 = 25, 8, 0.11, 0.013, 3e4, 17.0, 250.0
    pb = mkpb(orc, days=days, K=2, spd=spd, R0=R0, yD=np.full(days + 1, D0))
    tr = orc.simulate(pb, [0.0, 0.0, g, m, I0])
    dt = 1.0 / spd
    k = np.arange(days + 1) * spd
    I_exact = I0 * (1.0 - dt * (g + m)) ** k
    assert np.allclose(tr["I"], I_exact, rtol=1e-12)
    assert np.allclose(tr["D"], D0 + m / (g + m) * (I0 - I_exact), rtol=1e-12)
    assert np.allclose(tr["R"], R0 + g / (g + m) * (I0 - I_exact), rtol=1e-12)
    assert np.all(tr["S"] == tr["S"][0])
    # and it tends to exponential decay as dt -> 0
    errs = []
    for s in (4, 8, 16, 32):
        t2 = orc.simulate(mkpb(orc, days=days, K=1, spd=s, yD=np.zeros(days + 1)), [0.0, g, m, I0])
        errs.append(abs(t2["I"][-1] - I0 * math.exp(-(g + m) * days)))
    assert all(1.8 < errs[i] / errs[i + 1] < 2.2 for i in range(3))


@pytest.mark.parametrize("mu", [0.0, 0.004])
def test_final_size_relation(orc, mu):
    # SIR final size with removed X = R + D: ln(S0/S_inf) = beta (N - S_inf - X0) / ((gamma+mu) N).
    beta, g, I0, days = 0.3, 0.1, 1e3, 700
    res = []
    for spd in (5, 10, 20):
        pb = mkpb(orc, days=days, K=1, spd=spd)
        tr = orc.simulate(pb, [beta, g, mu, I0], days)
        S0, Sinf = tr["S"][0], tr["S"][-1]
        assert tr["I"][-1] < 1e-3 * I0
        res.append(math.log(S0 / Sinf) - beta * (N - Sinf) / ((g + mu) * N))
    assert abs(res[-1]) < 5e-3
    assert 1.8 < res[0] / res[1] < 2.2 and 1.8 < res[1] / res[2] < 2.2


def test_first_order_convergence_to_ode_solution(orc):
    scipy_integrate = pytest.importorskip("scipy.integrate")
    beta, g, m, I0, R0, D0, T = 0.32, 0.1, 0.01, 5e4, 1e3, 20.0, 40

    def rhs(t, u):
        S, I, R, D = u
        return [-beta * S * I / N, beta * I * S / N - (g + m) * I, g * I, m * I]

    sol = scipy_integrate.solve_ivp(rhs, (0, T), [N - I0 - R0 - D0, I0, R0, D0], method="DOP853",
                                    rtol=1e-13, atol=1e-8)
    D_ref = sol.y[3, -1]
    errs = []
    for spd in (10, 20, 40, 80):
        pb = mkpb(orc, days=T, K=1, spd=spd, R0=R0, yD=np.full(T + 1, D0))
        errs.append(orc.simulate(pb, [beta, g, m, I0])["D"][-1] - D_ref)
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(1.85 < r < 2.15 for r in ratios), ratios
    assert abs(errs[-1]) < 2e-2 * D_ref


def test_pwc_segment_schedule(orc):
    th = [0.1, 0.2, 0.3, 0.4, 0.1, 0.01, 1e4]
    pb = mkpb(orc, days=60, K=4, spd=10)
    # 600 steps in 4 equal segments: boundaries at steps 150, 300, 450
    for k, want in [(0, 0.1), (149, 0.1), (150, 0.2), (299, 0.2), (300, 0.3), (450, 0.4), (599, 0.4), (650, 0.4)]:
        assert orc.beta_at(pb, th, k) == want
    # ragged: 22 days * 10 steps / 6 segments -> boundary after step 36.67, i.e. at step 37
    th6 = [1, 2, 3, 4, 5, 6, 0.1, 0.01, 1e4]
    pb6 = mkpb(orc, days=22, K=6, spd=10)
    assert orc.beta_at(pb6, th6, 36) == 1 and orc.beta_at(pb6, th6, 37) == 2
    assert orc.beta_at(pb6, th6, 219) == 6
    # K equal rates reduce to the constant-rate model, bit for bit
    a = orc.simulate(mkpb(orc, days=60, K=4), [0.25] * 4 + [0.1, 0.002, 1e4])
    b = orc.simulate(mkpb(orc, days=60, K=1), [0.25, 0.1, 0.002, 1e4])
    assert all(np.array_equal(a[c], b[c]) for c in "SIRD")


def test_ramp_beta(orc):
    days, spd = 36, 10
    ramp = mkpb(orc, days=days, beta_form=orc.BETA_RAMP, spd=spd)
    two = mkpb(orc, days=days, K=2, spd=spd)
    # t1 = t2 = window midpoint: a step from beta1 to beta2, i.e. two equal segments
    a = orc.simulate(ramp, [0.3, 0.15, 18.0, 18.0, 0.1, 0.004, 2e4])
    b = orc.simulate(two, [0.3, 0.15, 0.1, 0.004, 2e4])
    assert all(np.array_equal(a[c], b[c]) for c in "SIRD")
    # beta1 == beta2 is the constant model whatever t1, t2
    c = orc.simulate(ramp, [0.2, 0.2, 3.3, 20.9, 0.1, 0.004, 2e4])
    d = orc.simulate(mkpb(orc, days=days, K=1, spd=spd), [0.2, 0.1, 0.004, 2e4])
    assert all(np.allclose(c[x], d[x], rtol=1e-14) for x in "SIRD")
    # the ramp is linear: midpoint of [t1, t2) gives the mean rate; ends give beta1 / beta2
    th = [0.5, 0.1, 10.0, 20.0, 0.1, 0.004, 2e4]
    assert orc.beta_at(ramp, th, 150) == pytest.approx(0.3, rel=1e-15)
    assert orc.beta_at(ramp, th, 99) == 0.5 and orc.beta_at(ramp, th, 100) == 0.5
    assert orc.beta_at(ramp, th, 200) == 0.1 and orc.beta_at(ramp, th, 125) == pytest.approx(0.4, rel=1e-15)
    # swapping t1 and t2 changes nothing (the smaller one is the start of the ramp)
    e = orc.simulate(ramp, [0.5, 0.1, 20.0, 10.0, 0.1, 0.004, 2e4])
    f = orc.simulate(ramp, th)
    assert all(np.array_equal(e[x], f[x]) for x in "SIRD")


# ------------------------------------------------------------------ costs

def _model_D(orc, pb, th):
    return orc.simulate(pb, th)["D"]


@pytest.mark.parametrize("D0", [0.0, 5.0])
def test_cost_closed_forms(orc, D0):
    days, th = 30, [0.27, 0.1, 0.003, 1e4]
    n = days + 1
    base = mkpb(orc, days=days, yD=np.full(n, D0))
    Dh = _model_D(orc, base, th)
    c = 37.5
    y = Dh.copy()
    y[1:] += c
    mk = lambda cost: mkpb(orc, days=days, yD=y, cost=cost)
    assert orc.loss(mk(orc.MSE), th) == pytest.approx(c * c * (n - 1) / n, rel=1e-9)
    assert orc.loss(mk(orc.MAE), th) == pytest.approx(c * (n - 1) / n, rel=1e-9)
    assert orc.loss(mk(orc.MXSE), th) == pytest.approx(c * c, rel=1e-9)
    # one larger error on day 7 decides MXSE
    y2 = y.copy()
    y2[7] = Dh[7] - 3 * c
    assert orc.loss(mkpb(orc, days=days, yD=y2, cost=orc.MXSE), th) == pytest.approx(9 * c * c, rel=1e-9)
    # relative offset rho: |e/y| = rho/(1+rho) on days >= 1; day 0 is 0 or skipped when y0 = 0
    rho = 0.04
    y3 = Dh.copy()
    y3[1:] *= 1 + rho
    mape = orc.loss(mkpb(orc, days=days, yD=y3, cost=orc.MAPE), th)
    kept = n if D0 != 0 else n - 1
    assert mape == pytest.approx(100 * rho / (1 + rho) * (n - 1) / kept, rel=1e-9)
    # zero loss at the truth for all four costs
    for cost in (orc.MSE, orc.MXSE, orc.MAE, orc.MAPE):
        assert orc.loss(mkpb(orc, days=days, yD=Dh, cost=cost), th) == 0.0


def test_per_step_schedule_is_the_same_scheme(orc):
    # the generator of the long synthetic series integrates with a per-step rate; fed the PWC
    # model's rates step by step it gives the model's trajectory bit for bit (and so inherits the
    # scheme's pins above)
    days, spd, K = 40, 10, 4
    th = [0.3, 0.2, 0.25, 0.12, 0.1, 0.003, 1.5e4]
    pb = mkpb(orc, days=days, K=K, spd=spd, R0=300.0, yD=np.full(days + 1, 12.0))
    beta = [orc.beta_at(pb, th, k) for k in range(days * spd)]
    tr = orc.simulate(pb, th)
    S0 = N - th[-1] - 300.0 - 12.0
    sc = orc.simulate_schedule(N, (S0, th[-1], 300.0, 12.0), beta, th[K], th[K + 1], spd, days)
    for q in "SIRD":
        assert np.array_equal(sc[q], tr[q]), q


def test_one_day_window(orc):
    # two observations: D after one day at beta = 0 is D0 + mu/(gamma+mu) (I0 - I0 (1 - dt (gamma+mu))^spd),
    # and the MSE is e_1^2 / 2 (e_0 = 0: the scheme starts from the first observation)
    g, m, I0, spd, D0 = 0.1, 0.004, 2e4, 10, 30.0
    D1 = D0 + m / (g + m) * (I0 - I0 * (1 - (g + m) / spd) ** spd)
    for cost, want in ((orc.MSE, 25.0 ** 2 / 2), (orc.MAE, 25.0 / 2), (orc.MXSE, 25.0 ** 2)):
        pb = mkpb(orc, days=1, K=1, spd=spd, yD=[D0, D1 + 25.0], cost=cost)
        assert orc.loss(pb, [0.0, g, m, I0]) == pytest.approx(want, rel=1e-9)
    assert orc.simulate(mkpb(orc, days=1, yD=[D0, 0.0]), [0.0, g, m, I0])["D"][1] == pytest.approx(D1, rel=1e-14)


def test_r2_and_ird(orc):
    days, th = 35, [0.3, 0.1, 0.004, 1e4]
    n = days + 1
    pb = mkpb(orc, days=days)
    tr = orc.simulate(pb, th)
    assert orc.r2_D(mkpb(orc, days=days, yD=tr["D"]), th) == 1.0
    # R^2 = 1 - SS_res / SS_tot by its definition: D offset by c on days 1.. gives SS_res = (n-1) c^2
    yc = tr["D"].copy()
    yc[1:] += 120.0
    want_r2 = 1.0 - (n - 1) * 120.0 ** 2 / np.sum((yc - yc.mean()) ** 2)
    assert orc.r2_D(mkpb(orc, days=days, yD=yc), th) == pytest.approx(want_r2, rel=1e-12)
    # F_IRD^MSE with exact I and R and D offset by c: (c/range(yD))^2 (n-1)/n
    c = 50.0
    yD = tr["D"].copy()
    yD[1:] += c
    common = dict(days=days, yD=yD, objective=orc.FIT_IRD, fit_I0=True)
    p = mkpb(orc, yI=tr["I"], yR=tr["R"], cost=orc.MSE, **common)
    rngD = yD.max() - yD.min()
    assert orc.loss(p, th) == pytest.approx((c / rngD) ** 2 * (n - 1) / n, rel=1e-9)
    # each compartment is scaled by its own series' range: R offset by c alone gives (c/range(yR))^2 (n-1)/n
    yR = tr["R"].copy()
    yR[1:] += c
    pR = mkpb(orc, days=days, yD=tr["D"], yI=tr["I"], yR=yR, cost=orc.MSE, objective=orc.FIT_IRD, fit_I0=True)
    assert orc.loss(pR, th) == pytest.approx((c / (yR.max() - yR.min())) ** 2 * (n - 1) / n, rel=1e-9)
    # the max picks the worst compartment: shift I by a larger relative amount
    yI = tr["I"] * 1.0
    yI[1:] += 0.5 * (yI.max() - yI.min())
    p2 = mkpb(orc, yI=yI, yR=tr["R"], cost=orc.MXSE, **common)
    rngI = yI.max() - yI.min()
    want = max((0.5 * (tr["I"].max() - tr["I"].min()) / rngI) ** 2, (c / rngD) ** 2)
    assert orc.loss(p2, th) == pytest.approx(want, rel=1e-9)
    # MAPE is not normalised: relative offsets of 20% on I (day 0 included, I0 != 0) and 10% on
    # R (day 0 skipped, R0 = 0); the max is I's 100 * 0.2 / 1.2, R's alone 100 * 0.1 / 1.1
    p3 = mkpb(orc, yI=tr["I"] * 1.2, yR=tr["R"] * 1.1, cost=orc.MAPE, **common)
    assert orc.loss(p3, th) == pytest.approx(100 * 0.2 / 1.2, rel=1e-9)
    p4 = mkpb(orc, yI=tr["I"], yR=tr["R"] * 1.1, cost=orc.MAPE, **common)
    assert orc.loss(p4, th) == pytest.approx(100 * (0.1 / 1.1) * (n - 1) / (n - 1), rel=1e-9)


# ------------------------------------------------------------------ adjoint

def _fd(orc, pb, th, j, h_rel=1e-6):
    th = np.array(th, float)
    h = h_rel * max(abs(th[j]), 1e-3)
    tp, tm = th.copy(), th.copy()
    tp[j] += h
    tm[j] -= h
    return (orc.loss(pb, tp) - orc.loss(pb, tm)) / (2 * h)


@pytest.mark.parametrize("form,cost", [("pwc", "mse"), ("pwc", "mae"), ("pwc", "mxse"), ("pwc", "mape"),
                                       ("ramp", "mse"), ("ramp_swapped", "mae")])
def test_adjoint_matches_central_fd(orc, form, cost):
    ser = synth.load_series("60d")
    y = ser["yD"][:41]
    if form == "pwc":
        pb = mkpb(orc, days=40, K=4, yD=y, cost=orc.COSTS[cost])
        th = [0.235, 0.18, 0.171, 0.12, 0.097, 0.0021, 9.1e3]
    else:
        pb = mkpb(orc, days=40, beta_form=orc.BETA_RAMP, yD=y, cost=orc.COSTS[cost])
        th = [0.24, 0.15, 11.37, 27.61, 0.1, 0.0019, 1.05e4]
        if form == "ramp_swapped":  # t1 > t2 in theta: the derivatives follow the swap
            th[2], th[3] = th[3], th[2]
    L, g, gu = orc.loss_grad(pb, th)
    assert L == pytest.approx(orc.loss(pb, th), rel=1e-14)
    fd = np.array([_fd(orc, pb, th, j) for j in range(len(th))])
    scale = np.abs(fd) + 1e-6 * np.max(np.abs(fd))
    assert np.all(np.abs(g - fd) <= 2e-5 * scale), (g, fd)


def _ird_problem(orc, form, cost, dominant, fit_I0):
    # reported series from the trajectory at the evaluation point with 0.2% noise, one compartment
    # moved 5-8% off it so that its normalised cost is the largest of the three (Sec. 3.1,
    # F_IRD^C = max over I, R, D); returns the problem, theta and the compartment costs
    ser = synth.load_series("60d")
    days, R0 = 35, 800.0
    if form == "pwc":
        ref = [0.23, 0.19, 0.17, 0.13, 0.1, 0.002, 1.1e4]
        kw = dict(K=4)
    else:
        ref = [0.25, 0.14, 9.5, 24.25, 0.1, 0.002, 1.1e4]
        kw = dict(beta_form=orc.BETA_RAMP)
    th = np.array(ref) * (1 + 0.03 * np.sin(np.arange(len(ref)) + 1.0))
    base = orc.Problem(yD=np.zeros(days + 1), N=ser["N"], R0=R0, spd=10, **kw)
    tr = orc.simulate(base, th, days)
    rng = np.random.default_rng(3)
    wob = lambda v, a: v * (1 + a * rng.normal(size=v.size))
    yI = wob(tr["I"], 2e-3)
    yR = R0 + wob(tr["R"] - R0, 2e-3)
    yD = tr["D"][0] + wob(tr["D"] - tr["D"][0], 2e-3)
    t = np.linspace(0.0, 1.0, days + 1)
    if dominant == "I":
        yI = yI * (1 + 0.08 * t)
    elif dominant == "R":
        yR = R0 + (yR - R0) * (1 + 0.08 * t)
    else:
        yD = yD + 0.08 * t * (yD - yD[0])
    pb = orc.Problem(yD=yD, yI=yI, yR=yR, N=ser["N"], R0=R0, I0=float(yI[0]), fit_I0=fit_I0, spd=10,
                     objective=orc.FIT_IRD, cost=orc.COSTS[cost], **kw)
    th = th if fit_I0 else th[:-1]
    tr = orc.simulate(pb, th, days)
    costs = []
    for y, yh in ((yI, tr["I"]), (yR, tr["R"]), (yD, tr["D"])):
        if pb.cost == orc.MAPE:
            m = y != 0
            costs.append(100 * np.mean(np.abs((y[m] - yh[m]) / y[m])))
        else:
            e = (y - yh) / (y.max() - y.min())
            costs.append({orc.MSE: np.mean(e * e), orc.MAE: np.mean(np.abs(e)), orc.MXSE: np.max(e * e)}[pb.cost])
    return pb, th, costs


@pytest.mark.parametrize("form,cost,dominant,fit_I0", [
    ("pwc", "mse", "I", True), ("pwc", "mse", "R", True), ("pwc", "mse", "D", True),
    ("pwc", "mae", "R", True), ("pwc", "mape", "D", True), ("pwc", "mxse", "I", True),
    ("ramp", "mxse", "I", False), ("ramp", "mxse", "R", False), ("ramp", "mxse", "D", False),
    ("ramp", "mse", "D", False), ("ramp", "mape", "I", False), ("ramp", "mae", "D", True)])
def test_adjoint_f_ird_matches_central_fd(orc, form, cost, dominant, fit_I0):
    pb, th, costs = _ird_problem(orc, form, cost, dominant, fit_I0)
    assert "IRD"[int(np.argmax(costs))] == dominant and max(costs) > 2 * sorted(costs)[1], costs
    L, g, gu = orc.loss_grad(pb, th)
    assert L == orc.loss(pb, th)
    fd = np.array([_fd(orc, pb, th, j) for j in range(len(th))])
    scale = np.abs(fd) + 1e-6 * np.max(np.abs(fd))
    assert np.all(np.abs(g - fd) <= 2e-5 * scale), (g, fd)


def test_adjoint_f_ird_initial_state_gradient(orc):
    # R0 enters the recovered series (R = R0 + ...) and S0 = N - I0 - R0 - D0
    pb, th, _ = _ird_problem(orc, "ramp", "mse", "R", False)

    def L_of(R0):
        return orc.loss(orc.Problem(**{**pb.__dict__, "R0": R0, "_keep": []}), th)

    h = 1e-1
    _, _, gu = orc.loss_grad(pb, th)
    fd = (L_of(pb.R0 + h) - L_of(pb.R0 - h)) / (2 * h)
    assert gu[2] - gu[0] == pytest.approx(fd, rel=1e-5)


def test_adjoint_initial_state_gradient(orc):
    ser = synth.load_series("60d")
    th = [0.21, 0.2, 0.15, 0.13, 0.1, 0.002, 1e4]
    y = ser["yD"][:31]

    def L_of(R0):
        return orc.loss(mkpb(orc, days=30, K=4, yD=y, R0=R0), th)

    R0, h = 2e3, 1e-2
    _, _, gu = orc.loss_grad(mkpb(orc, days=30, K=4, yD=y, R0=R0), th)
    fd = (L_of(R0 + h) - L_of(R0 - h)) / (2 * h)
    # changing R0 in the problem also moves S0 = N - I0 - R0 - D0
    assert gu[2] - gu[0] == pytest.approx(fd, rel=1e-5)


# ------------------------------------------------------------------ PSO

@pytest.mark.parametrize("P,M", [(2, 64), (7, 256), (13, 4096)])
def test_pso_sphere_paper_constants(orc, P, M):
    # the paper's w = c1 = c2 = 0.5 reach the minimum once the swarm is large enough for the dimension
    pso = orc.PSO(None, M, [-5.0] * P, [5.0] * P, seed=0, objective_kind=orc.OBJ_SPHERE).init()
    pso.step(300)
    assert pso.gbest_f < 1e-10
    assert np.max(np.abs(pso.gbest)) < 1e-5


# Clerc-Kennedy constriction constants, the textbook setting that converges on these functions
CK_W, CK_C = 0.7298, 1.49618


@pytest.mark.parametrize("P", [2, 7, 13])
def test_pso_sphere_constriction(orc, P):
    pso = orc.PSO(None, 64, [-5.0] * P, [5.0] * P, w=CK_W, c1=CK_C, c2=CK_C, seed=3,
                  objective_kind=orc.OBJ_SPHERE).init()
    pso.step(600)
    assert pso.gbest_f < 1e-20


@pytest.mark.parametrize("P", [2, 4])
def test_pso_rosenbrock(orc, P):
    best = []
    for seed in range(3):
        pso = orc.PSO(None, 256, [-2.0] * P, [2.0] * P, w=CK_W, c1=CK_C, c2=CK_C, seed=seed,
                      objective_kind=orc.OBJ_ROSENBROCK).init()
        pso.step(2000)
        best.append((pso.gbest_f, pso.gbest.copy()))
    f, x = min(best, key=lambda t: t[0])
    assert f < 1e-6 and np.allclose(x, np.ones(P), atol=2e-3)


def test_pso_invariants(orc):
    zlb, zub = np.array([-1.0, 0.0, 2.0]), np.array([1.0, 3.0, 2.5])
    pso = orc.PSO(None, 37, zlb, zub, seed=9, objective_kind=orc.OBJ_ROSENBROCK).init()
    prev_pf, prev_g = pso.pbest_f.copy(), pso.gbest_f
    for _ in range(30):
        pso.step()
        assert np.all(pso.x >= zlb) and np.all(pso.x <= zub)
        assert np.all(pso.pbest_f <= prev_pf) and pso.gbest_f <= prev_g
        assert pso.gbest_idx == int(np.argmin(pso.pbest_f))
        assert np.array_equal(pso.gbest, pso.pbest[pso.gbest_idx])
        for p in range(37):
            assert pso.objective(pso.pbest[p]) == pso.pbest_f[p]
        prev_pf, prev_g = pso.pbest_f.copy(), pso.gbest_f
    # reproducible; a different stream word gives a different swarm
    a = orc.PSO(None, 37, zlb, zub, seed=9, objective_kind=orc.OBJ_ROSENBROCK).init().step(30)
    assert np.array_equal(a.x, pso.x)
    b = orc.PSO(None, 37, zlb, zub, seed=9, stream=1, objective_kind=orc.OBJ_ROSENBROCK).init()
    assert not np.array_equal(b.x, orc.PSO(None, 37, zlb, zub, seed=9, objective_kind=orc.OBJ_ROSENBROCK).init().x)


def test_pso_update_rule_special_cases(orc):
    zlb, zub = np.full(3, -10.0), np.full(3, 10.0)
    mk = lambda **kw: orc.PSO(None, 16, zlb, zub, seed=5, objective_kind=orc.OBJ_SPHERE, **kw).init()
    # w = c1 = c2 = 0: velocity becomes 0, nothing moves
    a = mk(w=0.0, c1=0.0, c2=0.0)
    x0 = a.x.copy()
    a.step()
    assert np.array_equal(a.x, x0) and np.all(a.v == 0)
    # c1 = c2 = 0: pure inertia, x' = clamp(x + w v)
    b = mk(w=0.7, c1=0.0, c2=0.0)
    x0, v0 = b.x.copy(), b.v.copy()
    b.step()
    assert np.allclose(b.v, 0.7 * v0, rtol=1e-15) and np.allclose(b.x, np.clip(x0 + 0.7 * v0, -10, 10), rtol=1e-15)
    # w = 0, c2 = 0, c1 = 1: the move is r1 (pbest - x) with r1 in [0,1): x' lies between x and pbest
    c = mk(w=0.0, c1=1.0, c2=0.0)
    c.step()  # first step: pbest == x, so nothing moves
    assert np.all(c.v == 0)
    # velocity is kept when a position is clamped at a bound
    d = mk(w=1.0, c1=0.0, c2=0.0)
    d.v[...] = 25.0
    d.step()
    assert np.all(d.x == 10.0) and np.all(d.v == 25.0)
    # social term only: with w = 0, c1 = 0 every particle moves toward gbest, never past it
    e = mk(w=0.0, c1=0.0, c2=1.0)
    x0, g0 = e.x.copy(), e.gbest.copy()
    e.step()
    t = (e.x - x0) / np.where(g0 - x0 == 0, 1, g0 - x0)
    assert np.all((t >= 0) & (t < 1))


def test_swarm_part_numbered_from_an_offset_is_that_part_of_the_swarm(orc):
    # particles are numbered globally in the random-number counter: a swarm of 7 starting at
    # particle 5 draws what particles 5..11 of a swarm of 16 draw
    full = orc.PSO(None, 16, [-1.0] * 5, [2.0] * 5, seed=21, stream=3, objective_kind=orc.OBJ_SPHERE).init()
    part = orc.PSO(None, 7, [-1.0] * 5, [2.0] * 5, seed=21, stream=3, objective_kind=orc.OBJ_SPHERE,
                   p_offset=5).init()
    assert np.array_equal(part.x, full.x[5:12]) and np.array_equal(part.v, full.v[5:12])
    assert np.array_equal(part.pbest_f, full.pbest_f[5:12])
    # with the whole swarm's global best set between steps, the part keeps following it
    for _ in range(3):
        part.set_state(part.x, part.v, part.pbest, part.pbest_f, 0, part.iter)
        part.gbest[:] = full.gbest
        full.step()
        part.step()
        assert np.array_equal(part.x, full.x[5:12]) and np.array_equal(part.pbest, full.pbest[5:12])


def test_argmin_nan_and_ties(orc):
    assert orc.argmin([3.0, np.nan, 1.0, 1.0]) == 2
    assert orc.argmin([np.nan, np.nan]) == 0
    assert orc.argmin([np.inf, 5.0, np.nan, 5.0]) == 1
    assert orc.argmin([np.nan, 5.0, 3.0]) == 2  # a NaN in front ranks last too


def test_nan_loss_counts_as_infinite(orc):
    # a parameter vector whose loss is NaN ranks last: the swarm's objective returns +inf for it
    pb = mkpb(orc, days=30, yD=np.arange(31.0))
    pso = orc.PSO(pb, 4, [0.0] * 4, [1.0] * 4)
    assert math.isnan(orc.loss(pb, [np.nan, 0.1, 0.002, 1e4]))
    assert pso.objective([np.nan, 0.1, 0.002, 1e4]) == np.inf
    assert pso.objective([0.2, 0.1, 0.002, 1e4]) == orc.loss(pb, [0.2, 0.1, 0.002, 1e4])


def test_store_f32_rounds_state(orc):
    pso = orc.PSO(None, 8, [-1.0] * 3, [1.0] * 3, seed=2, store_f32=True, objective_kind=orc.OBJ_SPHERE).init()
    pso.step(3)
    for arr in (pso.x, pso.v, pso.pbest, pso.pbest_f):
        assert np.array_equal(arr, arr.astype(np.float32).astype(np.float64))


def test_reeval_topk_is_best_of_k(orc):
    ser = synth.load_series("30d")
    pb = mkpb(orc, days=30, yD=ser["yD"])
    lb, ub = [1e-3, 1e-3, 1e-5, 1.0], [2.0, 1.0, 0.1, 1e6]
    pso = orc.PSO(pb, 48, np.log(lb), np.log(ub), logdim=[1, 1, 1, 1], seed=4, store_f32=True).init().step(5)
    idx, f = pso.reeval_topk(8)
    order = sorted(range(48), key=lambda p: (pso.pbest_f[p], p))[:8]
    exact = [orc.loss(pb, np.exp(pso.pbest[p])) for p in order]
    assert idx == order[int(np.argmin(exact))] and f == min(exact)
    # stored values that rank the candidates opposite to their true losses: the re-evaluation
    # looks at exactly the k best by stored value and returns the truly best of those
    true = np.array([orc.loss(pb, np.exp(z)) for z in pso.pbest])
    rank = np.argsort(-true, kind="stable")  # worst first
    fake = np.empty(48)
    fake[rank] = np.arange(48, dtype=float)
    pso.set_state(pso.x, pso.v, pso.pbest, fake, int(rank[0]), pso.iter)
    for k in (1, 5, 48, 60):
        idx, f = pso.reeval_topk(k)
        j = int(rank[min(k, 48) - 1])
        assert idx == j and f == true[j], k


# ------------------------------------------------------------------ calibration

def test_noise_free_recovery(orc):
    th_true = np.array([0.25, 0.1, 0.002, 1e4])
    pb = mkpb(orc, days=30)
    pb.yD = orc.simulate(pb, th_true)["D"]
    lb, ub = [0.0, 0.0, 0.0, 0.0], [2.0, 1.0, 0.1, 1e6]
    best = None
    for seed in range(2):
        pso = orc.PSO(pb, 128, lb, ub, seed=seed).init().step(300)
        if best is None or pso.gbest_f < best.gbest_f:
            best = pso
    # D alone pins the growth rate and mu*I0 but leaves a flat valley along the rest of
    # theta, so the swarm reaches a near-zero misfit without recovering theta itself
    scale = np.var(pb.yD)
    assert best.gbest_f < 1e-5 * scale
    b, g, m, I0 = best.gbest
    # identifiable combinations from D alone: the early growth rate and mu * I0
    assert (b - g - m) == pytest.approx(0.25 - 0.102, rel=2e-2)
    assert m * I0 == pytest.approx(20.0, rel=5e-2)


def test_brute_force_grid_contains_pso_optimum(orc):
    ser = synth.load_series("30d")
    pb = mkpb(orc, days=30, yD=ser["yD"], fit_I0=False, I0=1e4)
    # two free parameters (beta, mu); gamma pinned by equal bounds
    lb, ub = [0.1, 0.1, 0.0005], [0.4, 0.1, 0.005]
    bs = np.linspace(lb[0], ub[0], 61)
    ms = np.linspace(lb[2], ub[2], 61)
    grid = np.array([[orc.loss(pb, [b, 0.1, m]) for m in ms] for b in bs])
    i, j = np.unravel_index(np.argmin(grid), grid.shape)
    pso = orc.PSO(pb, 64, lb, ub, seed=1).init().step(150)
    assert pso.gbest_f <= grid.min()
    assert abs(pso.gbest[0] - bs[i]) <= 1.5 * (bs[1] - bs[0])
    assert abs(pso.gbest[2] - ms[j]) <= 1.5 * (ms[1] - ms[0])


def test_forecast(orc):
    days, H = 30, 14
    th = [0.22, 0.18, 0.1, 0.003, 1e4]
    pb = mkpb(orc, days=days, K=2)
    fc = orc.forecast(pb, th, H)
    full = orc.simulate(pb, th, days + H)["D"]
    assert np.array_equal(fc, full[days + 1:])
    # past the window the last segment's rate is used: beta = 0 there gives the closed form
    th0 = [0.3, 0.0, 0.1, 0.003, 1e4]
    st = orc.simulate(pb, th0, days)
    fc0 = orc.forecast(pb, th0, H)
    k = np.arange(1, H + 1) * pb.spd
    I_end = st["I"][-1]
    # the window's second segment already has beta = 0, so the decay law holds from its start too
    Ik = I_end * (1 - (0.1 + 0.003) / pb.spd) ** k
    assert np.allclose(fc0, st["D"][-1] + 0.003 / 0.103 * (I_end - Ik), rtol=1e-12)


# ---------------------------------------------------------------- ensemble bands (Sec. 4.2)

def test_ensemble_bands_of_identical_members_collapse_to_the_trajectory(orc):
    s = synth.load_series("60d")
    pb = orc.Problem(yD=s["yD"], N=s["N"], K=4, spd=10)
    th = np.asarray(s["theta_true"])
    b = orc.ensemble_bands(pb, np.tile(th, (6, 1)), 14)
    tr = orc.simulate(pb, th, pb.days + 14)
    for q in "SIRD":
        assert np.all(b[q] == tr[q][:, None])


def test_ensemble_bands_order_statistics_and_nesting(orc):
    # members differing only in mu: deaths increase with mu on every day after the first, so the
    # sorted members are the mu-sorted ones and the median is the middle member's trajectory
    s = synth.load_series("60d")
    pb = orc.Problem(yD=s["yD"], N=s["N"], K=4, spd=10)
    th = np.tile(np.asarray(s["theta_true"]), (9, 1))
    th[:, 5] = np.linspace(1e-3, 3e-3, 9)
    b = orc.ensemble_bands(pb, th[::-1], 10, fractions=(0.95, 0.5))
    D = np.stack([orc.simulate(pb, t, pb.days + 10)["D"] for t in th], axis=1)
    assert np.array_equal(b["D"][1:, 0], D[1:, 4])
    # drop = floor(9 * 0.05 / 2) = 0 and floor(9 * 0.5 / 2) = 2
    assert np.array_equal(b["D"][1:, 1], D[1:, 0]) and np.array_equal(b["D"][1:, 2], D[1:, 8])
    assert np.array_equal(b["D"][1:, 3], D[1:, 2]) and np.array_equal(b["D"][1:, 4], D[1:, 6])
    for q in b:
        assert np.all(b[q][:, 1] <= b[q][:, 3]) and np.all(b[q][:, 3] <= b[q][:, 0])
        assert np.all(b[q][:, 0] <= b[q][:, 4]) and np.all(b[q][:, 4] <= b[q][:, 2])


def test_ensemble_bands_reproduction_number_closed_form(orc):
    # constant beta: R0(t) = beta / (gamma + mu) on every day, inside the window and past it
    s = synth.load_series("30d")
    pb = orc.Problem(yD=s["yD"], N=s["N"], K=1, spd=10)
    th = np.array([[0.3, 0.1, 0.002, 1e4], [0.2, 0.12, 0.004, 2e4]])
    b = orc.ensemble_bands(pb, th, 21, fractions=())
    r = np.sort(th[:, 0] / (th[:, 1] + th[:, 2]))
    assert np.all(b["R0"][:, 0] == (r[0] + r[1]) * 0.5)
    assert b["R0"].shape == (31 + 21, 1)


def test_ensemble_bands_beta_is_the_ramp_at_each_day(orc):
    # one member of the ramp form: the beta band on day d is eq. (beta) at t = d, written out
    s = synth.load_series("30d")
    pb = orc.Problem(yD=s["yD"], N=s["N"], beta_form=orc.BETA_RAMP, spd=10)
    b1, b2, t1, t2 = 0.31, 0.12, 7.5, 19.25
    b = orc.ensemble_bands(pb, [b1, b2, t2, t1, 0.1, 0.002, 1e4], 5, fractions=())
    t = np.arange(31 + 5, dtype=float)
    want = np.where(t < t1, b1, np.where(t < t2, b1 + (b2 - b1) * (t - t1) / (t2 - t1), b2))
    assert np.allclose(b["beta"][:, 0], want, rtol=1e-14, atol=0)


# ---------------------------------------------------------------- parameter bands (Sec. 4.2)

def test_parameter_bands_of_shuffled_ranks(orc):
    # each parameter's k = 1000 values are c_d + 1 .. c_d + 1000 in a random order: the median is
    # c_d + 500.5 and the band holding f leaves floor(1000 (1 - f) / 2) = 25, 50, 250 values out
    s = synth.load_series("30d")
    pb = orc.Problem(yD=s["yD"], N=s["N"], K=2, spd=10)
    rng = np.random.default_rng(8)
    c = np.array([0.0, 10.0, -3.0, 1e4, 0.5])
    th = np.stack([c[d] + rng.permutation(np.arange(1, 1001, dtype=float)) for d in range(5)], axis=1)
    b = orc.parameter_bands(pb, th, fractions=(0.95, 0.9, 0.5))
    assert b.shape == (5, 7)
    want = np.array([500.5, 26, 975, 51, 950, 251, 750])
    for d in range(5):
        assert np.array_equal(b[d], c[d] + want), d


def test_parameter_bands_odd_count_and_whole_band(orc):
    # k = 7: the median is the 4th smallest; f = 1 keeps every value (the band is min .. max);
    # f = 0.5 leaves floor(7 * 0.25) = 1 out at each end
    s = synth.load_series("30d")
    pb = orc.Problem(yD=s["yD"], N=s["N"], K=1, spd=10, fit_I0=False)
    v = np.array([0.9, 0.1, 0.5, 0.7, 0.3, 1.3, 1.1])
    th = np.stack([v, 2 * v, -v], axis=1)
    b = orc.parameter_bands(pb, th, fractions=(1.0, 0.5))
    assert np.array_equal(b[0], [0.7, 0.1, 1.3, 0.3, 1.1])
    assert np.array_equal(b[1], 2 * b[0])
    assert np.array_equal(b[2], [-0.7, -1.3, -0.1, -1.1, -0.3])


def test_parameter_bands_count_definition_on_random_values(orc):
    # brute force: with distinct values, band b's low end has exactly drop_b values below it and
    # its high end exactly drop_b above; the even-count median lies between two order statistics
    s = synth.load_series("30d")
    pb = orc.Problem(yD=s["yD"], N=s["N"], K=1, spd=10)
    rng = np.random.default_rng(9)
    for k in (1, 2, 3, 40, 999):
        th = rng.normal(size=(k, 4))
        fr = (0.95, 0.9, 0.5)
        b = orc.parameter_bands(pb, th, fractions=fr)
        for d in range(4):
            x = th[:, d]
            for i, f in enumerate(fr):
                drop = int(np.floor(k * (1 - f) / 2 + 1e-9))
                assert np.sum(x < b[d, 1 + 2 * i]) == drop and np.sum(x > b[d, 2 + 2 * i]) == drop
            assert np.sum(x < b[d, 0]) == k // 2  # the middle value, or strictly between the two
            if k % 2:
                assert b[d, 0] in x


def test_parameter_bands_ramp_change_times_in_model_order(orc):
    # the ramp's change times are an unordered pair: t1 summarises min(t_a, t_b), t2 the max
    s = synth.load_series("30d")
    pb = orc.Problem(yD=s["yD"], N=s["N"], beta_form=orc.BETA_RAMP, spd=10)
    k = 5
    ta = np.array([3.0, 20.0, 4.0, 18.0, 5.0])
    tb = np.array([15.0, 2.0, 16.0, 1.0, 17.0])
    th = np.column_stack([np.full(k, 0.3), np.full(k, 0.1), ta, tb, np.full(k, 0.1), np.full(k, 2e-3),
                          np.full(k, 1e4)])
    b = orc.parameter_bands(pb, th, fractions=(1.0,))
    assert np.array_equal(b[2], [3.0, 1.0, 5.0])  # sorted minima 1, 2, 3, 4, 5
    assert np.array_equal(b[3], [17.0, 15.0, 20.0])  # sorted maxima 15, 16, 17, 18, 20
    assert np.array_equal(b[0], [0.3, 0.3, 0.3])
