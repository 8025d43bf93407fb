"""Forecast (Sec. 4.2 extension) and top-k export vs the oracle (GPU only)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2204_12346_gb300 import configs, sird, synth
from util import box_thetas, f32, log_box, rel_err, window

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    torch.cuda.set_device(0)
    O.build()


@pytest.mark.parametrize("precision", [64, 32])
def test_forecast_pwc_matches_oracle(precision):
    # the largest configuration's window: 120 days, 10 segments, dt = 0.05, 14 days ahead
    y, N, _, _ = window("134d", 120)
    th = box_thetas(10, 257, 77)
    th[:, :10] = np.clip(th[:, :10], 0.05, 0.6)  # keep trajectories from running out of susceptibles
    got = sird.forecast(y, N, th, 14, K=10, spd=20, precision=precision)
    pb = O.Problem(yD=y, N=N, K=10, spd=20)
    want = np.array([O.forecast(pb, t, 14) for t in th])
    if precision == 64:
        assert np.array_equal(got, want)
    else:
        assert rel_err(got, want).max() <= 1e-5


@pytest.mark.parametrize("precision", [64, 32])
def test_forecast_ramp_and_fixed_I0(precision):
    y, N, _, _ = window("60d", 35)
    rng = np.random.default_rng(4)
    M = 100
    th = f32(np.column_stack([rng.uniform(0.05, 0.5, M), rng.uniform(0.05, 0.5, M), rng.uniform(0, 35, M),
                              rng.uniform(0, 35, M), rng.uniform(0.02, 0.3, M), rng.uniform(1e-4, 0.01, M)]))
    got = sird.forecast(y, N, th, 21, beta_form=sird.BETA_RAMP, fit_I0=False, I0=8e3, R0=100.0, precision=precision)
    pb = O.Problem(yD=y, N=N, beta_form=O.BETA_RAMP, fit_I0=False, I0=8e3, R0=100.0)
    want = np.array([O.forecast(pb, t, 21) for t in th])
    if precision == 64:
        assert np.array_equal(got, want)
    else:
        assert rel_err(got, want).max() <= 1e-5


def test_topk_export_orders_personal_bests():
    y, N, _, _ = window("60d")
    lb, ub = log_box(4)
    zlb, zub = f32(np.log(lb)), f32(np.log(ub))
    M = 3000
    pso = O.PSO(O.Problem(yD=y, N=N, K=4, spd=10), M, zlb, zub, logdim=[1] * 7, seed=8, store_f32=True).init().step(2)
    cal = sird.Calibrator(y, N, K=4, spd=10, particles=M, iters=1, lb=lb, ub=ub, log_scale=[1] * 7, precision=32)
    cal.set_state(pso.x.T, pso.v.T, pso.pbest.T, pso.pbest_f, pso.gbest_idx, pso.iter)
    for k in (1, 64, 1024):
        th, lo = cal.topk(k)
        order = sorted(range(M), key=lambda p: (pso.pbest_f[p], p))[:k]
        assert np.array_equal(lo, pso.pbest_f[order])
        np.testing.assert_allclose(th, np.exp(pso.pbest[order]), rtol=1e-15)
