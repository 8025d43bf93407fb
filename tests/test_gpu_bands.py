"""Ensemble bands of repeated calibrations (Sec. 4.2) on the GPU vs the oracle (GPU only)."""
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


def near(th, M, seed, spread=0.08):
    return th * np.exp(np.random.default_rng(seed).normal(0.0, spread, (M, th.size)))


@pytest.mark.parametrize("k", [1, 2, 7, 1000, 4096])
def test_bands_bit_exact_pwc(k):
    s = synth.load_series("60d")
    th = near(np.asarray(s["theta_true"]), k, k)
    got = sird.ensemble_bands(s["yD"], s["N"], th, 21, K=4, spd=10)
    want = O.ensemble_bands(O.Problem(yD=s["yD"], N=s["N"], K=4, spd=10), th, 21)
    for q in sird.BAND_QUANTITIES:
        assert np.array_equal(got[q], want[q]), q


def test_bands_bit_exact_ramp_with_fixed_I0_and_R0():
    s = synth.load_series("60d")
    y = s["yD"][:36]
    rng = np.random.default_rng(3)
    M = 300
    th = np.column_stack([rng.uniform(0.15, 0.35, M), rng.uniform(0.1, 0.3, M), rng.uniform(0, 30, M),
                          rng.uniform(0, 30, M), rng.uniform(0.08, 0.12, M), rng.uniform(1e-3, 3e-3, M)])
    kw = dict(beta_form=sird.BETA_RAMP, fit_I0=False, I0=1.2e4, R0=500.0, spd=10)
    got = sird.ensemble_bands(y, s["N"], th, 21, fractions=(0.95, 0.9, 0.5, 1.0), **kw)
    pb = O.Problem(yD=y, N=s["N"], beta_form=O.BETA_RAMP, fit_I0=False, I0=1.2e4, R0=500.0, spd=10)
    want = O.ensemble_bands(pb, th, 21, fractions=(0.95, 0.9, 0.5, 1.0))
    for q in sird.BAND_QUANTITIES:
        assert np.array_equal(got[q], want[q]), q


def test_repeated_calibrations_of_one_window_as_one_batch():
    # the stability test of Sec. 4.2: one window calibrated many times (distinct Philox streams)
    # in one batched launch, then the ensemble's bands with a 21-day extension
    s = synth.load_series("450d")
    T, L, reps = 120, 35, 64
    lay = {"L": np.full(reps, L), "M": np.full(reps, 512), "T": np.full(reps, T)}
    wins = synth.rolling_window_problems(s, lay)
    lb, ub = configs.bounds_ramp()
    res = sird.Batch(wins, beta_form=sird.BETA_RAMP, K=1, spd=10, iters=20, lb=lb, ub=ub, seed=1).calibrate()
    th = np.array([r["theta"] for r in res])
    assert len({tuple(t) for t in th}) > 1  # independent repetitions differ
    w = wins[0]
    got = sird.ensemble_bands(w["yD"], w["N"], th, 21, beta_form=sird.BETA_RAMP, R0=w["R0"], spd=10)
    pb = O.Problem(yD=w["yD"], N=w["N"], R0=w["R0"], beta_form=O.BETA_RAMP, spd=10)
    want = O.ensemble_bands(pb, th, 21)
    for q in sird.BAND_QUANTITIES:
        assert np.array_equal(got[q], want[q]), q
    assert got["D"].shape == (L + 1 + 21, 7)
