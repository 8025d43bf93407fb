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
    # the stability of the parameters themselves (beta1, beta2, t1, t2, gamma, mu, I0)
    pg = sird.parameter_bands(w["yD"], w["N"], th, beta_form=sird.BETA_RAMP, R0=w["R0"], spd=10)
    assert np.array_equal(pg, O.parameter_bands(pb, th))
    assert pg.shape == (7, 7) and np.all(pg[2, 0] <= pg[3, 0])


@pytest.mark.parametrize("k", [1, 2, 7, 1000, 4095, 4096])
def test_parameter_bands_bit_exact_pwc(k):
    s = synth.load_series("60d")
    th = near(np.asarray(s["theta_true"]), k, 100 + k)
    got = sird.parameter_bands(s["yD"], s["N"], th, fractions=(0.95, 0.9, 0.5, 1.0), K=4, spd=10)
    want = O.parameter_bands(O.Problem(yD=s["yD"], N=s["N"], K=4, spd=10), th, fractions=(0.95, 0.9, 0.5, 1.0))
    assert got.shape == (7, 9)
    assert np.array_equal(got, want)


def test_parameter_bands_bit_exact_ramp_with_ties_and_swapped_times():
    # ties (a parameter held at one value by many members) and change times given in either order
    s = synth.load_series("60d")
    y = s["yD"][:36]
    rng = np.random.default_rng(12)
    M = 1001
    ta, tb = rng.uniform(0, 30, M), rng.uniform(0, 30, M)
    th = np.column_stack([rng.choice([0.2, 0.25, 0.3], M), rng.uniform(0.1, 0.3, M), ta, tb,
                          np.full(M, 0.1), rng.uniform(1e-3, 3e-3, M)])
    kw = dict(beta_form=sird.BETA_RAMP, fit_I0=False, I0=1.2e4, R0=500.0, spd=10)
    got = sird.parameter_bands(y, s["N"], th, fractions=(0.95, 0.5), **kw)
    pb = O.Problem(yD=y, N=s["N"], beta_form=O.BETA_RAMP, fit_I0=False, I0=1.2e4, R0=500.0, spd=10)
    assert np.array_equal(got, O.parameter_bands(pb, th, fractions=(0.95, 0.5)))
    assert np.all(got[4] == 0.1)


def test_parameter_bands_refusals():
    s = synth.load_series("60d")
    th = np.tile(np.asarray(s["theta_true"]), (3, 1))
    with pytest.raises(sird.SirdError):
        sird.parameter_bands(s["yD"], s["N"], th, fractions=(1.5,), K=4, spd=10)
    bad = th.copy()
    bad[1, 2] = np.nan
    with pytest.raises(sird.SirdError):
        sird.parameter_bands(s["yD"], s["N"], bad, K=4, spd=10)
    with pytest.raises(sird.SirdError):
        sird.parameter_bands(s["yD"], s["N"], np.tile(th[:1], (4097, 1)), K=4, spd=10)
