"""The seeded synthetic inputs (CPU only): the stored series are what their committed generator
writes from the oracle, and every generator follows the recipe it states (seeded, inside its
box or series, the stated distributions and layouts)."""
import filecmp
import importlib.util
import os

import numpy as np
import pytest

from paper_2204_12346_gb300 import configs, synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NAMES = ("30d", "60d", "90d", "134d", "450d")


def test_stored_series_are_what_the_generator_writes(tmp_path, orc):
    spec = importlib.util.spec_from_file_location("make_series", os.path.join(GOLDEN, "make_series.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.main(str(tmp_path))
    for name in NAMES:
        f = f"series_{name}.json"
        assert filecmp.cmp(os.path.join(GOLDEN, f), os.path.join(tmp_path, f), shallow=False), f


@pytest.mark.parametrize("name,days,spd,K", [("30d", 30, 10, 1), ("60d", 60, 10, 4), ("90d", 90, 20, 4),
                                             ("134d", 120, 20, 10)])
def test_window_series_follow_their_ground_truth(orc, name, days, spd, K):
    s = synth.load_series(name)
    n = days + 1 + int(s["held_out_days"])
    assert s["N"] == 38e6 and s["days"] == days and s["spd"] == spd and s["K"] == K
    assert all(len(s[k]) == n for k in ("yD", "D_true", "I_true", "R_true"))
    th = np.asarray(s["theta_true"])
    assert th[K] == 0.1 and th[K + 1] == 0.002 and th[K + 2] == 1e4
    pb = orc.Problem(yD=np.zeros(days + 1), N=s["N"], K=K, spd=spd)
    tr = orc.simulate(pb, th, n - 1)
    assert np.array_equal(tr["D"], s["D_true"]) and np.array_equal(tr["I"], s["I_true"])
    # observed deaths: cumulative counts, non-decreasing, starting at the true D0 = 0, close to the curve
    y = s["yD"]
    assert y[0] == 0.0 and np.all(np.diff(y) >= 0) and np.all(y == np.round(y))
    assert abs(y[-1] - s["D_true"][-1]) <= 5 * np.sqrt(s["D_true"][-1]) + 1


def test_long_series_and_its_reported_I_and_R(orc):
    s = synth.load_series("450d")
    assert len(s["yD"]) == 451 and s["gamma"] == 0.1 and s["mu"] == 0.002
    # the identity gamma (D - D0) = mu (R - R0) of the Euler scheme holds for the stored curves
    assert np.allclose(0.1 * s["D_true"], 0.002 * s["R_true"], rtol=1e-12, atol=1e-6)
    r = synth.reported_IR(s, seed=1)
    assert np.array_equal(r["yI"], synth.reported_IR(s, seed=1)["yI"])  # seeded
    assert not np.array_equal(r["yI"], synth.reported_IR(s, seed=2)["yI"])
    assert np.all(np.diff(r["yR"]) >= 0) and r["yR"][0] == np.round(s["R_true"][0])
    # Poisson around the curve: standardised residuals of I have mean ~0 and variance ~1
    z = (r["yI"] - s["I_true"]) / np.sqrt(s["I_true"])
    assert abs(z.mean()) < 0.2 and 0.7 < z.var() < 1.3


def test_poisson_cumulative():
    rng = np.random.default_rng(3)
    D = np.concatenate([[12.4], 12.4 + np.cumsum(np.full(4000, 50.0))])
    y = synth.poisson_cumulative(D, rng)
    assert y[0] == 12.0 and np.all(np.diff(y) >= 0)
    inc = np.diff(y)
    assert abs(inc.mean() - 50.0) < 0.5 and abs(inc.var() - 50.0) < 5.0
    # a decreasing true curve adds nothing (increments clipped at zero)
    assert np.all(synth.poisson_cumulative(D[::-1], np.random.default_rng(0))[1:] == np.round(D[-1]))


def test_box_sample_is_uniform_in_the_search_coordinates():
    lb, ub = configs.bounds(4, log=True)
    mask = [1, 0, 1, 1, 0, 1, 1]
    th = synth.box_sample(lb, ub, mask, 20000, np.random.default_rng(4))
    assert th.shape == (20000, 7) and np.all(th >= lb) and np.all(th <= ub)
    for d in range(7):
        z = np.log(th[:, d]) if mask[d] else th[:, d]
        lo, hi = (np.log(lb[d]), np.log(ub[d])) if mask[d] else (lb[d], ub[d])
        u = (z - lo) / (hi - lo)
        assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.005, d
    assert np.array_equal(th, synth.box_sample(lb, ub, mask, 20000, np.random.default_rng(4)))


def test_rolling_window_layout():
    lay = synth.rolling_windows(W=512, seed=0)
    L, M, T = lay["L"], lay["M"], lay["T"]
    assert len(L) == len(M) == len(T) == 512
    assert L.min() >= 21 and L.max() <= 90 and M.min() >= 256 and M.max() <= 2048 and np.all(M % 32 == 0)
    assert np.all(T >= 0) and np.all(T + L <= 450)  # every window inside the 451 observations
    assert np.array_equal(T, (3 * np.arange(512)) % (450 - L))  # shifted by delta = 3 days, wrapped
    again = synth.rolling_windows(W=512, seed=0)
    assert all(np.array_equal(lay[k], again[k]) for k in lay)


def test_rolling_window_problems_cut_the_series():
    s = synth.reported_IR(synth.load_series("450d"), seed=0)
    lay = synth.rolling_windows(W=40, seed=5)
    wins = synth.rolling_window_problems(s, lay)
    for w, win in enumerate(wins):
        T, L = int(lay["T"][w]), int(lay["L"][w])
        assert np.array_equal(win["yD"], s["yD"][T:T + L + 1]) and win["particles"] == lay["M"][w]
        # with reported I and R the window starts from them
        assert win["I0"] == s["yI"][T] and win["R0"] == s["yR"][T]
        assert np.array_equal(win["yI"], s["yI"][T:T + L + 1]) and np.array_equal(win["yR"], s["yR"][T:T + L + 1])
    plain = synth.rolling_window_problems(synth.load_series("450d"), lay)
    assert all("I0" not in w and w["R0"] == np.round(s["R_true"][int(lay["T"][i])]) for i, w in enumerate(plain))
