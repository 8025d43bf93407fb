"""Writes the stored synthetic series ``series_<name>.json`` (into this folder, or the folder
given as the first argument).

The noise-free curves are integrated by the FP64 oracle (explicit Euler on
eq. (SIRD), Sec. 2.2 / 3.1) at ground-truth rates; deaths are then observed
with Poisson count noise drawn by ``synth.poisson_cumulative`` (numpy
``default_rng(seed)``).  Nothing here touches the CUDA path.

Ground truths (N = 38e6, gamma = 0.1, mu = 0.002, R0 = D0 = 0):
  30d   beta = 0.25 constant, I0 = 1e4, 30 days, dt = 0.1
  60d   beta = (0.22, 0.19, 0.16, 0.13) on 4 equal segments, I0 = 1e4, 60 days, dt = 0.1
  90d   beta as 60d on 4 segments over 90 days, dt = 0.05
  134d  10 segments from 0.22 down to 0.11 and back to 0.13, I0 = 1e4, 120 days
      plus 14 held-out days with the last segment's rate, dt = 0.05
  450d  one 450-day series, dt = 0.1, beta piecewise linear through the knots below,
      I0 = 2e4 at day 0; windows are cut from it at run time
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2204_12346_gb300 import synth  # noqa: E402

N = synth.N_POLAND
GAMMA, MU = 0.1, 0.002
KNOTS_450D = [0, 45, 90, 150, 200, 260, 330, 390, 450]
BETA_450D = [0.20, 0.13, 0.11, 0.16, 0.12, 0.21, 0.15, 0.25, 0.17]


def window_series(name, K, beta, days, spd, I0, extra_days=0, seed=0):
    theta = np.array(list(beta) + [GAMMA, MU, I0])
    pb = O.Problem(yD=np.zeros(days + 1), N=N, R0=0.0, fit_I0=True, K=K, spd=spd)
    tr = O.simulate(pb, theta, days + extra_days)
    y = synth.poisson_cumulative(tr["D"], np.random.default_rng(seed))
    return {
        "name": name, "N": N, "K": K, "days": days, "spd": spd, "R0": 0.0, "I0_true": I0,
        "theta_true": theta.tolist(), "held_out_days": extra_days,
        "yD": y.tolist(), "D_true": tr["D"].tolist(), "I_true": tr["I"].tolist(), "R_true": tr["R"].tolist(),
    }


def long_series(seed=0):
    days, spd = 450, 10
    t = np.arange(days * spd) / spd
    beta = np.interp(t, KNOTS_450D, BETA_450D)
    tr = O.simulate_schedule(N, (N - 2e4, 2e4, 0.0, 0.0), beta, GAMMA, MU, spd, days)
    y = synth.poisson_cumulative(tr["D"], np.random.default_rng(seed))
    return {
        "name": "450d", "N": N, "days": days, "spd": spd, "beta_knots": KNOTS_450D, "beta_values": BETA_450D,
        "gamma": GAMMA, "mu": MU, "yD": y.tolist(), "D_true": tr["D"].tolist(),
        "I_true": tr["I"].tolist(), "R_true": tr["R"].tolist(),
    }


def main(out_dir=None):
    """Writes every series into out_dir (default: this folder, where the stored copies live)."""
    out = {
        "30d": window_series("30d", 1, [0.25], 30, 10, 1e4),
        "60d": window_series("60d", 4, [0.22, 0.19, 0.16, 0.13], 60, 10, 1e4),
        "90d": window_series("90d", 4, [0.22, 0.19, 0.16, 0.13], 90, 20, 1e4),
        "134d": window_series("134d", 10, [0.22, 0.20, 0.18, 0.16, 0.14, 0.12, 0.11, 0.11, 0.12, 0.13],
                            120, 20, 1e4, extra_days=14),
        "450d": long_series(),
    }
    here = out_dir or os.path.dirname(os.path.abspath(__file__))
    for name, d in out.items():
        with open(os.path.join(here, f"series_{name}.json"), "w") as f:
            json.dump(d, f, indent=None, separators=(",", ":"))
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else None)
