"""Seeded synthetic inputs shared by the CUDA path, its tests and the benchmark.

This module holds no arithmetic of the calibration method: it draws count noise,
random parameter vectors and window layouts, and loads the stored synthetic
series.  The noise-free epidemic curves in those series were integrated at
ground-truth rates by ``tests/golden/make_series.py`` (see that script); here
they are only read.

The paper's own data (OxCOVID19, Poland, Sec. 2.1) is not available, so every
input is synthetic at the paper's scale: N = 38e6, daily windows, deaths in the
1e3..1e5 range.
"""
from __future__ import annotations

import json
import os

import numpy as np

N_POLAND = 38.0e6

_GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")


def poisson_cumulative(D_true: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """Observed cumulative counts: D_true[0] plus the cumulative sum of Poisson(daily increment)."""
    inc = np.clip(np.diff(np.asarray(D_true, dtype=np.float64)), 0.0, None)
    noisy = rng.poisson(inc).astype(np.float64)
    return np.concatenate([[np.round(D_true[0])], np.round(D_true[0]) + np.cumsum(noisy)])


def box_sample(lb, ub, log_mask, M: int, rng: np.random.Generator) -> np.ndarray:
    """M parameter vectors uniform in the box (log-uniform on the dims where log_mask is set)."""
    lb = np.asarray(lb, dtype=np.float64)
    ub = np.asarray(ub, dtype=np.float64)
    log_mask = np.asarray(log_mask, dtype=bool)
    zl = np.where(log_mask, np.log(np.where(log_mask, lb, 1.0)), lb)
    zu = np.where(log_mask, np.log(np.where(log_mask, ub, 1.0)), ub)
    z = zl + (zu - zl) * rng.random((M, lb.size))
    return np.where(log_mask, np.exp(np.where(log_mask, z, 0.0)), z)


def reported_IR(series: dict, seed: int = 0) -> dict:
    """Reported infectious and recovered series for the F_IRD objective: I as Poisson counts
    around the series' I, R as R[0] plus cumulative Poisson daily increments (as for D).
    Returns a copy of the series with keys yI and yR added."""
    rng = np.random.default_rng(seed)
    out = dict(series)
    out["yI"] = rng.poisson(np.clip(np.asarray(series["I_true"], dtype=np.float64), 0.0, None)).astype(np.float64)
    out["yR"] = poisson_cumulative(np.asarray(series["R_true"], dtype=np.float64), rng)
    return out


def rolling_windows(W: int = 512, series_days: int = 450, L_min: int = 21, L_max: int = 90,
                    M_min: int = 256, M_max: int = 2048, delta: int = 3, seed: int = 0):
    """Layout of W rolling windows of uneven length (batched calibration).

    Window w has length L_w ~ U{L_min..L_max} days (L_w + 1 observations), a swarm of
    M_w ~ U{M_min..M_max} particles rounded to a multiple of 32, and starts at day
    T_w = (delta * w) mod (series_days - L_w), the paper's shift of delta days
    between consecutive windows (Sec. 3.1) wrapped to stay inside the series.
    """
    rng = np.random.default_rng(seed)
    L = rng.integers(L_min, L_max + 1, size=W)
    M = (rng.integers(M_min, M_max + 1, size=W) // 32) * 32
    M = np.clip(M, M_min, M_max)
    T = (delta * np.arange(W)) % (series_days - L)
    return {"L": L.astype(np.int64), "M": M.astype(np.int64), "T": T.astype(np.int64)}


def load_series(name: str) -> dict:
    """Loads a stored synthetic series (``tests/golden/series_<name>.json``) as numpy arrays."""
    with open(os.path.join(_GOLDEN, f"series_{name}.json")) as f:
        d = json.load(f)
    return {k: (np.asarray(v, dtype=np.float64) if isinstance(v, list) else v) for k, v in d.items()}


def rolling_window_problems(series: dict, layout: dict) -> list:
    """Cuts windows out of a long stored series: window w covers days T_w .. T_w + L_w; its
    observed deaths are the noisy cumulative counts on those days (the Euler scheme starts from
    the first one), R0 is the series' recovered count on day T_w rounded (when the series
    carries reported I and R, the window carries them too and takes R0 and I0 from their values
    on day T_w), and its swarm size is layout["M"][w]."""
    y = series["yD"]
    R = series["R_true"]
    out = []
    for w, (L, M, T) in enumerate(zip(layout["L"], layout["M"], layout["T"])):
        win = {"yD": y[T:T + L + 1].copy(), "N": float(series["N"]), "R0": float(np.round(R[T])),
               "particles": int(M), "T": int(T), "L": int(L)}
        if "yI" in series:  # reported I and R: R0 and I0 are then the reported values on day T
            win["yI"] = series["yI"][T:T + L + 1].copy()
            win["yR"] = series["yR"][T:T + L + 1].copy()
            win["R0"] = float(win["yR"][0])
            win["I0"] = float(win["yI"][0])
        out.append(win)
    return out

