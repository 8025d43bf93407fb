"""Helpers shared by the tests (no method arithmetic)."""
import numpy as np

from paper_2204_12346_gb300 import configs, synth


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def rel_err(got, want):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    return np.abs(got - want) / np.maximum(np.abs(want), 1e-300)


def window(name, days=None):
    """(yD, N, K, spd) of a stored series, optionally cut to its first `days` days."""
    s = synth.load_series(name)
    y = s["yD"] if days is None else s["yD"][: days + 1]
    return y, s["N"], int(s.get("K", 1)), int(s["spd"])


def log_box(K):
    lb, ub = configs.bounds(K, log=True)
    return np.array(lb), np.array(ub)


def box_thetas(K, M, seed, extra=0):
    lb, ub = log_box(K)
    return f32(synth.box_sample(lb, ub, [1] * len(lb), M, np.random.default_rng(seed)))
