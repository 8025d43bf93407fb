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


# The contract's tolerance for FP32 losses against the oracle's FP64 losses at the same
# (FP32-representable) parameter vector: 1e-5 relative, at every point -- near a fit too.
TOL32 = 1e-5


def assert_fp32_losses(got, want, what=""):
    """Every FP32 loss within TOL32 (relative) of the oracle's FP64 loss; returns the largest
    relative error seen (the tests print it)."""
    err = rel_err(got, want)
    worst = float(np.max(err)) if err.size else 0.0
    bad = np.flatnonzero(err > TOL32)
    assert bad.size == 0, (what, bad[:8].tolist(), err[bad[:8]].tolist())
    return worst
