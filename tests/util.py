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


RHO_F32 = 4e-6  # relative accuracy of the FP32 trajectory's D: 2^-24 x (sqrt(1800 steps) + 90 day folds) ~ 3.5e-6


def fp32_loss_tol(O, pb, theta, cost="mse", base=1e-5, rho=RHO_F32):
    """Relative tolerance of an FP32 loss at theta: `base` (the contract's 1e-5), plus the change
    that relative errors rho of the trajectory's D_i can cause through the residuals, relative
    to the loss.  Far from a fit the second term is tiny; at a good fit (small residuals against
    large counts) it is what FP32 can resolve.  O is the oracle module."""
    y = np.asarray(pb.yD, dtype=np.float64)
    n = y.size
    D = O.simulate(pb, theta)["D"][:n]
    e = y - D
    dD = rho * np.abs(D)
    if cost == "mse":
        L, dL = np.mean(e * e), (2.0 / n) * np.sum(np.abs(e) * dD)
    elif cost == "mxse":
        i = int(np.argmax(e * e))
        L, dL = e[i] ** 2, 2.0 * abs(e[i]) * dD[i]
    elif cost == "mae":
        L, dL = np.mean(np.abs(e)), np.sum(dD) / n
    else:
        keep = y != 0
        L = 100.0 * np.mean(np.abs(e[keep] / y[keep]))
        dL = 100.0 * np.sum(dD[keep] / np.abs(y[keep])) / max(int(keep.sum()), 1)
    return base + dL / max(L, 1e-300)
