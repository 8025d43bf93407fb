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
    traj = O.simulate(pb, theta)

    def cost_and_bound(yx, xhat, scale):
        e = (yx - xhat) / scale
        dx = rho * np.abs(xhat) / scale
        if cost == "mse":
            return np.mean(e * e), (2.0 / n) * np.sum(np.abs(e) * dx)
        if cost == "mxse":
            i = int(np.argmax(e * e))
            return e[i] ** 2, 2.0 * abs(e[i]) * dx[i]
        if cost == "mae":
            return np.mean(np.abs(e)), np.sum(dx) / n
        keep = yx != 0
        return (100.0 * np.mean(np.abs((yx[keep] - xhat[keep]) / yx[keep])),
                100.0 * np.sum(rho * np.abs(xhat[keep]) / np.abs(yx[keep])) / max(int(keep.sum()), 1))

    if getattr(pb, "objective", 0) == 1:  # F_IRD: the largest of the three normalised costs
        parts = []
        for key, yx in (("I", pb.yI), ("R", pb.yR), ("D", pb.yD)):
            yx = np.asarray(yx, dtype=np.float64)
            rng = yx.max() - yx.min()
            scale = 1.0 if cost == "mape" or not rng > 0 else rng
            parts.append(cost_and_bound(yx, traj[key][:n], scale))
        L = max(c for c, _ in parts)
        dL = max(b for _, b in parts)
    else:
        L, dL = cost_and_bound(y, traj["D"][:n], 1.0)
    return base + dL / max(L, 1e-300)
