"""Discrete-adjoint gradient on the GPU vs the FP64 oracle and central differences (GPU only)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2204_12346_gb300 import sird, synth
from util import box_thetas, f32, rel_err, window

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    torch.cuda.set_device(0)
    O.build()


def near_truth(name, K, M, seed, spread=0.05):
    s = synth.load_series(name)
    t = np.asarray(s["theta_true"], dtype=np.float64)
    if K != len(t) - 3:
        t = np.concatenate([np.full(K, t[:len(t) - 3].mean()), t[-3:]])
    rng = np.random.default_rng(seed)
    return t * np.exp(rng.normal(0.0, spread, (M, t.size)))


def gpu_loss_grad(cal, th, ckpt=16):
    T = torch.from_numpy(np.ascontiguousarray(th.T)).cuda()
    L, G, GU = cal.loss_grad(T, ckpt_every=ckpt, grad_u0=True)
    torch.cuda.synchronize()
    return L.cpu().numpy(), G.cpu().numpy().T, GU.cpu().numpy().T


@pytest.mark.parametrize("cost", ["mse", "mxse", "mae", "mape"])
@pytest.mark.parametrize("ckpt", [1, 7, 16, 64])
def test_adjoint_f64_bit_exact_90_day_window(cost, ckpt):
    # the differentiation configuration: 90 days at dt = 0.05 (1800 steps), 4 segments + gamma, mu, I0
    y, N, _, _ = window("90d")
    th = np.concatenate([near_truth("90d", 4, 40, 1), box_thetas(4, 24, 2)])
    cal = sird.Calibrator(y, N, K=4, spd=20, cost=sird.COSTS[cost], particles=32, iters=1, lb=[1e-3] * 7,
                          ub=[1e6] * 7, precision=64)
    L, G, GU = gpu_loss_grad(cal, th, ckpt)
    pb = O.Problem(yD=y, N=N, K=4, spd=20, cost=O.COSTS[cost])
    for j in range(th.shape[0]):
        Lo, Go, GUo = O.loss_grad(pb, th[j])
        assert L[j] == Lo
        assert np.array_equal(G[j], Go), (j, rel_err(G[j], Go))
        assert np.array_equal(GU[j], GUo)


def test_adjoint_f64_ramp_form_bit_exact():
    y, N, _, _ = window("60d", 40)
    rng = np.random.default_rng(6)
    M = 64
    th = np.column_stack([rng.uniform(0.1, 0.4, M), rng.uniform(0.1, 0.4, M), rng.uniform(1, 39, M),
                          rng.uniform(1, 39, M), rng.uniform(0.05, 0.2, M), rng.uniform(1e-3, 4e-3, M),
                          rng.uniform(5e3, 2e4, M)])
    cal = sird.Calibrator(y, N, beta_form=sird.BETA_RAMP, particles=32, iters=1, lb=[1e-3] * 7, ub=[1e6] * 7,
                          precision=64)
    L, G, _ = gpu_loss_grad(cal, th, 16)
    pb = O.Problem(yD=y, N=N, beta_form=O.BETA_RAMP)
    for j in range(M):
        Lo, Go, _ = O.loss_grad(pb, th[j])
        assert L[j] == Lo and np.array_equal(G[j], Go)


def test_adjoint_matches_central_differences_of_gpu_loss():
    # central differences (h = 1e-6 relative) of the GPU's own FP64 loss
    y, N, _, _ = window("90d")
    th = near_truth("90d", 4, 8, 3)
    cal = sird.Calibrator(y, N, K=4, spd=20, particles=32, iters=1, lb=[1e-3] * 7, ub=[1e6] * 7, precision=64)
    _, G, _ = gpu_loss_grad(cal, th, 16)
    P = th.shape[1]
    h = 1e-6 * np.abs(th)
    plus = np.repeat(th, P, axis=0)
    minus = plus.copy()
    for j in range(th.shape[0]):
        for d in range(P):
            plus[j * P + d, d] += h[j, d]
            minus[j * P + d, d] -= h[j, d]
    Lp = cal.eval(torch.from_numpy(np.ascontiguousarray(plus.T)).cuda()).cpu().numpy()
    Lm = cal.eval(torch.from_numpy(np.ascontiguousarray(minus.T)).cuda()).cpu().numpy()
    fd = ((Lp - Lm) / (2 * h.reshape(-1))).reshape(th.shape)
    scale = np.abs(fd).max(axis=1, keepdims=True)
    assert np.all(np.abs(G - fd) <= 1e-5 * scale + 1e-6 * np.abs(fd))


def test_autograd_function_wraps_the_adjoint():
    y, N, _, _ = window("60d")
    th = near_truth("60d", 4, 5, 4)
    cal = sird.Calibrator(y, N, K=4, spd=10, particles=32, iters=1, lb=[1e-3] * 7, ub=[1e6] * 7, precision=64)
    T = torch.from_numpy(np.ascontiguousarray(th.T)).cuda().requires_grad_(True)
    loss = sird.SirdLoss.apply(cal, T)
    (loss * torch.arange(1, 6, dtype=torch.float64, device="cuda")).sum().backward()
    L, G = cal.loss_grad(T.detach())
    assert torch.equal(loss.detach(), L)
    assert torch.allclose(T.grad, G * torch.arange(1, 6, dtype=torch.float64, device="cuda"), rtol=0, atol=0)


def test_polish_never_worsens_and_reports_its_own_fp64_loss():
    y, N, _, _ = window("60d")
    lb, ub = [1e-3] * 4 + [1e-3, 1e-5, 1.0], [2.0] * 4 + [1.0, 0.1, 1e6]
    cal = sird.Calibrator(y, N, K=4, spd=10, particles=512, iters=40, lb=lb, ub=ub, log_scale=[1] * 7,
                          precision=32, reeval_topk=8, seed=2)
    r0 = cal.calibrate()
    r1 = cal.polish(k=8, iters=30, first_step=1e-2)
    assert r1["loss"] <= r0["loss"]
    assert all(lo <= t <= hi for t, lo, hi in zip(r1["theta"], lb, ub))
    T = torch.from_numpy(np.asarray(r1["theta"]).reshape(-1, 1)).cuda()
    assert cal.eval(T).item() == r1["loss"]


# ---------------------------------------------------------------- FP32 adjoint

def f32_loss_grad(cal, th):
    T = torch.from_numpy(np.ascontiguousarray(th.T).astype(np.float32)).cuda()
    L, G, GU = cal.loss_grad(T, grad_u0=True)
    E = cal.eval(T)
    torch.cuda.synchronize()
    return (L.cpu().numpy(), G.cpu().numpy().T.astype(np.float64), GU.cpu().numpy().T.astype(np.float64),
            E.cpu().numpy())


RHO_F32 = 4e-7  # relative accuracy of the FP32 trajectory's D assumed by the gradient bound: 100x what the losses' 1e-5 at good fits imply (~3e-9)


def residual_bound(pb, th, cost, rho=RHO_F32):
    """|theta_j| times the change of dL/dtheta_j that errors of rho*D_i in the trajectory's D_i can
    cause through the residuals e_i = y_i - D_i (the FP32 path integrates the same map with
    ~rho relative error).  Sensitivities theta_j dD_i/dtheta_j by central differences of the
    oracle's trajectory (h = 1e-5 relative)."""
    n = pb.n_obs if hasattr(pb, "n_obs") else len(pb.yD)
    D = O.simulate(pb, th)["D"][:n]
    y = np.asarray(pb.yD, dtype=np.float64)
    Sens = np.zeros((n, th.size))
    for j in range(th.size):
        tp, tm = th.copy(), th.copy()
        tp[j] *= 1 + 1e-5
        tm[j] *= 1 - 1e-5
        Sens[:, j] = (O.simulate(pb, tp)["D"][:n] - O.simulate(pb, tm)["D"][:n]) / 2e-5
    dD = rho * np.abs(D)
    e = y - D
    if cost == "mse":
        return (2.0 / n) * (dD[:, None] * np.abs(Sens)).sum(0)
    if cost == "mxse":
        i = int(np.argmax(e * e))
        return 2.0 * (dD[i] + np.abs(e[i])) * np.abs(Sens[i]) if np.sort(e * e)[-2] > (1 - 1e-4) * e[i] ** 2 \
            else 2.0 * dD[i] * np.abs(Sens[i])
    w = np.full(n, 1.0 / n) if cost == "mae" else np.where(y != 0, 100.0 / np.maximum(np.abs(y), 1e-300)
                                                           / max(int((y != 0).sum()), 1), 0.0)
    flip = np.abs(e) <= dD  # a residual within the error band may change sign
    return 2.0 * ((w * flip)[:, None] * np.abs(Sens)).sum(0)


def check_f32_gradient(pb, th, L, G, E, cost="mse"):
    """The FP32 loss is the FP32 evaluation's bit for bit; the FP32 gradient equals the oracle's
    FP64 gradient at the same (FP32-representable) theta within
        |theta_j (g32_j - g64_j)| <= 1e-5 (|theta . g64|_inf + L) + residual_bound_j :
    the adjoint's own rounding (lambda recursions compensated, sums per day in FP32, over days in
    FP64) stays near 1e-6 of the gradient's scale, and the FP32 trajectory's error reaches the
    gradient through the residuals, which residual_bound measures."""
    assert np.array_equal(L, E)
    worst = 0.0
    for j in range(th.shape[0]):
        Lo, Go, _ = O.loss_grad(pb, th[j])
        tol = 1e-5 * (np.abs(th[j] * Go).max() + abs(Lo)) + residual_bound(pb, th[j], cost)
        worst = max(worst, (np.abs(th[j] * (G[j] - Go)) / tol).max())
    print("worst gradient error / tolerance", worst)
    assert worst <= 1.0, worst


@pytest.mark.parametrize("cost", ["mse", "mxse", "mae", "mape"])
def test_adjoint_f32_90_day_window(cost):
    y, N, _, _ = window("90d")
    th = f32(np.concatenate([near_truth("90d", 4, 40, 1), box_thetas(4, 24, 2)]))
    cal = sird.Calibrator(y, N, K=4, spd=20, cost=sird.COSTS[cost], particles=32, iters=1, lb=[1e-3] * 7,
                          ub=[1e6] * 7, precision=32)
    L, G, GU, E = f32_loss_grad(cal, th)
    check_f32_gradient(O.Problem(yD=y, N=N, K=4, spd=20, cost=O.COSTS[cost]), th, L, G, E, cost)
    assert np.all(GU[:, 2] == 0.0)


@pytest.mark.parametrize("spd,K,days", [(10, 4, 60), (7, 3, 31), (1, 2, 45)])
def test_adjoint_f32_other_step_counts(spd, K, days):
    # spd 10 (unrolled day), 7 and 1 (generic day loop); K segments not aligned with days
    y, N, _, _ = window("60d", days)
    th = f32(np.concatenate([near_truth("60d", K, 16, 5), box_thetas(K, 16, 6)]))
    cal = sird.Calibrator(y, N, K=K, spd=spd, particles=32, iters=1, lb=[1e-3] * (K + 3), ub=[1e6] * (K + 3),
                          precision=32)
    L, G, _, E = f32_loss_grad(cal, th)
    check_f32_gradient(O.Problem(yD=y, N=N, K=K, spd=spd), th, L, G, E)


def test_adjoint_f32_ramp_form():
    y, N, _, _ = window("60d", 40)
    rng = np.random.default_rng(7)
    M = 48
    th = f32(np.column_stack([rng.uniform(0.1, 0.4, M), rng.uniform(0.1, 0.4, M), rng.uniform(1, 39, M),
                              rng.uniform(1, 39, M), rng.uniform(0.05, 0.2, M), rng.uniform(1e-3, 4e-3, M),
                              rng.uniform(5e3, 2e4, M)]))
    cal = sird.Calibrator(y, N, beta_form=sird.BETA_RAMP, particles=32, iters=1, lb=[1e-3] * 7, ub=[1e6] * 7,
                          precision=32)
    L, G, _, E = f32_loss_grad(cal, th)
    check_f32_gradient(O.Problem(yD=y, N=N, beta_form=O.BETA_RAMP), th, L, G, E)


def test_adjoint_f32_ragged_particle_count_and_leading_dimension():
    # M not a multiple of the block, theta rows padded (ld > M)
    y, N, _, _ = window("90d")
    th = f32(box_thetas(4, 131, 9))
    cal = sird.Calibrator(y, N, K=4, spd=20, particles=32, iters=1, lb=[1e-3] * 7, ub=[1e6] * 7, precision=32)
    T = torch.zeros(7, 160, dtype=torch.float32, device="cuda")
    T[:, :131] = torch.from_numpy(th.T.astype(np.float32)).cuda()
    L, G = cal.loss_grad(T[:, :131])
    L2, G2, _, _ = f32_loss_grad(cal, th)
    assert np.array_equal(L.cpu().numpy(), L2)
    assert np.array_equal(G.cpu().numpy().T.astype(np.float64), G2)


def test_polish_f32_improves_and_reports_fp64_loss():
    y, N, _, _ = window("60d")
    lb, ub = [1e-3] * 4 + [1e-3, 1e-5, 1.0], [2.0] * 4 + [1.0, 0.1, 1e6]
    cal = sird.Calibrator(y, N, K=4, spd=10, particles=512, iters=40, lb=lb, ub=ub, log_scale=[1] * 7,
                          precision=32, reeval_topk=8, seed=2)
    r0 = cal.calibrate()
    r32 = cal.polish(k=8, iters=30, first_step=1e-2, precision=32)
    assert r32["loss"] < r0["loss"]
    assert all(lo <= t <= hi for t, lo, hi in zip(r32["theta"], lb, ub))
    pb = O.Problem(yD=y, N=N, K=4, spd=10)
    assert O.loss(pb, r32["theta"]) == r32["loss"]
    r64 = cal.polish(k=8, iters=30, first_step=1e-2, precision=64)
    # both reach the same basin: within 1% of each other after 30 iterations
    assert abs(r32["loss"] - r64["loss"]) <= 1e-2 * r64["loss"]
