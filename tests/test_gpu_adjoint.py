"""Discrete-adjoint gradient on the GPU vs the FP64 oracle and central differences (GPU only)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2204_12346_gb300 import sird, synth
from util import box_thetas, rel_err, window

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
def test_adjoint_f64_bit_exact_c4_window(cost, ckpt):
    # the differentiation configuration: 90 days at dt = 0.05 (1800 steps), 4 segments + gamma, mu, I0
    y, N, _, _ = window("c4")
    th = np.concatenate([near_truth("c4", 4, 40, 1), box_thetas(4, 24, 2)])
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
    y, N, _, _ = window("c2", 40)
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
    y, N, _, _ = window("c4")
    th = near_truth("c4", 4, 8, 3)
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
    y, N, _, _ = window("c2")
    th = near_truth("c2", 4, 5, 4)
    cal = sird.Calibrator(y, N, K=4, spd=10, particles=32, iters=1, lb=[1e-3] * 7, ub=[1e6] * 7, precision=64)
    T = torch.from_numpy(np.ascontiguousarray(th.T)).cuda().requires_grad_(True)
    loss = sird.SirdLoss.apply(cal, T)
    (loss * torch.arange(1, 6, dtype=torch.float64, device="cuda")).sum().backward()
    L, G = cal.loss_grad(T.detach())
    assert torch.equal(loss.detach(), L)
    assert torch.allclose(T.grad, G * torch.arange(1, 6, dtype=torch.float64, device="cuda"), rtol=0, atol=0)


def test_polish_never_worsens_and_reports_its_own_fp64_loss():
    y, N, _, _ = window("c2")
    lb, ub = [1e-3] * 4 + [1e-3, 1e-5, 1.0], [2.0] * 4 + [1.0, 0.1, 1e6]
    cal = sird.Calibrator(y, N, K=4, spd=10, particles=512, iters=40, lb=lb, ub=ub, log_scale=[1] * 7,
                          precision=32, reeval_topk=8, seed=2)
    r0 = cal.calibrate()
    r1 = cal.polish(k=8, iters=30, first_step=1e-2)
    assert r1["loss"] <= r0["loss"]
    assert all(lo <= t <= hi for t, lo, hi in zip(r1["theta"], lb, ub))
    T = torch.from_numpy(np.asarray(r1["theta"]).reshape(-1, 1)).cuda()
    assert cal.eval(T).item() == r1["loss"]
