"""The entry point that allocates nothing (sird_pso_step_f32_noalloc) against sird_pso_step.

Callers that cannot allocate device memory when they need a step (a framework that owns the
whole device budget and lends only its own buffers, a latency-critical loop) use this entry
point on a swarm they own.  Both entry points run the same kernel on the same inputs, so this
file requires, through the C ABI, the same swarm bit for bit as the handle-based step on the
initialisation and on two iterations in a row -- positions, velocities, personal bests, their
losses, the global best and its index -- for MSE on the integer series and for MAE and MAPE on a
series that is not integer-valued and whose first observation is 0 (the reciprocals MAPE uses
come from the double observations in both paths; MAPE skips the zero).  It also checks that a
window longer than the fixed scratch holds is rejected.  It is collected last and also passes
on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

from paper_2204_12346_gb300 import configs, sird, synth

pytestmark = pytest.mark.gpu


def non_integer_series(y):
    """The stored deaths plus a fractional part on every day but the first (which stays 0)."""
    i = np.arange(y.size)
    z = y + np.where(i > 0, 0.25 + 0.2 * np.sin(1.7 * i), 0.0)
    assert z[0] == 0.0 and np.all(z[1:] != np.round(z[1:]))
    return z


@pytest.mark.parametrize("cost,integer", [(sird.COST_MSE, True), (sird.COST_MAE, False), (sird.COST_MAPE, False)])
def test_noalloc_step_matches_handle_step(cost, integer):
    torch.cuda.set_device(0)
    ser = synth.load_series("60d")
    y = ser["yD"] if integer else non_integer_series(ser["yD"])
    lb, ub = configs.bounds(4, log=True)
    M = 1000
    kw = dict(K=4, spd=10, cost=cost, lb=lb, ub=ub, log_scale=[1] * 7, seed=21, stream_id=3)
    ref = sird.Calibrator(y, ser["N"], particles=M, iters=2, precision=32,
                          launch_mode=sird.LAUNCH_PER_ITER, **kw)
    P = ref.P
    ld = 1024
    dev = torch.device("cuda", 0)
    x = torch.zeros(P, ld, dtype=torch.float32, device=dev)
    v = torch.zeros_like(x)
    pb = torch.zeros_like(x)
    pbf = torch.zeros(ld, dtype=torch.float32, device=dev)
    gb = torch.zeros(sird.MAX_PARAMS, dtype=torch.float32, device=dev)
    gidx = torch.zeros(1, dtype=torch.int32, device=dev)
    obs = torch.from_numpy((y - y[0]).astype(np.float32)).to(dev)  # the handle's FP32 copy

    ref.init()
    for it in range(3):  # the initialisation, then two iterations in a row
        if it > 0:
            ref.step(1)
        sird.step_f32_noalloc(y, ser["N"], obs, x, v, pb, pbf, gb, it, gbest_index=gidx, particles=M, **kw)
        torch.cuda.synchronize()
        st = ref.get_state()
        for name, got in (("x", x), ("v", v), ("pbest", pb)):
            g = got[:, :M].cpu().numpy()
            assert np.array_equal(g, st[name].astype(np.float32)), f"{name} at call {it}"
        assert np.array_equal(pbf[:M].cpu().numpy(), st["pbest_f"].astype(np.float32)), f"pbest_f at call {it}"
        assert int(gidx.item()) == st["gbest_idx"]
        assert np.array_equal(gb[:P].cpu().numpy(), st["pbest"][:, st["gbest_idx"]].astype(np.float32))


def test_noalloc_rejects_windows_beyond_its_scratch():
    torch.cuda.set_device(0)
    n = 4097
    y = np.arange(n, dtype=np.float64)
    dev = torch.device("cuda", 0)
    x, v, pb = (torch.zeros(4, 64, dtype=torch.float32, device=dev) for _ in range(3))
    pbf = torch.zeros(64, dtype=torch.float32, device=dev)
    gb = torch.zeros(4, dtype=torch.float32, device=dev)
    with pytest.raises(sird.SirdError) as e:
        sird.step_f32_noalloc(y, 38e6, torch.zeros(n, device=dev), x, v, pb, pbf, gb, 0,
                              particles=32, lb=[0] * 4, ub=[1, 1, 0.1, 1e6])
    assert e.value.status == sird.ERR_ARG and "SIRD_NOALLOC_MAX_OBS" in str(e.value)
