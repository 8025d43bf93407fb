"""The entry point that allocates nothing (sird_pso_step_f32_noalloc) against sird_pso_step.

Callers that cannot allocate device memory when they need a step (a framework that owns the
whole device budget and lends only its own buffers, a latency-critical loop) use this entry
point on a swarm they own.  This file checks, through the C ABI, that it gives the same
swarm as the handle-based step on the initialisation and on two iterations in a row, and
that it rejects a window longer than its fixed scratch holds.  It is collected last and also
passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

from paper_2204_12346_gb300 import configs, sird, synth

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.mark.parametrize("cost", [sird.COST_MSE, sird.COST_MAPE])
def test_noalloc_step_matches_handle_step(cost):
    torch.cuda.set_device(0)
    ser = synth.load_series("60d")
    y = ser["yD"]
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
    obs = torch.from_numpy(y.astype(np.float32)).to(dev)

    ref.init()
    for it in range(3):  # the initialisation, then two iterations in a row
        if it > 0:
            ref.step(1)
        sird.step_f32_noalloc(y, ser["N"], obs, x, v, pb, pbf, gb, it, gbest_index=gidx, particles=M, **kw)
        torch.cuda.synchronize()
        st = ref.get_state()
        for name, got in (("x", x), ("v", v), ("pbest", pb)):
            g = got[:, :M].cpu().numpy().astype(np.float64)
            want = st[name].astype(np.float64)
            np.testing.assert_allclose(g, want, rtol=TOL32, atol=0, err_msg=f"{name} at call {it}")
        np.testing.assert_allclose(pbf[:M].cpu().numpy(), st["pbest_f"], rtol=TOL32, atol=0)
        assert int(gidx.item()) == st["gbest_idx"]
        np.testing.assert_allclose(gb[:P].cpu().numpy(), st["pbest"][:, st["gbest_idx"]], rtol=TOL32, atol=0)


def test_noalloc_rejects_windows_beyond_its_scratch():
    torch.cuda.set_device(0)
    n = 4097
    y = np.arange(n, dtype=np.float64)
    dev = torch.device("cuda", 0)
    t = torch.zeros(4, 64, dtype=torch.float32, device=dev)
    with pytest.raises(sird.SirdError) as e:
        sird.step_f32_noalloc(y, 38e6, torch.zeros(n, device=dev), t, t, t, t[0], t[:, 0], 0,
                              particles=32, lb=[0] * 4, ub=[1, 1, 0.1, 1e6])
    assert e.value.status == sird.ERR_ARG and "SIRD_NOALLOC_MAX_OBS" in str(e.value)
