"""Argument checks of the binding of the no-allocation step (CPU: CPU tensors stand in for device
buffers, with the device check switched off; one test keeps it on)."""
import numpy as np
import pytest
import torch

from paper_2204_12346_gb300 import sird

P, M, LD, N_OBS = 7, 100, 128, 61


def bufs():
    x = torch.zeros(P, LD, dtype=torch.float32)
    return dict(obs=torch.zeros(N_OBS, dtype=torch.float32), x=x, v=torch.zeros_like(x), pbest=torch.zeros_like(x),
                pbest_f=torch.zeros(LD, dtype=torch.float32), gbest=torch.zeros(P, dtype=torch.float32),
                gbest_index=torch.zeros(1, dtype=torch.int32))


def check(b, require_cuda=False, M_=M):
    return sird.check_noalloc_buffers(P, M_, N_OBS, b["obs"], b["x"], b["v"], b["pbest"], b["pbest_f"], b["gbest"],
                                      b["gbest_index"], require_cuda=require_cuda)


def test_consistent_buffers_pass():
    assert check(bufs()) == LD
    b = bufs()
    big = torch.zeros(P, 300, dtype=torch.float32)
    b["x"], b["v"], b["pbest"] = big[:, :M], torch.zeros(P, 300)[:, :M], torch.zeros(P, 300)[:, :M]
    b["pbest_f"] = torch.zeros(300)
    assert check(b) == 300


@pytest.mark.parametrize("name,bad,msg", [
    ("v", torch.zeros(P, 64, dtype=torch.float32), "leading dimension"),
    ("v", torch.zeros(P, 256, dtype=torch.float32), "leading dimension"),
    ("pbest", torch.zeros(P, LD, dtype=torch.float64), "float32"),
    ("x", torch.zeros(P - 1, LD, dtype=torch.float32), "P=7"),
    ("x", torch.zeros(LD, P, dtype=torch.float32).t(), "unit stride"),
    ("pbest_f", torch.zeros(LD - 1, dtype=torch.float32), "at least 128"),
    ("gbest", torch.zeros(P - 1, dtype=torch.float32), "at least 7"),
    ("obs", torch.zeros(N_OBS - 1, dtype=torch.float32), "at least 61"),
    ("obs", torch.zeros(N_OBS, dtype=torch.float64), "float32"),
    ("gbest_index", torch.zeros(1, dtype=torch.int64), "int32"),
])
def test_each_mismatch_is_refused(name, bad, msg):
    b = bufs()
    b[name] = bad
    with pytest.raises(ValueError, match=msg):
        check(b)


def test_fewer_columns_than_particles_is_refused():
    with pytest.raises(ValueError, match="fewer than 200 particles"):
        check(bufs(), M_=200)


def test_host_tensors_are_refused_when_device_buffers_are_needed():
    with pytest.raises(ValueError, match="CUDA device"):
        check(bufs(), require_cuda=True)


def test_the_step_refuses_before_calling_the_library():
    """step_f32_noalloc checks its buffers before any library call: mismatched host tensors are
    refused even where the library cannot run."""
    y = np.linspace(0.0, 100.0, N_OBS)
    b = bufs()
    with pytest.raises(ValueError, match="CUDA device"):
        sird.step_f32_noalloc(y, 38e6, b["obs"], b["x"], b["v"], b["pbest"], b["pbest_f"], b["gbest"], 0, K=4,
                              lb=[1e-3] * 4 + [1e-3, 1e-5, 1.0], ub=[2.0] * 4 + [1.0, 0.1, 1e6], log_scale=[1] * 7)
