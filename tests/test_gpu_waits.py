"""Failure detection of the device-side bounded waits (GPU only).

The cooperative kernels wait for one another at a grid barrier (flat batch form) or for the
other blocks' exchange slots (persistent single-window launch).  Every such wait polls a limited
number of times; a block that gives up raises an abort flag that releases the others, the kernel
returns early, and the host reads SIRD_ERR_TIMEOUT.  The tests make the waits run out by setting
the poll limit to one (SIRD_WAIT_LIMIT=1) — no fault, trap or endless loop — and check the
status, then that the context still runs a normal calibration."""
import numpy as np
import pytest
import torch

from paper_2204_12346_gb300 import configs, sird, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    torch.cuda.set_device(0)


def windows():
    ser = synth.load_series("450d")
    lay = {"L": np.array([30, 40, 25]), "M": np.array([600, 900, 300]), "T": np.array([0, 100, 200])}
    return synth.rolling_window_problems(ser, lay)


def test_flat_batch_barrier_wait_runs_out(monkeypatch):
    lb, ub = configs.bounds(6, log=True)
    kw = dict(K=6, spd=10, lb=lb, ub=ub, log_scale=[1] * 9, seed=1, block_size=256, launch_mode=sird.LAUNCH_FLAT)
    monkeypatch.setenv("SIRD_WAIT_LIMIT", "1")
    batch = sird.Batch(windows(), iters=20, **kw)
    with pytest.raises(sird.SirdError) as err:
        batch.calibrate()
    assert err.value.status == sird.ERR_TIMEOUT
    batch.close()
    monkeypatch.delenv("SIRD_WAIT_LIMIT")
    ok = sird.Batch(windows(), iters=20, **kw).calibrate()
    ref = sird.Batch(windows(), iters=20, **dict(kw, launch_mode=sird.LAUNCH_WINDOW_PER_BLOCK)).calibrate()
    assert [r["index"] for r in ok] == [r["index"] for r in ref]


def test_persistent_exchange_wait_runs_out(monkeypatch):
    s = synth.load_series("60d")
    lb, ub = configs.bounds(4, log=True)
    kw = dict(K=4, spd=10, particles=4096, iters=30, lb=lb, ub=ub, log_scale=[1] * 7, precision=32,
              launch_mode=sird.LAUNCH_PERSISTENT, seed=2)
    monkeypatch.setenv("SIRD_WAIT_LIMIT", "1")
    cal = sird.Calibrator(s["yD"], s["N"], **kw)
    with pytest.raises(sird.SirdError) as err:
        cal.calibrate()
    assert err.value.status == sird.ERR_TIMEOUT
    cal.close()
    monkeypatch.delenv("SIRD_WAIT_LIMIT")
    r = sird.Calibrator(s["yD"], s["N"], **kw).calibrate()
    r2 = sird.Calibrator(s["yD"], s["N"], **dict(kw, launch_mode=sird.LAUNCH_PER_ITER)).calibrate()
    assert r["index"] == r2["index"] and r["loss"] == r2["loss"]
