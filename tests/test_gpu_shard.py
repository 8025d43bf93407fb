"""One FP32 swarm split by particle over shard handles (GPU only): the shards, exchanging their
best between iterations, hold exactly the personal bests of the unsharded swarm, and the FP64
re-evaluation of the gathered top-k gives the unsharded answer.  The exchange runs on the host
between launches (in-process, and across two gloo ranks sharing the GPU), so no kernel waits on
another."""
import os
import socket

import numpy as np
import pytest
import torch

from paper_2204_12346_gb300 import configs, shard as S, sird
from util import window

pytestmark = pytest.mark.gpu

TOTAL, ITERS, TOPK = 4000 + 37, 12, 16  # ragged; shards of <= 2048 (one top-k call)


@pytest.fixture(scope="module", autouse=True)
def _dev():
    torch.cuda.set_device(0)


def setup():
    y, N, _, _ = window("60d")
    lb, ub = configs.bounds(4, True)
    return y, N, dict(K=4, spd=10, lb=lb, ub=ub, log_scale=[1] * 7, seed=11, stream_id=3, iters=ITERS, precision=32)


def shard_handles(world):
    y, N, kw = setup()
    hs = []
    for r in range(world):
        off, cnt = S.shard_range(TOTAL, r, world)
        hs.append(sird.Calibrator(y, N, particles=cnt, launch_mode=sird.LAUNCH_PER_ITER, **kw).set_shard(off, TOTAL))
    return hs


def unsharded():
    y, N, kw = setup()
    cal = sird.Calibrator(y, N, particles=TOTAL, reeval_topk=TOPK, **kw)
    r = cal.calibrate()
    return cal.get_state()["pbest_f"], r


def gather_pbest_f(hs, offsets):
    f = np.full(TOTAL, np.nan, dtype=np.float64)
    for h, off, end in zip(hs, offsets[:-1], offsets[1:]):
        _, lo, idx = h.topk(end - off, with_index=True)  # every personal best, with its global index
        f[idx] = lo
    return f


@pytest.mark.parametrize("world", [2, 3])
def test_shards_in_one_process_follow_the_unsharded_swarm(world):
    hs = shard_handles(world)
    offsets = S.shard_offsets(TOTAL, world)

    def exchange():
        bests = [h.shard_best() for h in hs]
        loss, idx, z = min(bests, key=lambda b: S.best_key(b[0], b[1]))
        for h in hs:
            h.set_gbest(z, loss, idx)
        return loss, idx

    for h in hs:
        h.init()
    exchange()
    for _ in range(ITERS):
        for h in hs:
            h.step(1)
        g = exchange()
    want_f, want = unsharded()
    got_f = gather_pbest_f(hs, offsets)
    assert np.array_equal(got_f, want_f.astype(np.float64))
    assert g[1] == int(np.lexsort((np.arange(TOTAL), want_f))[0])
    # the answer: FP64 re-evaluation of the gathered top-k
    rows = []
    for h in hs:
        th, lo, idx = h.topk(TOPK, with_index=True)
        rows += [(lo[j], idx[j], th[j]) for j in range(TOPK)]
    rows.sort(key=lambda t: (t[0], t[1]))
    top = rows[:TOPK]
    f64 = hs[0].eval64(np.array([t[2] for t in top]))
    best = min(range(TOPK), key=lambda j: (f64[j], top[j][1]))
    assert top[best][1] == want["index"] and f64[best] == want["loss"]
    # a shard's own result reports its best with the global index
    r = hs[-1].result()
    assert offsets[-2] <= r["index"] < offsets[-1]


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    y, N, kw = setup()
    off, cnt = S.shard_range(TOTAL, rank, world)
    cal = sird.Calibrator(y, N, particles=cnt, launch_mode=sird.LAUNCH_PER_ITER, **kw).set_shard(off, TOTAL)
    sw = S.ShardedSwarm(cal, S.shard_offsets(TOTAL, world))
    g = sw.run(ITERS)
    res = sw.result(TOPK)
    _, lo, idx = cal.topk(cnt, with_index=True)
    q.put((rank, idx, lo, g[:2], res["index"], res["loss"]))
    dist.destroy_process_group()


def test_shards_on_two_gloo_ranks_follow_the_unsharded_swarm():
    import torch.multiprocessing as mp

    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    want_f, want = unsharded()
    f = np.full(TOTAL, np.nan)
    for _, idx, lo, _, _, _ in got:
        f[idx] = lo
    assert np.array_equal(f, want_f.astype(np.float64))
    for t in got:
        assert t[4] == want["index"] and t[5] == want["loss"]
        assert t[3][1] == int(np.lexsort((np.arange(TOTAL), want_f))[0])


def test_shard_calls_check_their_arguments():
    y, N, kw = setup()
    cal = sird.Calibrator(y, N, particles=64, launch_mode=sird.LAUNCH_PER_ITER, **kw)

    def status(fn, *a):
        with pytest.raises(sird.SirdError) as e:
            fn(*a)
        cal._lib.sird_pso_clear_error(cal.h)
        return e.value.status

    assert status(cal.set_shard, TOTAL - 10, TOTAL) == 1  # particles past the end of the swarm
    assert status(cal.set_shard, -1, TOTAL) == 1
    cal.set_shard(64, TOTAL)
    assert status(cal.shard_best) == 5  # before init
    assert status(cal.calibrate) == 5  # a shard does not calibrate on its own
    assert status(cal.get_state) == 7
    cal.init()
    assert status(cal.set_shard, 0, TOTAL) == 5  # after init
    assert status(cal.set_gbest, np.full(7, 50.0, np.float32), 1.0, 0) == 1  # outside the box
    loss, idx, z = cal.shard_best()
    assert 64 <= idx < 128
    assert status(cal.set_gbest, z, loss, TOTAL) == 1  # index past the swarm
    cal.set_gbest(z, loss, idx)
    cal.step(1)
    c64 = sird.Calibrator(y, N, particles=64, **dict(kw, precision=64))
    with pytest.raises(sird.SirdError) as e:
        c64.set_shard(0, TOTAL)
    assert e.value.status == 7
