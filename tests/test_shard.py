"""One swarm split by particle over CPU ranks (gloo): the key that orders shard bests, the
shard ranges, the exchange, and that shards of the oracle's swarm exchanging their best follow
the unsharded swarm exactly (Sec. 3.3: the particles are independent, the synchronous global
best is their only coupling)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from paper_2204_12346_gb300 import shard as S  # noqa: E402

TOTAL, ITERS, TOPK, SEED = 37, 6, 8, 3


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleShard:
    """Particles offset .. offset + count - 1 of the oracle's FP32-stored swarm, in the shard
    interface of paper_2204_12346_gb300.shard (linear bounds: theta = z)."""

    def __init__(self, O, pb, offset, count, lb, ub):
        self.O, self.pb, self.off = O, pb, offset
        self.pso = O.PSO(pb, count, lb, ub, logdim=[0] * len(lb), seed=SEED, store_f32=True, p_offset=offset)

    def init(self):
        self.pso.init()

    def step(self, n):
        self.pso.step(n)

    def shard_best(self):
        g = self.O.argmin(self.pso.pbest_f)
        return float(self.pso.pbest_f[g]), g + self.off, self.pso.pbest[g].astype(np.float32)

    def set_gbest(self, z, loss, index):
        self.pso.gbest[:] = np.asarray(z, dtype=np.float64)
        self.pso.st.gbest_idx = int(index)
        self.pso.st.gbest_f = float(loss)

    def topk(self, k, with_index=True):
        f = np.where(np.isnan(self.pso.pbest_f), np.inf, self.pso.pbest_f)
        order = np.lexsort((np.arange(f.size), f))[:k]
        return self.pso.pbest[order].copy(), self.pso.pbest_f[order].copy(), order + self.off

    def eval64(self, thetas):
        return self.O.losses(self.pb, thetas)


def _problem(O):
    from paper_2204_12346_gb300 import configs
    from util import window

    y, N, _, _ = window("30d")
    lb, ub = configs.bounds(1, log=False)
    return O.Problem(yD=y, N=N, K=1, spd=10), lb, ub


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    import oracle as O

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pb, lb, ub = _problem(O)
    off, cnt = S.shard_range(TOTAL, rank, world)
    sh = OracleShard(O, pb, off, cnt, lb, ub)
    sw = S.ShardedSwarm(sh, S.shard_offsets(TOTAL, world))
    g = sw.run(ITERS)
    res = sw.result(TOPK)
    q.put((rank, off, sh.pso.pbest_f.copy(), g[:2], (res["index"], res["loss"], res["loss_search"])))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_oracle_swarm_follows_the_unsharded_one(world):
    import torch.multiprocessing as mp

    import oracle as O

    O.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    pb, lb, ub = _problem(O)
    ref = O.PSO(pb, TOTAL, lb, ub, logdim=[0] * len(lb), seed=SEED, store_f32=True).init().step(ITERS)
    pbest_f = np.concatenate([t[2] for t in got])
    assert [t[1] for t in got] == S.shard_offsets(TOTAL, world)[:-1]
    assert np.array_equal(pbest_f, ref.pbest_f)
    for t in got:  # every rank agrees on the global best and the re-evaluated answer
        assert t[3] == (ref.gbest_f, ref.gbest_idx)
        idx, f = ref.reeval_topk(TOPK)
        assert t[4][0] == idx and t[4][1] == f and t[4][2] == ref.pbest_f[idx]


def test_shard_ranges_cover_the_swarm():
    for total in (1, 5, 37, 1 << 20):
        for world in (1, 2, 3, 8):
            parts = [S.shard_range(total, r, world) for r in range(world)]
            assert sum(c for _, c in parts) == total
            assert all(parts[r][0] + parts[r][1] == parts[r + 1][0] for r in range(world - 1))
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
            offs = S.shard_offsets(total, world)
            for i in {0, total // 2, total - 1}:
                r = S.owner_of(i, offs)
                assert parts[r][0] <= i < parts[r][0] + parts[r][1]


def test_best_key_orders_by_loss_then_index():
    rng = np.random.default_rng(0)
    vals = [(float(v), int(i)) for v, i in zip(rng.choice([-3.0, 0.0, 0.5, 1.0, 2.5e7, np.inf], 200),
                                                 rng.integers(0, 1 << 26, 200))]
    vals += [(np.nan, 5), (np.nan, 2)]
    want = sorted(vals, key=lambda t: (np.inf if np.isnan(t[0]) else t[0], t[1]))
    got = sorted(vals, key=lambda t: S.best_key(*t))
    assert [(np.inf if np.isnan(a) else a, b) for a, b in got] == [(np.inf if np.isnan(a) else a, b)
                                                                   for a, b in want]
    for v, i in vals:
        f, j = S.key_parts(S.best_key(v, i))
        assert j == i and (f == v or (np.isnan(v) and f == np.inf))
    assert all(-(1 << 63) <= S.best_key(v, i) < (1 << 63) for v, i in vals)


class _LeavingShard:
    """Wraps a shard; the rank with leave=True exits the process at the start of its step number
    `at` (between steps: its previous exchange is complete, nothing of it is in flight)."""

    def __init__(self, shard, leave, at):
        self.shard, self.leave, self.at, self.steps = shard, leave, at, 0

    def __getattr__(self, name):
        return getattr(self.shard, name)

    def step(self, n):
        self.steps += 1
        if self.leave and self.steps == self.at:
            os._exit(3)
        self.shard.step(n)


def _rank_leave_main(rank, world, port, q, leaving_rank, at):
    from datetime import timedelta

    import torch.distributed as dist

    import oracle as O

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=20))
    pb, lb, ub = _problem(O)
    off, cnt = S.shard_range(TOTAL, rank, world)
    sh = _LeavingShard(OracleShard(O, pb, off, cnt, lb, ub), rank == leaving_rank, at)
    try:
        S.ShardedSwarm(sh, S.shard_offsets(TOTAL, world)).run(ITERS)
        q.put((rank, "finished", None))
    except S.ShardFailure as e:
        q.put((rank, "failed", e.step))
    q.close()
    q.join_thread()
    os._exit(0)  # the process group lost a member: leave without a collective shutdown


def test_a_rank_that_leaves_is_detected_at_the_next_exchange():
    # failure detection on the host: rank 2 of 3 leaves at the start of its second step; the
    # other two finish that step and their next exchange fails (a lost peer or the process
    # group's timeout), reported as ShardFailure naming the exchange after iteration 2
    import time

    import torch.multiprocessing as mp

    import oracle as O

    O.build()
    world, leaving, at = 3, 2, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_leave_main, args=(r, world, port, q, leaving, at)) for r in range(world)]
    t0 = time.monotonic()
    for p in procs:
        p.start()
    try:
        got = sorted((q.get(timeout=120) for _ in range(world - 1)), key=lambda t: t[0])
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert got == [(0, "failed", at), (1, "failed", at)], got
    assert procs[leaving].exitcode == 3 and procs[0].exitcode == 0 and procs[1].exitcode == 0
    assert time.monotonic() - t0 < 90


def _rank_groups_main(rank, world, port, q):
    import torch.distributed as dist

    import oracle as O

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    groups = [dist.new_group([0, 1]), dist.new_group([2, 3])]  # every rank creates every group
    g = rank // 2
    pb, lb, ub = _problem(O)
    sub_rank, sub_world = rank % 2, 2
    off, cnt = S.shard_range(TOTAL, sub_rank, sub_world)
    sh = OracleShard(O, pb, off, cnt, lb, ub)
    sh.pso = O.PSO(pb, cnt, lb, ub, logdim=[0] * len(lb), seed=SEED + g, store_f32=True, p_offset=off)
    sw = S.ShardedSwarm(sh, S.shard_offsets(TOTAL, sub_world), group=groups[g])
    gb = sw.run(ITERS)
    res = sw.result(TOPK)
    q.put((rank, gb[:2], res["index"], res["loss"]))
    dist.destroy_process_group()


def test_two_swarms_on_subgroups_of_four_ranks():
    # two windows' swarms side by side, each split over its own pair of ranks: the exchange
    # addresses the owner through its global rank, and each pair reproduces its own swarm
    import torch.multiprocessing as mp

    import oracle as O

    O.build()
    world = 4
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_groups_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    pb, lb, ub = _problem(O)
    for g in (0, 1):
        ref = O.PSO(pb, TOTAL, lb, ub, logdim=[0] * len(lb), seed=SEED + g, store_f32=True).init().step(ITERS)
        idx, f = ref.reeval_topk(TOPK)
        for t in got[2 * g:2 * g + 2]:
            assert t[1] == (ref.gbest_f, ref.gbest_idx) and t[2] == idx and t[3] == f
    assert got[0][1] != got[2][1]  # the two swarms differ
