"""Host logic of the multi-process benchmark path on CPU ranks (gloo, world size 2).

The GPU path shards the batched workload by window across ranks with no data-path
collective; the only cross-rank steps are the barrier around the timed region and the
max-over-ranks of the elapsed time, both exercised here without a GPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    bench._barrier(world)
    q.put((rank, bench._max_over_ranks(1.5 + rank, world)))
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 2.5, 1: 2.5}


def test_window_shards_are_disjoint_streams():
    import bench

    shards = [bench.batch_windows("batch512", r)[1] for r in range(4)]
    ids = [{w["stream_id"] for w in sh} for sh in shards]
    for a in range(4):
        assert len(ids[a]) == len(shards[a])
        for b in range(a + 1, 4):
            assert not ids[a] & ids[b]
    # every rank calibrates the same layout (weak scaling): only the Philox stream words differ
    for sh in shards[1:]:
        assert [(w["T"], w["L"], w["particles"]) for w in sh] == [(w["T"], w["L"], w["particles"]) for w in shards[0]]


def test_topk_launch_count():
    import bench

    assert bench.topk_launches(4096, 32) == 1
    assert bench.topk_launches(1 << 20, 32) == 3
    assert bench.topk_launches(1 << 20, 1024) == 5


@pytest.mark.timeout(600)
def test_reference_arm_two_ranks_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--gpus", "2", "--impl", "reference",
           "--workload", "plain64", "--steps", "1", "--warmup", "3", "--ref-units", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=540, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["value"] > 0
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["cpu_baseline"]["kind"] == "oracle"


@pytest.mark.timeout(600)
def test_bench_starts_its_own_ranks_for_several_gpus():
    """`bench.py --gpus 2` without an outer launcher starts two ranks itself and prints one line
    with n_gpus 2."""
    cmd = [sys.executable, "bench.py", "--gpus", "2", "--impl", "reference", "--workload", "plain64", "--steps", "1",
           "--warmup", "3", "--ref-units", "1"]
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    env["OMP_NUM_THREADS"] = "1"
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=540, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2


def test_bench_refuses_a_rank_count_that_differs_from_gpus():
    env = dict(os.environ, WORLD_SIZE="2", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, "bench.py", "--gpus", "4", "--impl", "reference"], cwd=ROOT,
                       capture_output=True, text=True, timeout=120, env=env)
    assert r.returncode != 0 and "WORLD_SIZE" in r.stderr
