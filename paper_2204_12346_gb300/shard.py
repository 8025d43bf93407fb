"""One window's FP32 swarm split by particle across the ranks of a process group.

Sec. 3.3: every particle's trajectory and loss are computed independently; the synchronous
global best is the only coupling between particles.  Rank r holds the contiguous particles
offset_r .. offset_r + count_r - 1 (counts differ by at most one).  After the initialisation
and after every iteration the ranks agree on the particle with the lowest personal-best loss
(lowest global index on ties) through one all-gather of every rank's 64-bit key and position:
(8 + 4P) bytes from each rank per iteration, one collective and one wait.  With every shard numbering
its particles globally (sird_pso_set_shard), the shards together follow the unsharded swarm
exactly.  The final answer is the FP64 re-evaluation of the swarm's k best personal bests,
gathered from the shards.

A shard is any object with init(), step(n), shard_best() -> (loss, index, z),
set_gbest(z, loss, index), topk(k, with_index=True) -> (theta [k, P], loss [k], index [k])
and eval64(theta [k, P]) -> FP64 losses: sird.Calibrator (after set_shard) on a GPU.

Failure detection: the exchange is the only point where ranks wait on one another, and it runs
on the host between launches.  A rank that leaves (between steps, with nothing in flight) makes
the others' next exchange fail -- the backend reports the closed connection, or the process
group's timeout ends the wait -- and ShardedSwarm raises ShardFailure naming the exchange.
"""
from __future__ import annotations

import numpy as np


def shard_range(total: int, rank: int, world: int) -> tuple[int, int]:
    """(offset, count) of rank's particles: contiguous, the first total % world ranks one more."""
    base, extra = divmod(int(total), int(world))
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def shard_offsets(total: int, world: int) -> list[int]:
    return [shard_range(total, r, world)[0] for r in range(world)] + [int(total)]


def owner_of(index: int, offsets: list[int]) -> int:
    """Rank holding global particle `index` (offsets as from shard_offsets)."""
    for r in range(len(offsets) - 1):
        if offsets[r] <= index < offsets[r + 1]:
            return r
    raise ValueError(f"particle {index} outside the swarm")


def best_key(loss: float, index: int) -> int:
    """Signed 64-bit key ordered as (loss, index): the FP32 loss's bits mapped to an unsigned
    integer of the same order (NaN counts as +inf) in the high word, the index in the low word,
    and the top bit flipped so that signed order equals that unsigned order."""
    f = np.float32(loss)
    if np.isnan(f):
        f = np.float32(np.inf)
    bits = int(np.array([f], dtype=np.float32).view(np.uint32)[0])
    ordered = (~bits & 0xFFFFFFFF) if bits & 0x80000000 else (bits | 0x80000000)
    u = (ordered << 32) | (int(index) & 0xFFFFFFFF)
    return u - (1 << 63)  # = u xor 2^63, read as a signed value


def key_parts(key: int) -> tuple[float, int]:
    """(loss, index) of a key from best_key."""
    u = int(key) + (1 << 63)
    ordered, index = u >> 32, u & 0xFFFFFFFF
    bits = (ordered & 0x7FFFFFFF) if ordered & 0x80000000 else (~ordered & 0xFFFFFFFF)
    return float(np.array([bits], dtype=np.uint32).view(np.float32)[0]), int(index)


def exchange_best(loss: float, index: int, z, offsets: list[int], group=None, device=None):
    """The swarm's global best from every rank's shard best: one all-gather of each rank's record
    (its 64-bit key, then its position as FP32 bits two to a 64-bit word), then the record with
    the lowest key -- the same on every rank, with one collective and one wait per exchange.
    Returns (loss, index, z [P] float32)."""
    import torch
    import torch.distributed as dist

    zf = np.ascontiguousarray(np.asarray(z, dtype=np.float32)).ravel()
    P = zf.size
    words = (P + 1) // 2
    rec = np.zeros(1 + words, dtype=np.int64)
    rec[0] = best_key(loss, index)
    zpad = np.zeros(2 * words, dtype=np.float32)
    zpad[:P] = zf
    rec[1:] = zpad.view(np.int64)
    mine = torch.from_numpy(rec).to(device)
    parts = [torch.empty_like(mine) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, mine, group=group)
    recs = torch.stack(parts).cpu().numpy()
    win = int(np.argmin(recs[:, 0]))  # keys are distinct: every particle index is held once
    gloss, gidx = key_parts(int(recs[win, 0]))
    if owner_of(gidx, offsets) != win:
        raise RuntimeError(f"shard exchange: particle {gidx} reported by rank {win}, which does not hold it")
    return gloss, gidx, recs[win, 1:].copy().view(np.float32)[:P].copy()


class ShardFailure(RuntimeError):
    """The exchange after `step` completed iterations (0: after the initialisation) failed,
    e.g. because another rank left the process group."""

    def __init__(self, step: int, cause: BaseException):
        super().__init__(f"shard exchange after iteration {step} failed: {cause}")
        self.step = int(step)


class ShardedSwarm:
    """Runs a sharded swarm: shard is this rank's part (see the module docstring), offsets the
    first particle of every rank's part plus the total (shard_offsets)."""

    def __init__(self, shard, offsets: list[int], group=None, device=None):
        self.shard = shard
        self.offsets = list(offsets)
        self.group = group
        self.device = device
        self.gbest = None

    def _exchange(self, step: int):
        loss, index, z = self.shard.shard_best()
        try:
            self.gbest = exchange_best(loss, index, z, self.offsets, self.group, self.device)
        except RuntimeError as e:  # the backends raise RuntimeError subclasses for lost peers and timeouts
            raise ShardFailure(step, e) from e
        self.shard.set_gbest(self.gbest[2], self.gbest[0], self.gbest[1])

    def run(self, iters: int):
        """Initialisation and iters synchronous iterations; returns the global best (loss,
        index, z) after the last.  Raises ShardFailure if an exchange fails."""
        self.shard.init()
        self._exchange(0)
        for t in range(int(iters)):
            self.shard.step(1)
            self._exchange(t + 1)
        return self.gbest

    def result(self, k: int) -> dict:
        """FP64 re-evaluation of the swarm's k best personal bests (best FP32 loss first, lowest
        index on ties), gathered from all shards; the reported point is the FP64 argmin (lowest
        index on ties), as in the unsharded re-evaluation."""
        import torch
        import torch.distributed as dist

        local = min(int(k), self.offsets[dist.get_rank(self.group) + 1] - self.offsets[dist.get_rank(self.group)])
        th, lo, idx = self.shard.topk(local, with_index=True)
        world = dist.get_world_size(self.group)
        rows = np.column_stack([lo, idx.astype(np.float64), th])  # index < 2^26: exact in FP64
        n = torch.tensor([rows.shape[0]], dtype=torch.int64, device=self.device)
        sizes = [torch.zeros_like(n) for _ in range(world)]
        dist.all_gather(sizes, n, group=self.group)
        width = rows.shape[1]
        cap = int(max(int(s.item()) for s in sizes))
        mine = torch.full((cap, width), np.inf, dtype=torch.float64, device=self.device)
        mine[: rows.shape[0]] = torch.from_numpy(rows).to(self.device)
        parts = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(parts, mine, group=self.group)
        allrows = np.concatenate([p.cpu().numpy()[: int(s.item())] for p, s in zip(parts, sizes)])
        order = np.lexsort((allrows[:, 1], allrows[:, 0]))[: int(k)]
        top = allrows[order]
        f64 = np.asarray(self.shard.eval64(top[:, 2:]), dtype=np.float64)
        f64 = np.where(np.isnan(f64), np.inf, f64)
        best = int(np.lexsort((top[:, 1], f64))[0])
        return {"theta": top[best, 2:].copy(), "loss": float(f64[best]), "loss_search": float(top[best, 0]),
                "index": int(top[best, 1]), "count": int(len(top))}
