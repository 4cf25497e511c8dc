"""Sharded MLMC on CPU ranks (gloo, world size 2): every rank evaluates its
block of each level's draws and the ranks combine only the FP64 level sums,
as (sum, compensation) pairs in one all-reduce; the result equals the
single-process Alg. 1."""
import math
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from test_mlmc_driver_host import SyntheticPairs, _draw


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_q):
    import torch.distributed as dist
    from paper_2106_11117_gb300 import mlmc
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ev = mlmc.ShardedLevelPairs(SyntheticPairs(), rank, world, mlmc.torch_allreduce())
        r = mlmc.alg1(ev, _draw, 2e-3, cost=lambda l: 4.0**l, N_init=lambda l: 33, alpha=2.0)
        out_q.put((rank, r.estimate, r.L, r.N, r.mse))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_sharded_alg1_equals_single_process(world):
    from paper_2106_11117_gb300 import mlmc
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = mlmc.alg1(SyntheticPairs(), _draw, 2e-3, cost=lambda l: 4.0**l, N_init=lambda l: 33, alpha=2.0)
    for rank, est, L, N, mse in res:
        assert L == ref.L and N == ref.N
        assert est == pytest.approx(ref.estimate, rel=1e-13)
        assert mse == pytest.approx(ref.mse, rel=1e-10)
    # all ranks agree exactly
    assert len({r[1] for r in res}) == 1


def test_shard_blocks_cover_all_draws():
    from paper_2106_11117_gb300 import mlmc

    class Rec:
        def __init__(self):
            self.seen = {}

        def run(self, req):
            for l, x in req.items():
                self.seen.setdefault(l, []).append(x.copy())
            return {l: (x[:, 0], [float(x[:, 0].sum()), 0.0, 0.0, 0.0]) for l, x in req.items()}

    xi = np.arange(21, dtype=float).reshape(7, 3)
    recs = [Rec() for _ in range(3)]
    for r in range(3):
        mlmc.ShardedLevelPairs(recs[r], r, 3, lambda a: a).run({0: xi})
    rows = np.concatenate([recs[r].seen[0][0] for r in range(3)])
    np.testing.assert_array_equal(rows, xi)


def test_pairs_combine_exactly_in_rank_order():
    """The all-reduce adds arrays that are zero outside each rank's slot, so
    every pair arrives unchanged; the level sum is the correctly rounded sum
    of all pairs (math.fsum), which a plain sum of the rank values misses."""
    from paper_2106_11117_gb300 import mlmc

    vals = [1e16, 1.0, -1e16, 1.0]     # plain left-to-right sum: 1.0 (1e16 + 1 rounds)

    class One:
        def __init__(self, v):
            self.v = v

        def run(self, req):
            return {l: (np.zeros(1), [self.v, 0.0, 0.0, 0.0]) for l in req}

    bufs = {}

    def red_for(r):
        def red(a):
            bufs[r] = a
            return sum(bufs.get(k, np.zeros_like(a)) for k in range(4))
        return red

    outs = []
    for r in range(4):   # the last rank sees every slot filled
        outs.append(mlmc.ShardedLevelPairs(One(vals[r]), r, 4, red_for(r)).run({0: np.zeros((4, 1))}))
    assert outs[-1][0][1][0] == 2.0
    naive = 0.0
    for v in vals:
        naive += v
    assert math.fsum(vals) == 2.0 and naive == 1.0
