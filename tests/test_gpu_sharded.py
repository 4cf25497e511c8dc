"""Sharded MLMC over the CUDA library (needs a GB300): two ranks (processes,
gloo on CPU for the collective) both drive GpuLevelPairs on cuda:0, each on
its own block of every level's draws, and combine the FP64 level sums as
(sum, compensation) pairs in one all-reduce.  The ranks' kernels never wait
on one another (the only exchange is the host all-reduce between Alg. 1
iterations).  The result must equal the single-process GPU Alg. 1: same
levels and sample numbers, the same estimate to rounding of the summation
order, identical on both ranks."""
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS = 2e-3


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _levels():
    from gpu_common import small_level
    return [small_level(n=8 * 2**l, p=2, K=2, box=(0.375, 0.625, 0.375, 0.625), T=0.4,
                        qoi_box=(0.55, 0.8, 0.5, 0.75)) for l in range(4)]


def _draw(l, off, n):
    rng = np.random.default_rng(500 + l)
    return rng.uniform(-1, 1, size=(off + n, 2))[off:]


def _cost(hs):
    def c(l):
        w = hs[l].n_steps * (hs[l].info["n_free"] + hs[l].p * hs[l].info["n_R"])
        if l > 0:
            w += hs[l - 1].n_steps * (hs[l - 1].info["n_free"] + hs[l - 1].p * hs[l - 1].info["n_R"])
        return float(w)
    return c


def _alg1(lflts, ctx, hs, ev):
    from paper_2106_11117_gb300 import mlmc
    return mlmc.alg1(ev, _draw, EPS, _cost(hs), N_init=lambda l: 16, L_max=3)


def _worker(rank, world, port, out_q):
    import os
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    sys.path[:0] = [here, os.path.dirname(here)]
    import torch
    import torch.distributed as dist
    from paper_2106_11117_gb300 import lflts, mlmc
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ctx = lflts.Context(0)
        try:
            hs = [ctx.add_level(lv) for lv in _levels()]
            ev = mlmc.ShardedLevelPairs(mlmc.GpuLevelPairs(lflts, ctx, hs, precision=32), rank, world,
                                        mlmc.torch_allreduce())
            r = _alg1(lflts, ctx, hs, ev)
            out_q.put((rank, r.estimate, r.L, r.N, r.mse))
        finally:
            ctx.close()
    finally:
        dist.destroy_process_group()


def test_sharded_gpu_alg1_equals_single_process():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp
    from paper_2106_11117_gb300 import build, lflts, mlmc
    build.build()
    world = 2
    ctxm = mp.get_context("spawn")
    q = ctxm.Queue()
    port = _port()
    procs = [ctxm.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=600) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ctx = lflts.Context(0)
    try:
        hs = [ctx.add_level(lv) for lv in _levels()]
        ref = _alg1(lflts, ctx, hs, mlmc.GpuLevelPairs(lflts, ctx, hs, precision=32))
    finally:
        ctx.close()
    for rank, est, L, N, mse in res:
        assert L == ref.L and N == ref.N
        assert est == pytest.approx(ref.estimate, rel=1e-13, abs=1e-15)
        assert mse == pytest.approx(ref.mse, rel=1e-10)
    assert len({r[1] for r in res}) == 1   # every rank takes the same value
