"""CUDA-graph replay and autotuned launch shapes change nothing in the
results (needs a GB300)."""
import numpy as np
import pytest

from gpu_common import draws, small_level

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_11117_gb300 import build, lflts
    build.build()
    return lflts


def _jobs(lf, hs, xis, outs, prec):
    jobs = []
    for l in range(len(hs)):
        j = lf.PairJob()
        j.fine = hs[l].desc(prec)
        if l > 0:
            j.coarse = hs[l - 1].desc(prec)
            j.has_coarse = 1
        j.xi = xis[l].ctypes.data
        j.S = xis[l].shape[0]
        j.dQ, j.Qf, j.sums = (o.ctypes.data for o in outs[l])
        jobs.append(j)
    return jobs


@pytest.mark.parametrize("prec", [32, 64])
def test_graph_replay_and_autotune_bit_identical(lf, prec):
    levs = [small_level(n=8 * 2**l, p=2 + l, K=4, box=(0.375, 0.625, 0.375, 0.625)) for l in range(3)]
    xis = [draws(S, 4, seed=60 + S) for S in (64, 20, 9)]
    results = {}
    for graphs, tune in ((0, 0), (1, 0), (1, 1), (0, 1)):
        ctx = lf.Context(0)
        try:
            lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_GRAPHS, graphs)
            lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_AUTOTUNE, tune)
            hs = [ctx.add_level(l) for l in levs]
            runs = []
            for _ in range(3):  # first call captures, the next ones replay
                outs = [(np.zeros(x.shape[0]), np.zeros(x.shape[0]), np.zeros(4)) for x in xis]
                lf.lflts_run_pairs(ctx.h, _jobs(lf, hs, xis, outs, prec))
                runs.append(outs)
            st = lf.lflts_get_stats(ctx.h)
            if graphs:
                assert st["graph_launches"] >= 3 * 3
            else:
                assert st["graph_launches"] == 0
            if tune:
                assert st["tuned_shapes"] >= 3 and st["tune_launches"] > 0
        finally:
            ctx.close()
        for r in runs[1:]:
            for a, b in zip(r, runs[0]):
                for x, y in zip(a, b):
                    np.testing.assert_array_equal(x, y)
        results[(graphs, tune)] = runs[0]
    ref = results[(0, 0)]
    for key, r in results.items():
        for a, b in zip(r, ref):
            for x, y in zip(a, b):
                np.testing.assert_array_equal(x, y)


def test_unknown_option_rejected(lf):
    ctx = lf.Context(0)
    try:
        with pytest.raises(lf.LfltsError):
            lf.lflts_set_option(ctx.h, 99, 1)
    finally:
        ctx.close()


def _launches(lf, ctx):
    return lf.lflts_launch_count(ctx.h)


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("p", [2, 3, 5, 9])
@pytest.mark.parametrize("S", [40, 33, 130])
def test_fused_inner_kernel_bit_identical(lf, prec, p, S):
    """All p-1 inner substeps in one launch (R and the CTA's draws in shared
    memory) give the same values, bit for bit, as one launch per substep;
    ragged batches (S odd: one draw per thread) included, with a source.  The
    mesh keeps R small enough for shared memory (R, its coupling slots and
    their weights must fit in 200 KB)."""
    from workload import point_source
    lev = small_level(n=16 if p <= 5 else 8, p=p, K=4, box=(0.375, 0.625, 0.375, 0.625))
    nodes, w = point_source(lev["mesh"], (0.5, 0.52))
    lev = dict(lev, source={"nodes": nodes, "weights": w, "f0": 5.0, "t0": 0.2, "amp": 1.0})
    xi = draws(S, 4, seed=100 + p + S)
    out, launches = {}, {}
    for mode in (0, 2):
        ctx = lf.Context(0)
        try:
            lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_AUTOTUNE, 0)
            lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_FUSED_INNER, mode)
            h = ctx.add_level(lev)
            n0 = _launches(lf, ctx)
            out[mode] = ctx.solve(h, xi, precision=prec, state=True)
            launches[mode] = _launches(lf, ctx) - n0
            n_steps = h.n_steps
        finally:
            ctx.close()
    np.testing.assert_array_equal(out[2][1], out[0][1])
    np.testing.assert_array_equal(out[2][0], out[0][0])
    # one coarse and one fused launch per step instead of 1 + (p - 1)
    assert launches[0] - launches[2] == n_steps * (p - 2)


@pytest.mark.parametrize("prec", [32, 64])
def test_fused_inner_kernel_graded_lshape(lf, prec):
    """The graded L-shape (tiny R at the reentrant corner, p = 3 and 5, Ricker
    source): the fused path equals the per-substep path bit for bit, and the
    autotuner's choice (fused or not) changes nothing."""
    from workload import CONFIG_LSHAPE, lshape_level, xi_gaussian
    cfg = CONFIG_LSHAPE
    for l in (0, 1):
        lev = lshape_level(cfg, l, m0=6)
        lev = dict(lev, T=0.3, dt=0.3 / 400, n_steps=400)
        xi = xi_gaussian(cfg.seed, l, 24, cfg.K, cfg.sigma)
        out = {}
        for mode, tune in ((0, 0), (2, 0), (1, 1)):
            ctx = lf.Context(0)
            try:
                lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_AUTOTUNE, tune)
                lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_FUSED_INNER, mode)
                h = ctx.add_level(lev)
                out[(mode, tune)] = ctx.solve(h, xi, precision=prec, state=True)
            finally:
                ctx.close()
        for k, (Q, U) in out.items():
            np.testing.assert_array_equal(U, out[(0, 0)][1])
            np.testing.assert_array_equal(Q, out[(0, 0)][0])


def test_long_solves_launch_without_graph(lf):
    """Solves of more than 120,000 kernels launch directly instead of being
    captured into a graph; shorter solves on a stream are captured."""
    import torch
    lev = small_level(n=8, p=2, K=4, box=(0.375, 0.625, 0.375, 0.625))
    xi = torch.from_numpy(draws(8, 4, seed=5)).cuda()
    ctx = lf.Context(0)
    st = torch.cuda.Stream()
    try:
        lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_AUTOTUNE, 0)
        lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_FUSED_INNER, 0)
        h = ctx.add_level(lev)
        q = torch.zeros(8, dtype=torch.float64, device="cuda")
        for n_steps, graphed in ((1000, True), (61000, False)):
            d = h.desc(32)
            d.n_steps = n_steps
            g0 = lf.lflts_get_stats(ctx.h)["graph_launches"]
            lf.lflts_solve(ctx.h, d, xi, 8, q, None, lf.LFLTS_MEM_DEVICE, st.cuda_stream)
            st.synchronize()
            assert (lf.lflts_get_stats(ctx.h)["graph_launches"] - g0 == 1) == graphed
            assert torch.isfinite(q).all()
    finally:
        ctx.close()


def test_graph_cache_is_bounded(lf):
    """Solves with ever new batch sizes (as an adaptive Alg. 1 issues them)
    keep at most LFLTS_OPT_GRAPH_CACHE graphs per workspace: the least
    recently used are destroyed, a graph still held is replayed, and every
    result equals the run without graphs bit for bit."""
    import torch
    lev = small_level(n=12, p=3, K=4)
    st = torch.cuda.Stream()
    outs = {}
    for graphs in (0, 1):
        ctx = lf.Context(0)
        try:
            lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_AUTOTUNE, 0)
            lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_GRAPHS, graphs)
            lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_GRAPH_CACHE, 2)
            h = ctx.add_level(lev)
            d = h.desc(32)
            res = []
            for S in (8, 12, 16, 20, 16, 24, 8):
                xi = torch.from_numpy(draws(S, 4, seed=S)).cuda()
                Q = torch.zeros(S, dtype=torch.float64, device="cuda")
                lf.lflts_solve(ctx.h, d, xi, S, Q, None, lf.LFLTS_MEM_DEVICE, st.cuda_stream)
                st.synchronize()
                res.append(Q.cpu().numpy())
                assert lf.lflts_graph_cache_size(ctx.h) <= 2
            if graphs:
                assert lf.lflts_graph_cache_size(ctx.h) == 2
                assert lf.lflts_get_stats(ctx.h)["graph_launches"] == 7
            outs[graphs] = res
        finally:
            ctx.close()
    for a, b in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(a, b)
    with pytest.raises(lf.LfltsError):
        c2 = lf.Context(0)
        try:
            lf.lflts_set_option(c2.h, lf.LFLTS_OPT_GRAPH_CACHE, 0)
        finally:
            c2.close()
