"""Ragged batches (needs a GB300): lflts_run_pairs merges solves that differ
only in (dt, n_steps) into one batch per mesh in which every draw steps with
its own dt for its own count.  Each draw's QoI must equal the one from a
batch of its own segment alone (uniform path): to 1e-12 of the QoI scale in
FP64 (the draw's dt^2 enters through its edge weights instead of the step
constants, a different rounding order) and 1e-5 in FP32.  Segment sizes are
not multiples of the draws per thread, so segment ends fall inside vectors."""
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


def _level_with_source(p):
    from workload import point_source
    lev = small_level(n=12, p=p, K=4, T=0.5)
    nodes, w = point_source(lev["mesh"], (0.5, 0.47))
    return dict(lev, source={"nodes": nodes, "weights": w, "f0": 6.0, "t0": 0.2, "amp": 2.0})


# The jobs hold raw pointers: every array they point to must outlive the call.
_ALIVE = []


def _job(lf, h, prec, dt, n, x, outs):
    j = lf.PairJob()
    j.fine = h.desc(prec)
    j.fine.dt, j.fine.n_steps = dt, n
    j.xi, j.S = x.ctypes.data, x.shape[0]
    dQ, Qf, sums = np.zeros(x.shape[0]), np.zeros(x.shape[0]), np.zeros(4)
    j.dQ, j.Qf, j.sums = dQ.ctypes.data, Qf.ctypes.data, sums.ctypes.data
    _ALIVE.append((x, dQ, sums))
    outs.append(Qf)
    return j


@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 1e-5)])
@pytest.mark.parametrize("p", [1, 3])
def test_ragged_batch_matches_separate_batches(lf, prec, tol, p):
    lev = _level_with_source(p)
    T, n0 = lev["T"], lev["n_steps"]
    steps = [n0, int(round(1.25 * n0)), int(round(1.6 * n0)), 2 * n0]
    sizes = [5, 8, 3, 6]
    xis = [draws(S, 4, seed=40 + k) for k, S in enumerate(sizes)]
    ref, got = {}, {}
    for fused in (0, 2):
        ctx = lf.Context(0)
        try:
            lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_AUTOTUNE, 0)
            lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_FUSED_INNER, fused)
            h = ctx.add_level(lev)
            outs = []
            jobs = [_job(lf, h, prec, T / n, n, x, outs) for n, x in zip(steps, xis)]
            lf.lflts_run_pairs(ctx.h, jobs)          # one ragged batch of 22 draws
            got[fused] = [o.copy() for o in outs]
            sep = []
            for n, x in zip(steps, xis):             # each segment alone: uniform batches
                o = []
                lf.lflts_run_pairs(ctx.h, [_job(lf, h, prec, T / n, n, x, o)])
                sep.append(o[0])
            ref[fused] = sep
        finally:
            ctx.close()
    scale = max(np.abs(q).max() for q in ref[0])
    assert scale > 1e-4
    for a, b in zip(got[0], ref[0]):
        assert np.abs(a - b).max() <= tol * scale
    # the fused inner kernel narrows to the same draws, bit for bit
    for a, b in zip(got[2], got[0]):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(ref[2], ref[0]):
        np.testing.assert_array_equal(a, b)


def test_ragged_segments_ordered_by_steps(lf):
    """Jobs given in any order of step counts give the same per-draw QoI
    (segments are sorted inside the library); the merged batch is captured
    once and replayed on a second call with the same segments."""
    import torch
    lev = _level_with_source(3)
    T, n0 = lev["T"], lev["n_steps"]
    steps = [int(round(1.3 * n0)), n0, 2 * n0]
    xis = [draws(S, 4, seed=70 + S) for S in (4, 7, 2)]
    ctx = lf.Context(0)
    try:
        h = ctx.add_level(lev)
        res = []
        for order in ([0, 1, 2], [2, 0, 1], [2, 0, 1]):
            outs = []
            jobs = [_job(lf, h, 64, T / steps[k], steps[k], xis[k], outs) for k in order]
            st = torch.cuda.Stream()
            g0 = lf.lflts_get_stats(ctx.h)["graph_launches"]
            lf.lflts_run_pairs(ctx.h, jobs, lf.LFLTS_MEM_HOST, st.cuda_stream)
            assert lf.lflts_get_stats(ctx.h)["graph_launches"] - g0 == 1
            res.append({k: o for k, o in zip(order, outs)})
        for r in res[1:]:
            for k in range(3):
                np.testing.assert_array_equal(r[k], res[0][k])
    finally:
        ctx.close()
