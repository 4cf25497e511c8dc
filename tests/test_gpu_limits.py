"""Batch-size limits of the CUDA path (needs a GB300).

The largest batch a solve takes is 65,535 slabs of 32 draws (2,097,120
draws: the launch grid's y extent).  That batch is solved on a small
refined mesh in FP32 and FP64; sampled draws (the first ones, the last
slab, the very last draw) are compared with the FP64 oracle one by one and,
bit for bit, with the same draws solved as a batch of their own.  One draw
more, an empty batch, and a merged level-pair batch over the limit are
refused with LFLTS_ERR_ARG before anything runs.

Tolerances as in the other parity tests: QoI 1e-12 (FP64), 1e-5 (FP32)
of the sampled draws' largest |Q|."""
import numpy as np
import pytest

from gpu_common import draws, oracle_run, rel_err, small_level

pytestmark = pytest.mark.gpu

S_MAX = 65535 * 32
TOL_Q = {64: 1e-12, 32: 1e-5}


@pytest.fixture(scope="module")
def lf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_11117_gb300 import build, lflts
    build.build()
    return lflts


@pytest.fixture(scope="module")
def ctx(lf):
    c = lf.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def level():
    # 137 nodes, 105 of them in P, 15 outer steps
    return small_level(n=8, p=2, K=2)


@pytest.mark.parametrize("precision", [32, 64])
def test_largest_batch_matches_oracle(lf, ctx, level, precision):
    h = ctx.add_level(level)
    xi = draws(S_MAX, 2, seed=2106)
    Q = ctx.solve(h, xi, precision=precision)
    assert Q.shape == (S_MAX,) and np.isfinite(Q).all()
    pick = np.array([0, 1, 31, 32, 1234567, S_MAX - 33, S_MAX - 32, S_MAX - 2, S_MAX - 1])
    Qo, _ = oracle_run(level, xi[pick])
    assert rel_err(Q[pick], Qo) <= TOL_Q[precision], rel_err(Q[pick], Qo)
    np.testing.assert_array_equal(Q[pick], ctx.solve(h, xi[pick], precision=precision))


def test_batches_beyond_the_limit_are_refused(lf, ctx, level):
    h = ctx.add_level(level)
    xi = np.zeros((S_MAX + 1, 2))
    Q = np.zeros(S_MAX + 1)
    for S in (0, S_MAX + 1):
        with pytest.raises(lf.LfltsError) as e:
            lf.lflts_solve(ctx.h, h.desc(32), xi, S, Q)
        assert e.value.code == lf.LFLTS_ERR_ARG
        assert "S must be in [1, 2097120]" in str(e.value)
    # two jobs on the same mesh merge into one batch of S_MAX + 1 draws
    jobs = []
    dQ = [np.zeros(S_MAX), np.zeros(1)]
    for k, S in enumerate((S_MAX, 1)):
        j = lf.PairJob()
        j.fine, j.has_coarse = h.desc(32), 0
        j.xi, j.S, j.dQ = xi.ctypes.data, S, dQ[k].ctypes.data
        jobs.append(j)
    with pytest.raises(lf.LfltsError) as e:
        lf.lflts_run_pairs(ctx.h, jobs, lf.LFLTS_MEM_HOST, None)
    assert e.value.code == lf.LFLTS_ERR_ARG
    assert "merged batch larger than 2097120" in str(e.value)
