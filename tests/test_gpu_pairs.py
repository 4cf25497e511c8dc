"""Paired inner substeps (needs a GB300): two substeps of Alg. 2 per launch,
block by block (square cells of R plus a halo of their P neighbours, r_{m+1}
exchanged in shared memory).  The values must equal those of one launch per
substep bit for bit -- same couplings, same order, same roundings -- for
every block size (small blocks put most couplings across block borders),
FP32 and FP64, even and odd numbers of substeps, with a point source; and
on a full-size mesh of the benchmark hierarchy they must agree with the FP64
oracle over a short horizon."""
import numpy as np
import pytest

from gpu_common import draws, oracle_run, rel_err, small_level

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_11117_gb300 import build, lflts
    build.build()
    return lflts


def _solve(lf, lev, xi, prec, pair_mode, block=144, autotune=0):
    ctx = lf.Context(0)
    try:
        lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_AUTOTUNE, autotune)
        lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_FUSED_INNER, 0)
        lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_TILED_INNER, 0)
        lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_PAIRED_INNER, pair_mode)
        lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_PAIR_BLOCK, block)
        h = ctx.add_level(lev)
        n0 = lf.lflts_launch_count(ctx.h)
        Q, U = ctx.solve(h, xi, precision=prec, state=True)
        return Q, U, lf.lflts_launch_count(ctx.h) - n0, h
    finally:
        ctx.close()


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("p", [3, 4, 5, 8, 9])
def test_paired_substeps_bit_identical(lf, prec, p):
    from workload import point_source
    lev = small_level(n=16, p=p, K=4, box=(0.3, 0.7, 0.3, 0.7))
    nodes, w = point_source(lev["mesh"], (0.5, 0.52))
    lev = dict(lev, source={"nodes": nodes, "weights": w, "f0": 5.0, "t0": 0.2, "amp": 1.0})
    # 40 draws: one full slab of 32 and a partial one
    xi = draws(40, 4, seed=300 + p)
    Q0, U0, l0, h = _solve(lf, lev, xi, prec, 0)
    assert h.info["n_R"] > 256
    # modes 2, 3, 4: 4 (FP32) or 2 (FP64), 2 and 1 draws per thread
    for mode, block in ((2, 16), (2, 64), (2, 196), (3, 64), (4, 64), (4, 196)):
        Q, U, l1, _ = _solve(lf, lev, xi, prec, mode, block)
        np.testing.assert_array_equal(U, U0)
        np.testing.assert_array_equal(Q, Q0)
        # p - 1 substeps in p // 2 launches per step
        assert l0 - l1 == h.n_steps * ((p - 1) - p // 2)


def test_paired_substeps_fans_and_autotune(lf):
    """A mesh whose refined box closes with fan triangles (nodes with more
    than four couplings, slots beyond the fourth) and the autotuner's pick:
    every path gives the same values."""
    lev = small_level(n=20, p=4, K=4, box=(0.3, 0.62, 0.33, 0.71))
    xi = draws(24, 4, seed=19)
    Q0, U0, _, _ = _solve(lf, lev, xi, 32, 0)
    for mode, block, tune in ((2, 16, 0), (3, 32, 0), (4, 32, 0), (1, 196, 1), (2, 196, 1)):
        Q, U, _, _ = _solve(lf, lev, xi, 32, mode, block, tune)
        np.testing.assert_array_equal(U, U0)
        np.testing.assert_array_equal(Q, Q0)


def test_paired_substeps_fullsize_mesh_against_oracle(lf):
    """Level 2 of the benchmark hierarchy (512^2 base cells, 459 k free
    nodes, |R| = 202 k, p = 8): a few outer steps of 8 draws with the paired
    substeps against the FP64 oracle (FP32 path, 1e-5 of the state's scale)
    and against one launch per substep (bit for bit)."""
    from workload import CONFIG_BATCHED, level_problem, xi_uniform
    lev = level_problem(CONFIG_BATCHED, 2)
    lev = dict(lev, n_steps=6)
    xi = xi_uniform(CONFIG_BATCHED.seed, 2, 8, CONFIG_BATCHED.K)
    Qp, Up, _, h = _solve(lf, lev, xi, 32, 2)
    assert h.info["n_R"] > 100000
    Q0, U0, _, _ = _solve(lf, lev, xi, 32, 0)
    np.testing.assert_array_equal(Up, U0)
    Qo, Uo = oracle_run(lev, xi[:2])
    assert rel_err(Up[:, :2], Uo) <= 1e-5


def test_forced_pairs_respect_the_minimum_R(lf):
    """LFLTS_OPT_PAIR_MIN_R: forced paired substeps only on meshes whose R
    has at least that many nodes; the values stay the same either way."""
    lev = small_level(n=16, p=5, K=4, box=(0.3, 0.7, 0.3, 0.7))
    xi = draws(8, 4, seed=5)
    Q0, U0, l0, h = _solve(lf, lev, xi, 32, 0)
    n_R = h.info["n_R"]
    for min_r, paired in ((n_R + 1, False), (n_R, True)):
        ctx = lf.Context(0)
        try:
            lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_AUTOTUNE, 0)
            lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_FUSED_INNER, 0)
            lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_TILED_INNER, 0)
            lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_PAIRED_INNER, 2)
            lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_PAIR_MIN_R, min_r)
            hh = ctx.add_level(lev)
            n0 = lf.lflts_launch_count(ctx.h)
            Q, U = ctx.solve(hh, xi, precision=32, state=True)
            launches = lf.lflts_launch_count(ctx.h) - n0
        finally:
            ctx.close()
        np.testing.assert_array_equal(U, U0)
        assert (launches < l0) == paired
