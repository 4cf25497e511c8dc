"""The tiled inner kernel (needs a GB300): all p-1 substeps of Alg. 2 in one
launch, tile by tile (a compact core of R plus p-1 layers of P nodes, the
halo recomputed by neighbouring tiles), node state in registers.  Its values
must equal those of one launch per substep bit for bit -- same slots, same
order, same roundings -- for every tile size (small capacities force many
tiles and halos that cross tile borders), FP32 and FP64,
p = 2..9, with a point source; and on a full-size mesh of the benchmark
hierarchy it must agree with the FP64 oracle over a short horizon."""
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


def _solve(lf, lev, xi, prec, tile_mode, cap=0, autotune=0):
    ctx = lf.Context(0)
    try:
        lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_AUTOTUNE, autotune)
        lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_FUSED_INNER, 0)
        lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_TILED_INNER, tile_mode)
        lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_TILE_CAP, cap)
        h = ctx.add_level(lev)
        n0 = lf.lflts_launch_count(ctx.h)
        Q, U = ctx.solve(h, xi, precision=prec, state=True)
        return Q, U, lf.lflts_launch_count(ctx.h) - n0, h
    finally:
        ctx.close()


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("p", [2, 3, 5, 9])
def test_tiled_inner_kernel_bit_identical(lf, prec, p):
    from workload import point_source
    lev = small_level(n=16 if p <= 5 else 8, p=p, K=4, box=(0.375, 0.625, 0.375, 0.625))
    nodes, w = point_source(lev["mesh"], (0.5, 0.52))
    lev = dict(lev, source={"nodes": nodes, "weights": w, "f0": 5.0, "t0": 0.2, "amp": 1.0})
    xi = draws(40, 4, seed=200 + p)
    Q0, U0, l0, h = _solve(lf, lev, xi, prec, 0)
    assert h.info["n_R"] > 64
    modes = (2,)
    # capacities that still hold a core plus p - 2 computed layers (smaller
    # ones make no plan and the per-substep path runs)
    caps = {2: (0, 64, 16), 3: (0, 64, 16), 5: (0, 200, 64), 9: (0, 600)}[p]
    for mode in modes:
        for cap in caps:
            Q, U, l1, _ = _solve(lf, lev, xi, prec, mode, cap)
            np.testing.assert_array_equal(U, U0)
            np.testing.assert_array_equal(Q, Q0)
            # one coarse and one tiled launch per step instead of 1 + (p - 1)
            assert l0 - l1 == h.n_steps * (p - 2)


def test_tiled_inner_kernel_fans_and_autotune(lf):
    """A mesh whose refined box closes with fan triangles (nodes with more
    than four couplings, slots beyond the fourth) and the autotuner's pick:
    every path gives the same values."""
    lev = small_level(n=20, p=4, K=4, box=(0.3, 0.62, 0.33, 0.71))
    xi = draws(24, 4, seed=9)
    Q0, U0, _, _ = _solve(lf, lev, xi, 32, 0)
    for mode, cap, tune in ((2, 40, 0), (1, 0, 1), (2, 0, 1)):
        Q, U, _, _ = _solve(lf, lev, xi, 32, mode, cap, tune)
        np.testing.assert_array_equal(U, U0)
        np.testing.assert_array_equal(Q, Q0)


def test_tiled_inner_kernel_fullsize_mesh_against_oracle(lf):
    """Level 2 of the benchmark hierarchy (512^2 base cells, 459 k free
    nodes, |R| = 202 k, p = 8): a few outer steps of 8 draws with the tiled
    kernel against the FP64 oracle (FP32 path, 1e-5 of the state's scale)
    and against the per-substep path (bit for bit)."""
    from workload import CONFIG_BATCHED, level_problem, xi_uniform
    lev = level_problem(CONFIG_BATCHED, 2)
    lev = dict(lev, n_steps=6)
    xi = xi_uniform(CONFIG_BATCHED.seed, 2, 8, CONFIG_BATCHED.K)
    Qt, Ut, _, h = _solve(lf, lev, xi, 32, 2)
    assert h.info["n_R"] > 100000
    Q0, U0, _, _ = _solve(lf, lev, xi, 32, 0)
    np.testing.assert_array_equal(Ut, U0)
    Qo, Uo = oracle_run(lev, xi[:2])
    assert rel_err(Ut[:, :2], Uo) <= 1e-5
