"""The coarse launch that forms its coupling weights from xi and the field
basis (k_coarse_rc, LFLTS_OPT_COARSE_RC, off by default: measured 3x slower
on GB300) instead of reading the stored per-draw weights (needs a GB300): the same operations in the same order as
the weight kernel, so the states and QoIs equal those of k_coarse bit for
bit, FP32 and FP64, p = 1..8, with and without a point source; and on a
full-size mesh of the benchmark hierarchy the FP32 path agrees with the FP64
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


def _solve(lf, lev, xi, prec, rc, autotune=0):
    ctx = lf.Context(0)
    try:
        lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_AUTOTUNE, autotune)
        lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_COARSE_RC, rc)
        h = ctx.add_level(lev)
        Q, U = ctx.solve(h, xi, precision=prec, state=True)
        return Q, U
    finally:
        ctx.close()


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("p,K", [(1, 4), (3, 8), (5, 5), (8, 12)])
@pytest.mark.parametrize("source", [False, True])
def test_coarse_weights_formed_in_the_kernel_are_bit_identical(lf, prec, p, K, source):
    from workload import point_source
    lev = small_level(n=16, p=p, K=K, box=(0.3, 0.7, 0.3, 0.7))
    if source:
        nodes, w = point_source(lev["mesh"], (0.5, 0.52))
        lev = dict(lev, source={"nodes": nodes, "weights": w, "f0": 5.0, "t0": 0.2, "amp": 1.0})
    xi = draws(36, K, seed=40 + p)
    Q0, U0 = _solve(lf, lev, xi, prec, 0)
    Q1, U1 = _solve(lf, lev, xi, prec, 2)
    np.testing.assert_array_equal(U1, U0)
    np.testing.assert_array_equal(Q1, Q0)
    Q2, U2 = _solve(lf, lev, xi, prec, 1, autotune=1)  # whatever the autotuner keeps
    np.testing.assert_array_equal(U2, U0)


def test_coarse_weights_formed_in_the_kernel_fullsize_against_oracle(lf):
    """Level 2 of the benchmark hierarchy (459 k free nodes), 8 draws, 6
    outer steps: FP32 against the FP64 oracle (1e-5 of the state's scale)."""
    from workload import CONFIG_BATCHED, level_problem, xi_uniform
    lev = dict(level_problem(CONFIG_BATCHED, 2), n_steps=6)
    xi = xi_uniform(CONFIG_BATCHED.seed, 2, 8, CONFIG_BATCHED.K)
    Q, U = _solve(lf, lev, xi, 32, 2)
    Q0, U0 = _solve(lf, lev, xi, 32, 0)
    np.testing.assert_array_equal(U, U0)
    Qo, Uo = oracle_run(lev, xi[:2])
    assert rel_err(U[:, :2], Uo) <= 1e-5
