"""Alg. 1 on the GPU against the oracle's Alg. 1 on the same draws (needs a GB300).

* plain per-draw FP64 path: same levels and sample numbers as the oracle,
  estimate within 1e-10 relative;
* batched FP32 path: MLMC estimate within 0.1 eps of the FP64 one."""
import numpy as np
import pytest

from gpu_common import small_level

pytestmark = pytest.mark.gpu

EPS = 2e-3


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_11117_gb300 import build, lflts
    build.build()
    levels = [small_level(n=8 * 2**l, p=2, K=2, box=(0.375, 0.625, 0.375, 0.625), T=0.4,
                          qoi_box=(0.55, 0.8, 0.5, 0.75)) for l in range(4)]
    ctx = lflts.Context(0)
    hs = [ctx.add_level(l) for l in levels]
    yield lflts, ctx, hs, levels
    ctx.close()


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


def test_plain_fp64_alg1_matches_oracle(setup):
    from oracle import mlmc as omlmc
    from oracle.lts import solve_qoi
    from paper_2106_11117_gb300 import mlmc
    lflts, ctx, hs, levels = setup
    cost = _cost(hs)
    ev = mlmc.GpuLevelPairs(lflts, ctx, hs, plain=True)
    res = mlmc.alg1(ev, _draw, EPS, cost, N_init=lambda l: 16, L_max=3)

    def sample(l, off, n):
        xi = _draw(l, off, n)
        out = []
        for x in xi:
            q = solve_qoi(levels[l], x)
            out.append(q - solve_qoi(levels[l - 1], x) if l > 0 else q)
        return np.array(out)

    ref = omlmc.alg1(sample, EPS, cost, N_init=lambda l: 16, alpha=2.0, L_max=3)
    assert res.L == ref["L"] and res.N == ref["N"]
    assert res.estimate == pytest.approx(ref["estimate"], rel=1e-10)
    assert ev.calls == sum(res.N)  # one draw per call


def test_batched_fp32_alg1_within_tenth_eps(setup):
    from paper_2106_11117_gb300 import mlmc
    lflts, ctx, hs, levels = setup
    cost = _cost(hs)
    r64 = mlmc.alg1(mlmc.GpuLevelPairs(lflts, ctx, hs, plain=True), _draw, EPS, cost,
                    N_init=lambda l: 16, L_max=3)
    ev32 = mlmc.GpuLevelPairs(lflts, ctx, hs, precision=32)
    r32 = mlmc.alg1(ev32, _draw, EPS, cost, N_init=lambda l: 16, L_max=3)
    assert r32.L == r64.L
    assert abs(r32.estimate - r64.estimate) <= 0.1 * EPS
    assert r32.mse <= 1.05 * EPS**2
    assert ev32.calls == r32.iterations  # all levels of an iteration in one call
