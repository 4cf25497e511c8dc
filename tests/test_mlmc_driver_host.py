"""Host logic of the MLMC driver (Alg. 1) on the CPU: its formulas and its
adaptive loop agree with the oracle's independent implementation."""
import math

import numpy as np
import pytest

from oracle import mlmc as omlmc
from paper_2106_11117_gb300 import mlmc


def test_formulas_match_oracle():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(50) * 1e-3 + 2e-2
    s1, s2 = math.fsum(x), math.fsum(x * x)
    assert mlmc.level_variance(s1, s2, 50) == omlmc.variance(s1, s2, 50)
    assert mlmc.estimator([s1, 0.5], [50, 7]) == omlmc.estimator([s1, 0.5], [50, 7])
    V, C = [1e-4, 3e-6, 2e-7], [1.0, 8.0, 64.0]
    assert mlmc.optimal_samples(V, C, 1e-3) == omlmc.optimal_N(V, C, 1e-3)
    assert mlmc.bias(0.012, 2.0) == omlmc.bias_estimate(0.012, 2.0)


class SyntheticPairs:
    """dQ_l(xi) = a 4^-l + s 2^-l xi_0 (xi_0 ~ U(-1,1)): deterministic in the draw."""

    def __init__(self, a=0.3, s=0.2):
        self.a, self.s = a, s

    def dq(self, l, xi):
        return self.a * 4.0 ** (-l) + self.s * 2.0 ** (-l) * xi[:, 0]

    def run(self, requests):
        out = {}
        for l, xi in requests.items():
            d = self.dq(l, xi)
            out[l] = (d, [math.fsum(d), math.fsum(d * d), 0.0, 0.0])
        return out


def _draw(l, off, n):
    rng = np.random.default_rng(1000 + l)
    return rng.uniform(-1, 1, size=(off + n, 2))[off:]


def test_alg1_matches_oracle_driver():
    ev = SyntheticPairs()
    eps = 2e-3
    res = mlmc.alg1(ev, _draw, eps, cost=lambda l: 4.0**l, N_init=lambda l: 32, alpha=2.0)
    ref = omlmc.alg1(lambda l, off, n: ev.dq(l, _draw(l, off, n)), eps, cost=lambda l: 4.0**l,
                     N_init=lambda l: 32, alpha=2.0)
    assert res.L == ref["L"]
    assert res.N == ref["N"]
    assert res.estimate == pytest.approx(ref["estimate"], rel=1e-13)
    assert res.mse == pytest.approx(ref["mse"], rel=1e-10)
    assert res.mse <= 1.01 * eps * eps


def test_alg1_respects_level_cap():
    ev = SyntheticPairs(a=1.0)
    res = mlmc.alg1(ev, _draw, 1e-4, cost=lambda l: 4.0**l, N_init=lambda l: 16, L_max=3)
    assert res.L == 3
