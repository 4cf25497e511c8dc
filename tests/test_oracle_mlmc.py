"""Pins of the oracle's MLMC estimator and of Alg. 1 (no GPU)."""
import math

import numpy as np
import pytest

from oracle import mlmc
from oracle.lts import solve_qoi
from workload import box_qoi_weights, square_mesh


def test_level_sums_exact_on_representable_data():
    Qf = np.array([0.5, 0.25, -1.0, 2.0])
    Qc = np.array([0.25, 0.25, -0.5, 1.0])
    s = mlmc.level_sums(Qf, Qc)
    assert s == (0.25 + 0.0 - 0.5 + 1.0, 0.0625 + 0 + 0.25 + 1.0, 1.75, 0.25 + 0.0625 + 1 + 4)
    assert mlmc.level_sums(Qf)[:2] == (1.75, 5.3125)


def test_level_sums_cancellation():
    """Sums of huge cancelling terms stay exact (a naive loop returns 0)."""
    Qf = np.array([1e16, 1.0, -1e16, 1.0])
    assert mlmc.level_sums(Qf)[0] == 2.0


def test_estimator_variance_and_optimal_N_closed_forms():
    assert mlmc.estimator([3.0, 1.0], [3, 4]) == pytest.approx(1.25)
    x = np.array([1.0, 2.0, 4.0, 7.0])
    V = mlmc.variance(x.sum(), (x * x).sum(), len(x))
    assert V == pytest.approx(np.var(x, ddof=1), rel=1e-15)
    # two levels: N_l = 2/eps^2 sqrt(V_l/C_l) (sqrt(V0 C0) + sqrt(V1 C1))
    N = mlmc.optimal_N([4.0, 1.0], [1.0, 4.0], 0.1)
    assert N == [math.ceil(200 * 2 * 4), math.ceil(200 * 0.5 * 4)]
    # the optimum balances the variance part of the MSE at eps^2 / 2
    Nr = [200 * 2 * 4, 200 * 0.5 * 4]
    assert 4.0 / Nr[0] + 1.0 / Nr[1] == pytest.approx(0.1**2 / 2)


def test_bias_estimate_geometric_tail():
    """If E[dQ_l] = a 2^{-alpha l} exactly, Eq. bias_est is exact."""
    a, alpha, L = 0.3, 2.0, 4
    tail = sum(a * 2.0 ** (-alpha * l) for l in range(L + 1, 200))
    assert mlmc.bias_estimate(a * 2.0 ** (-alpha * L), alpha) == pytest.approx(tail, rel=1e-12)


def test_alg1_on_synthetic_hierarchy():
    """dQ_l = a 4^{-l} + s 2^{-l} Z (Z standard normal): E[Q_L] known, the
    MSE estimate of Alg. 1 must cover the true error."""
    a, s, eps = 1.0, 0.5, 2e-3
    rng = np.random.default_rng(11)

    def sample(l, off, n):
        return a * 4.0 ** (-l) + s * 2.0 ** (-l) * rng.standard_normal(n)

    res = mlmc.alg1(sample, eps, cost=lambda l: 4.0**l, N_init=lambda l: 64, alpha=2.0)
    L = res["L"]
    exact_L = sum(a * 4.0 ** (-l) for l in range(L + 1))
    assert math.isfinite(res["mse"]) and res["mse"] <= 1.01 * eps**2
    assert abs(res["estimate"] - exact_L) < 3 * math.sqrt(sum(
        (s * 2.0 ** (-l)) ** 2 / n for l, n in enumerate(res["N"])))
    assert (a * 4.0 ** (-L) / 3.0) ** 2 < eps**2 / 2
    assert all(n >= 64 for n in res["N"])


def _mode_level(n, K=1):
    m = square_mesh(n)
    psi = np.ones((m.n_tri, K))
    u0 = np.sin(np.pi * m.xy[:, 0]) * np.sin(np.pi * m.xy[:, 1])
    idx, g = box_qoi_weights(m, (0.2, 0.4, 0.3, 0.6))
    dt = 0.5 / n
    T = 0.6
    n_steps = int(math.ceil(T / dt))
    return {"mesh": m, "psi": psi, "u0": u0, "qoi_idx": idx, "qoi_w": g,
            "dt": T / n_steps, "n_steps": n_steps, "p": 1, "nu": 0.0, "T": T}


def _closed_form_Q(level, xi):
    n = level["mesh"].meta["n"]
    h = 1.0 / n
    lam = math.exp(xi) * 8 / h**2 * math.sin(math.pi * h / 2) ** 2
    th = math.acos(1 - level["dt"] ** 2 * lam / 2)
    Qphi = level["qoi_w"] @ level["u0"][level["qoi_idx"]]
    return math.cos(level["n_steps"] * th) * Qphi


def test_oracle_solve_matches_dispersion_closed_form():
    """Constant field c^2 = exp(xi) and a standing-mode initial datum: Q_l(xi)
    is cos(N theta(xi)) Q(phi) by the discrete dispersion relation."""
    lev = _mode_level(8)
    for xi in (-0.9, 0.0, 0.7):
        assert solve_qoi(lev, np.array([xi])) == pytest.approx(_closed_form_Q(lev, xi), abs=1e-13)


def test_alg1_with_oracle_solver_against_quadrature_mean():
    """MLMC of the standing mode with c^2 = exp(xi), xi ~ U(-1,1): the estimate
    lies within 3 RMSE of E[Q_L], computed by Gauss-Legendre quadrature of the
    closed form."""
    levels = [_mode_level(4 * 2**l) for l in range(4)]
    rng = np.random.default_rng(2)

    def sample(l, off, n):
        xs = rng.uniform(-1, 1, n)
        out = []
        for x in xs:
            qf = solve_qoi(levels[l], np.array([x]))
            qc = solve_qoi(levels[l - 1], np.array([x])) if l > 0 else 0.0
            out.append(qf - qc)
        return np.array(out)

    eps = 4e-3
    res = mlmc.alg1(sample, eps, cost=lambda l: 8.0**l, N_init=lambda l: 16, alpha=2.0, L_max=3)
    L = res["L"]
    xg, wg = np.polynomial.legendre.leggauss(200)
    EQ = 0.5 * sum(w * _closed_form_Q(levels[L], x) for x, w in zip(xg, wg))
    rmse = math.sqrt(sum(v / n for v, n in zip(res["V"], res["N"])))
    assert abs(res["estimate"] - EQ) < 3 * rmse + 1e-12
