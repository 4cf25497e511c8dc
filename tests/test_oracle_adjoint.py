"""Pins of the oracle's QoI derivative (tangent-linear model and central
finite differences) against closed forms and against each other (no GPU)."""
import math

import numpy as np
import pytest

from oracle.adjoint import fd_gradient, tangent_gradient
from oracle.lts import lts_constants, solve_qoi
from workload import box_qoi_weights, square_mesh

from gpu_common import small_level


def _mode_level(n=12, p=1, Pfull=False):
    m = square_mesh(n)
    if Pfull:
        m.P = (~m.dirichlet.astype(bool)).astype(np.uint8)
    u0 = np.sin(np.pi * m.xy[:, 0]) * np.sin(np.pi * m.xy[:, 1])
    idx, g = box_qoi_weights(m, (0.2, 0.45, 0.3, 0.6))
    return {"mesh": m, "psi": np.ones((m.n_tri, 1)), "u0": u0, "qoi_idx": idx, "qoi_w": g,
            "dt": 0.04, "n_steps": 20, "p": p, "nu": 0.01 if p > 1 else 0.0}


def _closed_form(lev, xi, lts):
    """Q and dQ/dxi for c^2 = exp(xi) on the (1,1) standing mode."""
    n = lev["mesh"].meta["n"]
    h, dt, N = 1.0 / n, lev["dt"], lev["n_steps"]
    lam = 8 / h**2 * math.sin(math.pi * h / 2) ** 2
    Qphi = lev["qoi_w"] @ lev["u0"][lev["qoi_idx"]]
    c2 = math.exp(xi)
    if lts:
        C = lts_constants(lev["p"], lev["nu"])
        d, om, p = C["delta"], C["omega"], lev["p"]
        def Tp(x):
            return math.cos(p * math.acos(x)) if abs(x) <= 1 else math.cosh(p * math.acosh(x))

        def dTp(x):
            if abs(x) < 1:
                return p * math.sin(p * math.acos(x)) / math.sqrt(1 - x * x)
            t = math.acosh(x)
            return p * math.sinh(p * t) / math.sinh(t)
        y = d - dt * dt * c2 * lam / om
        S = Tp(y) / math.cosh(p * math.acosh(d))
        dS = dTp(y) * (-dt * dt * c2 * lam / om) / math.cosh(p * math.acosh(d))
    else:
        S = 1 - dt * dt * c2 * lam / 2
        dS = -dt * dt * c2 * lam / 2
    th = math.acos(S)
    dth = -dS / math.sin(th)
    return math.cos(N * th) * Qphi, -N * math.sin(N * th) * dth * Qphi


@pytest.mark.parametrize("lts", [False, True])
def test_tangent_and_fd_match_closed_form(lts):
    lev = _mode_level(p=3 if lts else 1, Pfull=lts)
    for xi in (-0.6, 0.4):
        Qc, dQc = _closed_form(lev, xi, lts)
        Q, dQ = tangent_gradient(lev, np.array([xi]))
        assert Q == pytest.approx(Qc, abs=1e-13)
        assert dQ[0] == pytest.approx(dQc, rel=1e-9, abs=1e-13)
        assert fd_gradient(lev, np.array([xi]))[0] == pytest.approx(dQc, rel=1e-6, abs=1e-10)


def test_tangent_matches_fd_with_local_refinement():
    lev = small_level(n=10, p=3, K=3, T=0.3)
    xi = np.array([0.3, -0.8, 0.5])
    Q, dQ = tangent_gradient(lev, xi)
    assert Q == pytest.approx(solve_qoi(lev, xi), rel=1e-13)
    fd = fd_gradient(lev, xi)
    assert np.abs(dQ - fd).max() <= 1e-6 * np.abs(dQ).max()
