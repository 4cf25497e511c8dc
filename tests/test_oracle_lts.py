"""Pins of the FP64 oracle's time steppers against facts the paper and the
mathematics fix (no GPU).  Each test targets a plausible mistake: a wrong
constant, index or sign in Alg. 2 breaks one of the closed forms, the
symmetry/energy identity or the convergence order."""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sl

from oracle.lts import (Problem, chebyshev_T, chebyshev_T_prime, lts_constants,
                        lts_inner, lts_step, march_lf, march_lts)
from workload import coarse_dt, gaussian_bump, psi_sine, square_mesh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _Tp(p, x):
    """Chebyshev T_p by its trigonometric / hyperbolic closed form."""
    if abs(x) <= 1:
        return math.cos(p * math.acos(x))
    s = 1.0 if x > 0 or p % 2 == 0 else -1.0
    return s * math.cosh(p * math.acosh(abs(x)))


# ---------------------------------------------------------------- constants
def test_constants_worked_example_sec33():
    rows = {}
    for line in open(os.path.join(GOLDEN, "lts_constants_p2_nu001.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, val, tol = line.split()
        rows[name] = (float(val), float(tol))
    C = lts_constants(int(rows["p"][0]), 0.01, delta=rows["delta"][0])
    assert abs(C["omega"] - rows["omega"][0]) <= rows["omega"][1]
    assert abs(C["beta"][1] - rows["beta_1"][0]) <= rows["beta_1"][1]
    assert abs(C["beta_half"][1] - rows["beta_3/2"][0]) <= rows["beta_3/2"][1]
    # the closed forms printed beside the example
    d = 1.005
    assert C["omega"] == pytest.approx(2 * 4 * d / (2 * d * d - 1), rel=1e-15)
    assert C["beta"][1] == pytest.approx(1 / (2 * d * d - 1), rel=1e-15)
    assert C["beta_half"][1] == pytest.approx(d / (2 * d * d - 1), rel=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 8, 16])
@pytest.mark.parametrize("nu", [0.0, 0.01, 0.5, 1.0])
def test_constants_against_hyperbolic_closed_form(p, nu):
    C = lts_constants(p, nu)
    d = 1.0 + nu / p**2
    assert C["delta"] == d
    T = chebyshev_T(p, d)
    for k in range(p + 1):
        assert T[k] == pytest.approx(_Tp(k, d), rel=1e-13)
    if d > 1:
        th = math.acosh(d)
        Tp_prime = p * math.sinh(p * th) / math.sinh(th)
    else:
        Tp_prime = p * p
    assert chebyshev_T_prime(p, d) == pytest.approx(Tp_prime, rel=1e-12)
    assert C["omega"] == pytest.approx(2 * Tp_prime / _Tp(p, d), rel=1e-12)


@pytest.mark.parametrize("p", [1, 2, 5, 8])
def test_nu_zero_is_diaz_grote(p):
    """nu = 0: delta = 1, all beta = 1, omega = 2 p^2 (Sec. 3.3)."""
    C = lts_constants(p, 0.0)
    assert C["delta"] == 1.0
    assert C["omega"] == pytest.approx(2.0 * p * p, rel=1e-15)
    assert all(b == 1.0 for b in C["beta"].values())
    assert all(b == 1.0 for b in C["beta_half"].values())


# ------------------------------------------------------ uniform-mesh modes
def _uniform_mode(n=16, a=1, b=2, c2=1.0):
    m = square_mesh(n)
    h = 1.0 / n
    psi = np.zeros((m.n_tri, 1))
    xi = np.array([math.log(c2)])
    psi[:, 0] = 1.0
    pb = Problem(m.xy, m.tri, m.dirichlet, np.zeros(m.n_nodes), psi, xi)
    u0 = np.sin(a * np.pi * m.xy[:, 0]) * np.sin(b * np.pi * m.xy[:, 1])
    lam = c2 * 4 / h**2 * (math.sin(a * math.pi * h / 2) ** 2 + math.sin(b * math.pi * h / 2) ** 2)
    return m, pb, pb.to_z(u0), lam


def test_discrete_standing_mode_is_eigenvector():
    """On the "/"-split uniform grid, lumped P1: sin(a pi x) sin(b pi y) is an
    exact eigenvector of M^-1 K with the 5-point-Laplacian eigenvalue."""
    for c2 in (1.0, 2.5):
        _, pb, z0, lam = _uniform_mode(c2=c2)
        r = pb.A @ z0 - lam * z0
        assert np.abs(r).max() <= 1e-12 * lam * np.abs(z0).max()


def test_leapfrog_standing_mode_closed_form():
    """LF on an eigenvector: z_n = cos(n theta) z_0, cos theta = 1 - dt^2 lam / 2."""
    _, pb, z0, lam = _uniform_mode()
    dt, N = 0.02, 60
    zN = march_lf(pb.A, z0, 0 * z0, dt, N)
    th = math.acos(1 - dt * dt * lam / 2)
    assert np.abs(zN - math.cos(N * th) * z0).max() < 1e-13


@pytest.mark.parametrize("p,nu", [(1, 0.0), (2, 0.01), (3, 0.0), (4, 0.01), (8, 0.01), (5, 0.5)])
def test_lts_full_mask_closed_form(p, nu):
    """P = I: the inner recursion is the stabilised Chebyshev polynomial,
    q_1 = T_p(delta - dt^2 lam / omega) / T_p(delta) q_0, so on an eigenvector
    z_n = cos(n Theta) z_0 with cos Theta = that ratio (derived from Alg. 2 by
    the three-term recurrence of T_k; the closed form uses cos/cosh)."""
    _, pb, z0, lam = _uniform_mode()
    dt, N = 0.02, 60
    C = lts_constants(p, nu)
    zN = march_lts(pb.A, np.ones_like(z0), z0, 0 * z0, dt, N, p, nu)
    S = _Tp(p, C["delta"] - dt * dt * lam / C["omega"]) / _Tp(p, C["delta"])
    Th = math.acos(S)
    assert np.abs(zN - math.cos(N * Th) * z0).max() < 1e-12


@pytest.mark.parametrize("p,nu", [(2, 0.01), (4, 0.5), (7, 0.0)])
def test_lts_empty_mask_is_leapfrog(p, nu):
    """P = 0: Alg. 2 reduces to LF for any p, nu (Sec. 3.3)."""
    _, pb, z0, lam = _uniform_mode()
    dt, N = 0.02, 60
    zN = march_lts(pb.A, np.zeros_like(z0), z0, 0 * z0, dt, N, p, nu)
    th = math.acos(1 - dt * dt * lam / 2)
    assert np.abs(zN - math.cos(N * th) * z0).max() < 1e-12


# ---------------------------------------------------- locally refined mesh
def _refined_problem(n=12, p=3, K=4, seed=0):
    m = square_mesh(n, box=(0.35, 0.65, 0.35, 0.65), p=p)
    psi = psi_sine(m, K)
    xi = np.random.default_rng(seed).uniform(-1, 1, K)
    return m, Problem(m.xy, m.tri, m.dirichlet, m.P, psi, xi)


@pytest.mark.parametrize("p,nu", [(2, 0.0), (3, 0.01), (4, 0.5)])
def test_lts_step_operator_symmetric(p, nu):
    """B z = (2/dt^2)(z - q_1(z)) is symmetric: the LF-LTS step is a leapfrog
    step for a symmetric operator, the basis of its energy identity."""
    m, pb = _refined_problem(p=p)
    C = lts_constants(p, nu)
    dt, _ = coarse_dt(m.H, 4, 1.0)
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal((2, pb.A.shape[0]))
    Bx = x - lts_inner(x, pb.A, pb.Pd, dt, C)
    By = y - lts_inner(y, pb.A, pb.Pd, dt, C)
    assert abs(x @ By - y @ Bx) <= 1e-13 * abs(x @ By)


def test_lts_energy_conserved_with_local_refinement():
    m, pb = _refined_problem(p=3)
    C = lts_constants(3, 0.01)
    dt, _ = coarse_dt(m.H, 4, 1.0)
    B = lambda z: 2 / dt**2 * (z - lts_inner(z, pb.A, pb.Pd, dt, C))
    z0 = pb.to_z(gaussian_bump(m))
    zp, z = z0, lts_inner(z0, pb.A, pb.Pd, dt, C)
    E = []
    for _ in range(200):
        zn = lts_step(z, zp, pb.A, pb.Pd, dt, C)
        E.append(0.5 * np.sum(((zn - z) / dt) ** 2) + 0.5 * zn @ B(z))
        zp, z = z, zn
    E = np.asarray(E)
    assert (E.max() - E.min()) <= 1e-12 * E.mean()


def test_lts_second_order_to_semidiscrete_solution():
    """Error against z(T) = cos(T sqrt(A)) z_0 (eigendecomposition) falls by 4x
    per halving of dt: Alg. 2 is consistent and second order."""
    m, pb = _refined_problem(p=3)
    A = pb.A.toarray()
    w, V = sl.eigh(A)
    z0 = pb.to_z(gaussian_bump(m))
    T = 0.5
    zex = V @ (np.cos(T * np.sqrt(w)) * (V.T @ z0))
    errs = []
    for k in range(4):
        nst = 16 * 2**k
        zN = march_lts(pb.A, pb.Pd, z0, 0 * z0, T / nst, nst, 3, 0.01)
        errs.append(np.linalg.norm(zN - zex))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.8 < r < 4.3 for r in ratios), ratios


def test_lts_agrees_with_tiny_step_leapfrog():
    """Brute force: LF with dt/(8p) everywhere vs LF-LTS; the difference is the
    LTS time discretisation error, O(dt^2), small against the solution."""
    m, pb = _refined_problem(p=2)
    z0 = pb.to_z(gaussian_bump(m))
    T, nst = 0.3, 30
    z_lts = march_lts(pb.A, pb.Pd, z0, 0 * z0, T / nst, nst, 2, 0.01)
    z_ref = march_lf(pb.A, z0, 0 * z0, T / (nst * 16), nst * 16)
    rel = np.linalg.norm(z_lts - z_ref) / np.linalg.norm(z_ref)
    z_lts2 = march_lts(pb.A, pb.Pd, z0, 0 * z0, T / (2 * nst), 2 * nst, 2, 0.01)
    rel2 = np.linalg.norm(z_lts2 - z_ref) / np.linalg.norm(z_ref)
    assert rel < 2e-2 and rel2 < rel / 3.0


def test_lts_initial_velocity_start():
    """With v0 != 0 the start z_1 = q_1(z_0) + dt M^{1/2} v_0 is second order:
    the error against the exact solution falls ~4x per halving."""
    m, pb = _refined_problem(p=2)
    A = pb.A.toarray()
    w, V = sl.eigh(A)
    z0 = pb.to_z(gaussian_bump(m))
    zv = pb.to_z(gaussian_bump(m, center=(0.6, 0.5), a=80.0))
    T = 0.4
    sw = np.sqrt(w)
    zex = V @ (np.cos(T * sw) * (V.T @ z0) + np.sin(T * sw) / sw * (V.T @ zv))
    errs = [np.linalg.norm(march_lts(pb.A, pb.Pd, z0, zv, T / n, n, 2, 0.01) - zex)
            for n in (20, 40, 80)]
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


# ----------------------------------------------------------------- forcing
@pytest.mark.parametrize("lts", [False, True])
def test_constant_forcing_closed_form(lts):
    """Constant modal forcing F = f M phi from rest: the discrete solution is
    c_n = (f / lam)(1 - cos(n Theta)) phi with cos Theta = 1 - dt^2 lam / 2 (LF,
    P = 0) or T_p(delta - dt^2 lam / omega) / T_p(delta) (LTS, P = I): the
    step is affine with fixed point f / lam (where w_n + A P q_0 = 0)."""
    from oracle.fem import lumped_mass
    from oracle.lts import solve_sample
    n = 16
    m = square_mesh(n)
    h = 1.0 / n
    phi = np.sin(np.pi * m.xy[:, 0]) * np.sin(2 * np.pi * m.xy[:, 1])
    lam = 4 / h**2 * (math.sin(math.pi * h / 2) ** 2 + math.sin(math.pi * h) ** 2)
    f = 3.0
    mass = lumped_mass(m.xy, m.tri)
    free = np.nonzero(~m.dirichlet.astype(bool))[0]
    src = {"nodes": free, "weights": f * mass[free] * phi[free], "f0": 0.0, "t0": 0.0, "amp": 1.0}
    dt, N, p, nu = 0.02, 37, 3, 0.01
    Pm = (~m.dirichlet.astype(bool)).astype(np.uint8) if lts else np.zeros(m.n_nodes, np.uint8)
    u = solve_sample(m.xy, m.tri, m.dirichlet, Pm, np.zeros((m.n_tri, 1)), np.zeros(1),
                     np.zeros(m.n_nodes), dt, N, p, nu, source=src)
    if lts:
        C = lts_constants(p, nu)
        S = _Tp(p, C["delta"] - dt * dt * lam / C["omega"]) / _Tp(p, C["delta"])
    else:
        S = 1 - dt * dt * lam / 2
    expect = f / lam * (1 - math.cos(N * math.acos(S))) * phi
    assert np.abs(u - expect).max() < 1e-12 * np.abs(expect).max()


def test_ricker_wavelet_values():
    from oracle.lts import ricker
    assert ricker(0.3, 10.0, 0.3) == 1.0
    # zero crossings at |t - t0| = 1 / (sqrt(2) pi f0)
    assert abs(ricker(0.3 + 1 / (math.sqrt(2) * math.pi * 10.0), 10.0, 0.3)) < 1e-15
    assert ricker(1.0, 0.0, 0.0) == 1.0
