"""Leapfrog and stabilised leapfrog local time-stepping, FP64 (oracle;
test infrastructure only).

Everything here follows the paper's symmetric form (Sec. 3.1, Eq.
Wave_Galerkin_massI): z = M^{1/2} u, A = M^{-1/2} K M^{-1/2},
F~ = M^{-1/2} F, and the time steppers are written in the paper's order:

* leapfrog (Eq. LF2scheme)
      z_{n+1} - 2 z_n + z_{n-1} = dt^2 (F~_n - A z_n)
  with the start value z_1 = z_0 + dt M^{1/2} v_0 + dt^2/2 (F~_0 - A z_0).
  (The printed start has "- dt M^{1/2} v_0"; a Taylor start needs "+".)

* stabilised LF-LTS (Alg. 2), with P the diagonal 0/1 mask and
      delta = 1 + nu / p^2,  omega = 2 T_p'(delta) / T_p(delta),
      beta_m = T_{m-1}(delta) / T_{m+1}(delta),
      beta_{m+1/2} = T_m(delta) / T_{m+1}(delta),       m = 1 .. p-1
  (Sec. 3.3; the algorithm's loop variable is m, its constants are written
  with k: they are the same index).  One step, given z_n and z_{n-1}:
      q_0 = z_n,   w_n = A (I - P) q_0 - F~_n
      q_{1/p} = q_0 - 1/2 (dt/p)^2 (2 p^2 / (omega delta)) (w_n + A P q_0)
      q_{(m+1)/p} = (1 + beta_m) q_{m/p} - beta_m q_{(m-1)/p}
                    - (dt/p)^2 (2 p^2 / omega) beta_{m+1/2} (w_n + A P q_{m/p})
      z_{n+1} = -z_{n-1} + 2 q_1
  The algorithm is printed with zero forcing; the forcing enters through
  w_n, frozen over the step, which keeps Alg. 2 identical to leapfrog for
  P = 0.  No start value is printed for LTS; this oracle uses
  z_1 = q_1(z_0) + dt M^{1/2} v_0, which is the leapfrog start for P = 0.

The inner loop updates every degree of freedom (no restriction to the
neighbourhood of P): that skip is an optimisation the CUDA library makes and
this oracle deliberately does not.
"""
from __future__ import annotations

import numpy as np

from .fem import coefficient, free_system


# --------------------------------------------------------------------------
# constants of the stabilised scheme (Sec. 3.3)
# --------------------------------------------------------------------------
def chebyshev_T(n: int, x: float) -> list:
    """[T_0(x), ..., T_n(x)] by the three-term recurrence of the first kind."""
    T = [1.0, x]
    for _ in range(1, n):
        T.append(2.0 * x * T[-1] - T[-2])
    return T[: n + 1]


def chebyshev_T_prime(n: int, x: float) -> float:
    """T_n'(x) = n U_{n-1}(x), U of the second kind by its recurrence."""
    if n == 0:
        return 0.0
    U = [1.0, 2.0 * x]
    for _ in range(1, n - 1):
        U.append(2.0 * x * U[-1] - U[-2])
    return n * U[n - 1]


def lts_constants(p: int, nu: float, delta: float | None = None) -> dict:
    """delta_{p,nu}, omega_{p,nu}, beta_m and beta_{m+1/2} for m = 1..p-1.

    ``delta`` may be given explicitly (the paper's worked example quotes the
    constants for a given delta)."""
    if delta is None:
        delta = 1.0 + nu / p**2
    T = chebyshev_T(p, delta)
    omega = 2.0 * chebyshev_T_prime(p, delta) / T[p]
    beta = {m: T[m - 1] / T[m + 1] for m in range(1, p)}
    beta_half = {m: T[m] / T[m + 1] for m in range(1, p)}
    return {"p": p, "nu": nu, "delta": delta, "omega": omega,
            "beta": beta, "beta_half": beta_half}


# --------------------------------------------------------------------------
# one step of each scheme, z-form
# --------------------------------------------------------------------------
def lts_inner(q0, A, Pd, dt, C, Ft=None):
    """q_1 of Alg. 2 for q_0 (the p inner substeps with w_n frozen)."""
    p, omega, delta = C["p"], C["omega"], C["delta"]
    tau2 = (dt / p) ** 2
    w = A @ ((1.0 - Pd) * q0)
    if Ft is not None:
        w = w - Ft
    q_prev = q0
    q = q0 - 0.5 * tau2 * (2.0 * p**2 / (omega * delta)) * (w + A @ (Pd * q0))
    for m in range(1, p):
        b, bh = C["beta"][m], C["beta_half"][m]
        q_next = (1.0 + b) * q - b * q_prev - tau2 * (2.0 * p**2 / omega) * bh * (w + A @ (Pd * q))
        q_prev, q = q, q_next
    return q


def lts_step(z_n, z_nm1, A, Pd, dt, C, Ft=None):
    """z_{n+1} of Alg. 2."""
    return -z_nm1 + 2.0 * lts_inner(z_n, A, Pd, dt, C, Ft)


def lf_step(z_n, z_nm1, A, dt, Ft=None):
    """z_{n+1} of Eq. LF2scheme."""
    rhs = -(A @ z_n)
    if Ft is not None:
        rhs = rhs + Ft
    return 2.0 * z_n - z_nm1 + dt**2 * rhs


# --------------------------------------------------------------------------
# whole solves
# --------------------------------------------------------------------------
def march_lts(A, Pd, z0, zv0, dt, n_steps, p, nu, F=None):
    """z_N of Alg. 2 from z_0 and the z-velocity zv0 = M^{1/2} v_0.

    F, if given, is a callable t -> F~(t) (already scaled by M^{-1/2})."""
    C = lts_constants(p, nu)
    Ft = (lambda n: F(n * dt)) if F is not None else (lambda n: None)
    z_prev = z0
    z = lts_inner(z0, A, Pd, dt, C, Ft(0)) + dt * zv0
    for n in range(1, n_steps):
        z_prev, z = z, lts_step(z, z_prev, A, Pd, dt, C, Ft(n))
    return z


def march_lf(A, z0, zv0, dt, n_steps, F=None):
    """z_N of Eq. LF2scheme."""
    Ft = (lambda n: F(n * dt)) if F is not None else (lambda n: None)
    f0 = Ft(0)
    z = z0 + dt * zv0 + 0.5 * dt**2 * (-(A @ z0) + (f0 if f0 is not None else 0.0))
    z_prev = z0
    for n in range(1, n_steps):
        z_prev, z = z, lf_step(z, z_prev, A, dt, Ft(n))
    return z


class Problem:
    """Free-node system of one mesh for one coefficient draw, in z-form."""

    def __init__(self, xy, tri, dirichlet, P, psi, xi):
        self.n_nodes = xy.shape[0]
        c2 = coefficient(psi, np.asarray(xi, dtype=np.float64))
        self.free, self.m, K = free_system(xy, tri, dirichlet, c2)
        s = 1.0 / np.sqrt(self.m)
        self.A = (K.multiply(s[:, None]).multiply(s[None, :])).tocsr()
        self.Pd = np.asarray(P, dtype=np.float64)[self.free]
        self.sqrt_m = np.sqrt(self.m)

    def to_z(self, u):
        return self.sqrt_m * np.asarray(u, dtype=np.float64)[self.free]

    def to_u(self, z):
        u = np.zeros(self.n_nodes)
        u[self.free] = z / self.sqrt_m
        return u


def ricker(t, f0, t0):
    """Ricker wavelet r(t) = (1 - 2 pi^2 f0^2 (t - t0)^2) exp(-pi^2 f0^2 (t - t0)^2)."""
    a = (np.pi * f0 * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def source_forcing(pb, n_nodes, source):
    """F~(t) = M^{-1/2} F(t), F(t) = amp r(t) F_space, as a callable of t (z-form)."""
    if source is None:
        return None
    F = np.zeros(n_nodes)
    np.add.at(F, np.asarray(source["nodes"]), np.asarray(source["weights"], dtype=np.float64))
    Ft = F[pb.free] / pb.sqrt_m
    return lambda t: source["amp"] * ricker(t, source["f0"], source["t0"]) * Ft


def solve_sample(xy, tri, dirichlet, P, psi, xi, u0, dt, n_steps, p, nu, v0=None,
                 scheme="lts", source=None):
    """u_N (all nodes) for one draw xi: the per-sample hot path of Alg. 1."""
    pb = Problem(xy, tri, dirichlet, P, psi, xi)
    z0 = pb.to_z(u0)
    zv0 = pb.to_z(v0) if v0 is not None else np.zeros_like(z0)
    F = source_forcing(pb, xy.shape[0], source)
    if scheme == "lts":
        zN = march_lts(pb.A, pb.Pd, z0, zv0, dt, n_steps, p, nu, F=F)
    elif scheme == "lf":
        zN = march_lf(pb.A, z0, zv0, dt, n_steps, F=F)
    else:
        raise ValueError(scheme)
    return pb.to_u(zN)


def qoi(u, idx, g) -> float:
    """Q(u) = sum_k g_k u_{idx_k}: a linear functional of u_h(., T)."""
    return float(np.dot(np.asarray(g, dtype=np.float64), np.asarray(u)[np.asarray(idx)]))


def solve_qoi(level: dict, xi, scheme="lts") -> float:
    """Q_l(omega) for one draw on one level (dict as built by workload)."""
    m = level["mesh"]
    u = solve_sample(m.xy, m.tri, m.dirichlet, m.P, level["psi"], xi, level["u0"],
                     level["dt"], level["n_steps"], level["p"], level["nu"], scheme=scheme,
                     source=level.get("source"))
    return qoi(u, level["qoi_idx"], level["qoi_w"])
