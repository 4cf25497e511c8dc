"""Derivative of the QoI with respect to the field parameters xi, FP64 (oracle;
test infrastructure only).

Two plain definitions of dQ/dxi_k for one draw:

* ``tangent_gradient``: forward-mode differentiation of Alg. 2 line by line
  (z-form, as in ``oracle.lts``).  With dA/dxi_k = M^{-1/2} K_k M^{-1/2},
  K_k the stiffness assembled with the coefficient psi_{e,k} c_e^2 (the
  derivative of c_e^2 = exp(sum_k xi_k psi_{e,k})), every line of the step is
  differentiated:
      dw      = dA (I-P) q_0 + A (I-P) dq_0
      dq_{1/p} = dq_0 - 1/2 (dt/p)^2 2p^2/(omega delta) (dw + dA P q_0 + A P dq_0)
      dq_{(m+1)/p} = (1+beta_m) dq_{m/p} - beta_m dq_{(m-1)/p}
                     - (dt/p)^2 2p^2/omega beta_{m+1/2} (dw + dA P q_{m/p} + A P dq_{m/p})
      dz_{n+1} = -dz_{n-1} + 2 dq_1,    dz_0 = 0 (u0 does not depend on xi)
  and dQ/dxi_k = g . (M^{-1/2} dz_N).  This is the exact derivative of the
  discrete QoI, one forward pass per direction.
* ``fd_gradient``: central differences (Q(xi + h e_k) - Q(xi - h e_k)) / 2h.
"""
from __future__ import annotations

import numpy as np

from .fem import coefficient, stiffness
from .lts import Problem, lts_constants, qoi, solve_qoi, source_forcing


def _tangent_inner(q0, dq0, A, dA, Pd, dt, C, Ft=None):
    p, omega, delta = C["p"], C["omega"], C["delta"]
    tau2 = (dt / p) ** 2
    w = A @ ((1.0 - Pd) * q0)
    if Ft is not None:
        w = w - Ft  # the forcing does not depend on xi: it has no tangent
    dw = dA @ ((1.0 - Pd) * q0) + A @ ((1.0 - Pd) * dq0)
    a0 = 0.5 * tau2 * (2.0 * p**2 / (omega * delta))
    q_prev, dq_prev = q0, dq0
    q = q0 - a0 * (w + A @ (Pd * q0))
    dq = dq0 - a0 * (dw + dA @ (Pd * q0) + A @ (Pd * dq0))
    for m in range(1, p):
        b, bh = C["beta"][m], C["beta_half"][m]
        am = tau2 * (2.0 * p**2 / omega) * bh
        q_next = (1.0 + b) * q - b * q_prev - am * (w + A @ (Pd * q))
        dq_next = (1.0 + b) * dq - b * dq_prev - am * (dw + dA @ (Pd * q) + A @ (Pd * dq))
        q_prev, q = q, q_next
        dq_prev, dq = dq, dq_next
    return q, dq


def tangent_gradient(level: dict, xi) -> tuple:
    """(Q, dQ/dxi [K]) of one draw by forward-mode differentiation of Alg. 2."""
    m = level["mesh"]
    xi = np.asarray(xi, dtype=np.float64)
    psi = level["psi"]
    pb = Problem(m.xy, m.tri, m.dirichlet, m.P, psi, xi)
    c2 = coefficient(psi, xi)
    s = 1.0 / np.sqrt(pb.m)
    free = pb.free
    dt, N, p, nu = level["dt"], level["n_steps"], level["p"], level["nu"]
    C = lts_constants(p, nu)
    z0 = pb.to_z(level["u0"])
    F = source_forcing(pb, m.n_nodes, level.get("source"))
    Ft = (lambda n: F(n * dt)) if F is not None else (lambda n: None)
    grads = []
    zN = None
    for k in range(psi.shape[1]):
        Kk = stiffness(m.xy, m.tri, c2 * psi[:, k])[free][:, free]
        dA = Kk.multiply(s[:, None]).multiply(s[None, :]).tocsr()
        z_prev, dz_prev = z0, np.zeros_like(z0)
        z, dz = _tangent_inner(z0, dz_prev, pb.A, dA, pb.Pd, dt, C, Ft(0))
        for n in range(1, N):
            q, dq = _tangent_inner(z, dz, pb.A, dA, pb.Pd, dt, C, Ft(n))
            z_prev, z, dz_prev, dz = z, -z_prev + 2.0 * q, dz, -dz_prev + 2.0 * dq
        zN = z
        grads.append(qoi(pb.to_u(dz), level["qoi_idx"], level["qoi_w"]))
    Q = qoi(pb.to_u(zN), level["qoi_idx"], level["qoi_w"])
    return Q, np.array(grads)


def fd_gradient(level: dict, xi, h: float = 1e-6) -> np.ndarray:
    """Central finite differences of Q(xi), step h per component."""
    xi = np.asarray(xi, dtype=np.float64)
    out = []
    for k in range(xi.shape[0]):
        e = np.zeros_like(xi)
        e[k] = h
        out.append((solve_qoi(level, xi + e) - solve_qoi(level, xi - e)) / (2.0 * h))
    return np.array(out)
