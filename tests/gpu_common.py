"""Shared helpers of the GPU tests: small seeded problems and the oracle runs
they are compared against."""
import math

import numpy as np

from oracle.lts import solve_sample
from workload import box_qoi_weights, coarse_dt, gaussian_bump, psi_sine, square_mesh


def small_level(n=12, p=3, K=4, box=(0.35, 0.65, 0.35, 0.65), T=0.6, nu=0.01,
                qoi_box=(0.6, 0.85, 0.55, 0.8), refine=True):
    m = square_mesh(n, box=box if refine else None, p=p if refine else 1)
    dt, n_steps = coarse_dt(m.H, K, T)
    idx, g = box_qoi_weights(m, qoi_box)
    return {"mesh": m, "psi": psi_sine(m, K), "u0": gaussian_bump(m, (0.3, 0.3), 120.0),
            "qoi_idx": idx, "qoi_w": g, "dt": dt, "n_steps": n_steps, "p": p, "nu": nu, "T": T}


def oracle_run(level, xi, scheme="lts", P=True, p=None, v0=None, source=None):
    """(Q [S], u_N [n_nodes, S]) from the FP64 oracle, one sample at a time."""
    m = level["mesh"]
    Pm = m.P if P else np.zeros(m.n_nodes, np.uint8)
    us = []
    for x in xi:
        us.append(solve_sample(m.xy, m.tri, m.dirichlet, Pm, level["psi"], x, level["u0"],
                               level["dt"], level["n_steps"], level["p"] if p is None else p,
                               level["nu"], v0=v0, scheme=scheme, source=source))
    U = np.stack(us, axis=1)
    Q = level["qoi_w"] @ U[level["qoi_idx"]]
    return Q, U


def rel_err(a, b):
    """max |a - b| / max |b|: error relative to the batch's scale."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def draws(S, K, seed=0):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(S, K))
