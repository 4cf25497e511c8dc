"""Cost models of MLMC with leapfrog (LF) and with LF-LTS (Sec. 3.2-3.4).

Per solve on level l with H_l = H_0 / 2^l, polynomial degree k, dimension
d, relative volume r of the refined part and ratio p_l (constants dropped):

  Eq. cost_waveeq_LF : C_LF[u_l]  ~ T k^{2(d+1)} p_l / H_l^{d+1} ((1 - r) + r p_l^d)
  Eq. cost_waveeq_LTS: C_LTS[u_l] ~ T k^{2(d+1)}       / H_l^{d+1} ((1 - r) + r p_l^{d+1})

A level-l sample dQ_l costs the fine and the coarse solve (Eqs. C_l_LF,
C_l_LTS), and with the optimal sample numbers the total cost is
(2/eps^2) (sum_l sqrt(V_l C_l))^2, so the speed-up of LTS over LF (Prop. 3.2,
Eq. fullQ_eff) is

  S = (sum_l sqrt(V_l C_l^LF))^2 / (sum_l sqrt(V_l C_l^LTS))^2.

``solve_work`` gives the measured counterpart in DOF updates:
N_steps (n_free + p |R|) for LTS and (p N_steps) n_free for leapfrog with
the fine step dt/p.
"""
from __future__ import annotations

import math


def cost_lf(T, k, d, H, p, r):
    return T * k ** (2 * (d + 1)) * p / H ** (d + 1) * ((1 - r) + r * p**d)


def cost_lts(T, k, d, H, p, r):
    return T * k ** (2 * (d + 1)) / H ** (d + 1) * ((1 - r) + r * p ** (d + 1))


def level_costs(T, k, d, H0, p_levels, r, scheme):
    """C_l of one dQ_l sample (fine + coarse solve), l = 0 .. L."""
    f = cost_lf if scheme == "lf" else cost_lts
    out = []
    for l, p in enumerate(p_levels):
        c = f(T, k, d, H0 / 2**l, p, r)
        if l > 0:
            c += f(T, k, d, H0 / 2 ** (l - 1), p_levels[l - 1], r)
        out.append(c)
    return out


def speedup_S(V, C_lf, C_lts):
    """Prop. 3.2: ratio of the optimal MLMC total costs, LF over LTS."""
    a = math.fsum(math.sqrt(v * c) for v, c in zip(V, C_lf))
    b = math.fsum(math.sqrt(v * c) for v, c in zip(V, C_lts))
    return (a / b) ** 2


def solve_work(n_steps, n_free, n_R, p, scheme):
    """DOF updates of one solve: the measured analogue of the cost model."""
    if scheme == "lts":
        return n_steps * (n_free + p * n_R)
    return p * n_steps * n_free
