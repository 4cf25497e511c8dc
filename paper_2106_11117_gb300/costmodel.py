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


# ---------------------------------------------------------------------------
# Graded meshes T_{m,s} (Sec. 3.5): m layers, grading s, the first q layers
# form the region of the small step.
# ---------------------------------------------------------------------------
def cost_lf_graded(m, d, s):
    """Eq. cost_waveeq_LFgraded: elements / h_1 ~ m^{s+d}."""
    return float(m) ** (s + d)


def cost_lts_graded(m, d, s, q):
    """Eq. cost_waveeq_LTSgraded: the first q layers step with h_1, the rest
    with h_{q+1} ~ ((q+1)^s - q^s) / m^s."""
    g = (q + 1.0) ** s - float(q) ** s
    return (float(m) ** (s + d) + float(m) ** s * float(q) ** d * (g - 1.0)) / g


def speedup_graded(m, d, s, q):
    """Eq. speedup_det_graded: one LF solve over one LTS solve."""
    g = (q + 1.0) ** s - float(q) ** s
    return float(m) ** d * g / (float(m) ** d + float(q) ** d * (g - 1.0))


def ddq_speedup_graded(m, d, s, q):
    """Left-hand side of Eq. ddqS: the numerator of d/dq of speedup_graded
    (its sign is the sign of the derivative)."""
    g = (q + 1.0) ** s - q**s
    gp = (q + 1.0) ** (s - 1) - q ** (s - 1)
    md = float(m) ** d
    return (s * gp * (md + q**d * (g - 1.0))
            - g * q ** (d - 1) * (d * (g - 1.0) + s * q * gp))


def q_opt_graded(m, d, s):
    """Integer number of fine layers q in [1, m] with the largest speed-up."""
    return max(range(1, int(m) + 1), key=lambda q: speedup_graded(m, d, s, q))


def graded_rates(d, s, k=1):
    """Cost exponents of Cor. cor:totalcostLFgraded and the rate of the
    speed-up in Eq. Qeff_graded for beta < s + d^2/(d+s-1):
    (gamma_LF, gamma_LTS, exponent e of S = O(eps^-e)), k the order."""
    g_lf = s + d
    g_lts = s + d * d / (d + s - 1.0)
    return g_lf, g_lts, d * (s - 1.0) / ((k + 1.0) * (s + d - 1.0))
