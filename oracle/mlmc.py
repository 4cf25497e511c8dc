"""Multilevel Monte Carlo estimator and adaptive driver, FP64 (oracle; test
infrastructure only).  Sec. 2.2 of the paper.

* estimator (Eq. MLMCestimator): Q^ML = sum_l N_l^{-1} sum_i dQ_l(w^{(i,l)}),
  dQ_0 = Q_0 and dQ_l = Q_l - Q_{l-1} evaluated on the same draw w^{(i,l)};
* variance estimate (Eq. Vell_est):
  V_l ~ (sum_i |dQ_l|^2 - |sum_i dQ_l|^2 / N_l) / (N_l - 1);
* optimal sample numbers (Eq. optimal_Nl):
  N_l >= 2 / eps^2 * sqrt(V_l / C_l) * sum_l' sqrt(V_l' C_l');
* bias estimate (Eq. bias_est): E[Q - Q_L] ~ E[Q_L - Q_{L-1}] / (2^alpha - 1),
  and the test |E[Q - Q_L]|^2 < eps^2 / 2;
* Alg. 1: start with L = 2, compute the missing samples, update V_l and N_l,
  add a level while the bias test fails, until no N_l grows.

Sums use math.fsum (correctly rounded), the plainest exact reference.
"""
from __future__ import annotations

import math

import numpy as np


def level_sums(Qf, Qc=None):
    """(sum dQ, sum dQ^2, sum Qf, sum Qf^2), correctly rounded."""
    Qf = np.asarray(Qf, dtype=np.float64)
    dQ = Qf - np.asarray(Qc, dtype=np.float64) if Qc is not None else Qf
    return (math.fsum(dQ), math.fsum(dQ * dQ), math.fsum(Qf), math.fsum(Qf * Qf))


def estimator(sum_dQ, N):
    """Q^ML = sum_l sum_dQ[l] / N[l]."""
    return math.fsum(s / n for s, n in zip(sum_dQ, N))


def variance(sum1, sum2, N):
    """Unbiased V_l estimate, Eq. Vell_est."""
    if N < 2:
        return float("nan")
    return (sum2 - sum1 * sum1 / N) / (N - 1)


def optimal_N(V, C, eps):
    """N_l = ceil(2/eps^2 sqrt(V_l/C_l) sum_l' sqrt(V_l' C_l')), Eq. optimal_Nl."""
    total = math.fsum(math.sqrt(v * c) for v, c in zip(V, C))
    return [int(math.ceil(2.0 / eps**2 * math.sqrt(v / c) * total)) for v, c in zip(V, C)]


def bias_estimate(mean_dQ_L, alpha):
    """|E[Q - Q_L]| estimated from the finest level difference, Eq. bias_est."""
    return abs(mean_dQ_L) / (2.0**alpha - 1.0)


def bias_test_passes(mean_dQ_L, alpha, eps):
    return bias_estimate(mean_dQ_L, alpha) ** 2 < eps**2 / 2.0


def mse_split(V, N, bias):
    """e^2 = sum_l V_l / N_l + bias^2, Eq. MSE_splitform."""
    return math.fsum(v / n for v, n in zip(V, N)) + bias**2


def alg1(sample_level, eps, cost, N_init, alpha=2.0, L_max=None, L_start=2):
    """Adaptive MLMC (Alg. 1).

    sample_level(l, offset, n) -> array of dQ_l for draws offset..offset+n-1
    cost(l) -> C_l, the cost of one sample dQ_l
    N_init(l) -> initial N_l for a newly opened level
    Returns dict(estimate, L, N, V, sums, bias, mse).
    """
    L = L_start
    N = [int(N_init(l)) for l in range(L + 1)]
    done = [0] * (L + 1)
    s1 = [0.0] * (L + 1)
    s2 = [0.0] * (L + 1)
    parts1 = [[] for _ in range(L + 1)]
    parts2 = [[] for _ in range(L + 1)]
    increased = True
    while increased:
        increased = False
        # step 2a: remaining samples on every level
        for l in range(L + 1):
            if N[l] > done[l]:
                dq = np.asarray(sample_level(l, done[l], N[l] - done[l]), dtype=np.float64)
                parts1[l].extend(dq.tolist())
                parts2[l].extend((dq * dq).tolist())
                done[l] = N[l]
                s1[l] = math.fsum(parts1[l])
                s2[l] = math.fsum(parts2[l])
        # step 2b: estimator and variances
        V = [variance(s1[l], s2[l], done[l]) for l in range(L + 1)]
        # step 2c: optimal sample numbers (never fewer than already computed)
        C = [cost(l) for l in range(L + 1)]
        Nopt = optimal_N([max(v, 0.0) for v in V], C, eps)
        for l in range(L + 1):
            if Nopt[l] > N[l]:
                N[l] = Nopt[l]
                increased = True
        # step 2d: bias test on the finest level
        mean_L = s1[L] / done[L]
        if not bias_test_passes(mean_L, alpha, eps) and (L_max is None or L < L_max):
            L += 1
            N.append(int(N_init(L)))
            done.append(0)
            s1.append(0.0)
            s2.append(0.0)
            parts1.append([])
            parts2.append([])
            increased = True
    V = [variance(s1[l], s2[l], done[l]) for l in range(L + 1)]
    bias = bias_estimate(s1[L] / done[L], alpha)
    return {"estimate": estimator(s1, done), "L": L, "N": done, "V": V,
            "sums": list(zip(s1, s2)), "bias": bias, "mse": mse_split(V, done, bias)}
