"""L2(D)-valued QoI and vector MLMC, FP64 (oracle; test infrastructure only).

The paper's experiments estimate E[u(., T)] in V = L2(D) (Sec. 4); the MSE
is taken in the V-norm (Eq. errordef), the estimator is the sum of the level
means of dQ_l (Eq. MLMCestimator), the level variances are estimated in the
V-norm (Eq. Vell_est) and the bias from the last level mean (Eq. bias_est).

On level l a draw's QoI is the P1 function u_l(., T) on that level's mesh.
The paper does not say how a difference of functions on two meshes is
formed; here (reading): dQ_l = u_l - I u_{l-1} on the finer mesh of the pair,
I the nodal interpolation of the coarse P1 function at the fine mesh's
nodes (exact for linear functions, an exact embedding when the meshes are
nested), and the level means are interpolated to the finest mesh before
they are summed.  Norms are the exact integrals of P1 functions (consistent
mass matrix, |T|/12 (1 + delta_ab) per element).

Point location is brute force (every node against every triangle): plain
and slow, for the small meshes of the tests.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .fem import barycentric_gradients


def barycentric(xy_tri: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """lambda[point, triangle, a] of every point in every triangle (vertices
    xy_tri [n_tri, 3, 2]), from x = x0 + (x1 - x0) l1 + (x2 - x0) l2."""
    x0 = xy_tri[:, 0]
    e1 = xy_tri[:, 1] - x0
    e2 = xy_tri[:, 2] - x0
    det = e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]
    d = pts[:, None, :] - x0[None, :, :]
    l1 = (d[..., 0] * e2[None, :, 1] - d[..., 1] * e2[None, :, 0]) / det[None, :]
    l2 = (e1[None, :, 0] * d[..., 1] - e1[None, :, 1] * d[..., 0]) / det[None, :]
    return np.stack([1.0 - l1 - l2, l1, l2], axis=2)


def interpolation_matrix(xy_c: np.ndarray, tri_c: np.ndarray, xy_f: np.ndarray,
                         tol: float = 1e-10, chunk: int = 256) -> sp.csr_matrix:
    """I [n_f, n_c]: (I u_c)_i = u_c evaluated at fine node i (the P1 function
    on the coarse mesh; a node on an edge or vertex takes any triangle that
    contains it, the value is the same by continuity)."""
    X = xy_c[tri_c]
    rows, cols, vals = [], [], []
    for s in range(0, xy_f.shape[0], chunk):
        pts = xy_f[s:s + chunk]
        lam = barycentric(X, pts)                       # [n_pts, n_tri, 3]
        worst = lam.min(axis=2)
        t = worst.argmax(axis=1)                        # the most interior triangle
        if np.any(worst[np.arange(pts.shape[0]), t] < -tol):
            raise ValueError("a fine node lies outside the coarse mesh")
        w = lam[np.arange(pts.shape[0]), t]             # [n_pts, 3]
        for a in range(3):
            rows.append(np.arange(s, s + pts.shape[0]))
            cols.append(tri_c[t, a])
            vals.append(w[:, a])
    I = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(xy_f.shape[0], xy_c.shape[0])).tocsr()
    I.sum_duplicates()
    return I


def mass_matrix(xy: np.ndarray, tri: np.ndarray) -> sp.csr_matrix:
    """Consistent P1 mass matrix M_ij = (phi_j, phi_i)_{L2(D)} (Sec. 3.1,
    before lumping): |T|/12 (1 + delta_ab) on every element."""
    area, _ = barycentric_gradients(xy, tri)
    rows, cols, vals = [], [], []
    for a in range(3):
        for b in range(3):
            rows.append(tri[:, a])
            cols.append(tri[:, b])
            vals.append(area * (2.0 if a == b else 1.0) / 12.0)
    n = xy.shape[0]
    M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    M.sum_duplicates()
    return M


def l2_norm2(M: sp.csr_matrix, v: np.ndarray) -> float:
    """||v||^2_{L2(D)} = v^T M v of a P1 function given by its nodal values."""
    return float(v @ (M @ v))


def field_sums(dU: np.ndarray, M: sp.csr_matrix):
    """Sums of one level's draws dU [N, n] (nodal vectors on that level's
    mesh): (sum_i dU_i [n], sum_i ||dU_i||^2) with math.fsum."""
    s1 = np.array([math.fsum(dU[:, j]) for j in range(dU.shape[1])])
    s2 = math.fsum(l2_norm2(M, u) for u in dU)
    return s1, s2


def field_mean_and_variance(s1: np.ndarray, s2: float, N: int, M: sp.csr_matrix):
    """Level mean sum_i dU_i / N (Eq. MLMCestimator) and the V-norm variance
    estimate of Eq. Vell_est: (sum ||dU_i||^2 - ||sum dU_i||^2 / N) / (N - 1)."""
    mean = s1 / N
    V = (s2 - l2_norm2(M, s1) / N) / (N - 1) if N > 1 else float("nan")
    return mean, V


def mlmc_field_estimate(means: list, to_finest: list) -> np.ndarray:
    """sum_l I_{l -> L} mean_l: the level means carried to the finest mesh
    (to_finest[l]: interpolation matrix from mesh l to mesh L, None for L)."""
    out = None
    for mean, I in zip(means, to_finest):
        v = mean if I is None else I @ mean
        out = v.copy() if out is None else out + v
    return out


def field_bias_estimate(mean_L: np.ndarray, M_L: sp.csr_matrix, alpha: float) -> float:
    """Eq. bias_est in the V-norm (alpha the rate of ||E dQ_l||, as for the
    scalar QoI): ||mean dQ_L|| / (2^alpha - 1)."""
    return math.sqrt(l2_norm2(M_L, mean_L)) / (2.0**alpha - 1.0)


def alg1_field(sample_level, eps, cost, N_init, mass, to_finest, alpha=2.0, L_max=None, L_start=2):
    """Alg. 1 for a V-valued QoI (V = L2(D)), with the steps of the scalar
    driver: the missing samples of every level, V_l by Eq. Vell_est in the
    V-norm, N_l by Eq. optimal_Nl (never decreased), a new level while the
    bias test of Eq. bias_est fails in the V-norm.

    sample_level(l, offset, n) -> dU [n, n_nodes_l], nodal differences on
        level l's mesh for draws offset..offset+n-1
    cost(l) -> C_l;  N_init(l) -> initial N_l;  mass(l) -> M_l
    to_finest(l, L) -> interpolation matrix from mesh l to mesh L (None if l == L)
    Returns dict(estimate [n_nodes_L], L, N, V, bias, mse).
    """
    from . import mlmc as scalar

    L = L_start
    N = [int(N_init(l)) for l in range(L + 1)]
    draws = [[] for _ in range(L + 1)]
    done = [0] * (L + 1)
    increased = True
    while increased:
        increased = False
        for l in range(L + 1):
            if N[l] > done[l]:
                draws[l].extend(np.asarray(sample_level(l, done[l], N[l] - done[l]), dtype=np.float64))
                done[l] = N[l]
        stats = [field_mean_and_variance(*field_sums(np.array(draws[l]), mass(l)), done[l], mass(l))
                 for l in range(L + 1)]
        V = [v for _, v in stats]
        C = [cost(l) for l in range(L + 1)]
        Nopt = scalar.optimal_N([max(v, 0.0) for v in V], C, eps)
        for l in range(L + 1):
            if Nopt[l] > N[l]:
                N[l] = Nopt[l]
                increased = True
        if field_bias_estimate(stats[L][0], mass(L), alpha) ** 2 >= eps**2 / 2.0 and (L_max is None or L < L_max):
            L += 1
            N.append(int(N_init(L)))
            draws.append([])
            done.append(0)
            increased = True
    stats = [field_mean_and_variance(*field_sums(np.array(draws[l]), mass(l)), done[l], mass(l))
             for l in range(L + 1)]
    V = [v for _, v in stats]
    bias = field_bias_estimate(stats[L][0], mass(L), alpha)
    est = mlmc_field_estimate([m for m, _ in stats], [to_finest(l, L) for l in range(L + 1)])
    return {"estimate": est, "L": L, "N": done, "V": V, "bias": bias, "mse": scalar.mse_split(V, done, bias)}
