"""P1 finite elements with mass lumping, FP64 (oracle; test infrastructure only).

Sec. 3.1 of the paper: conforming P1 elements, mass matrix M_ij = (phi_j, phi_i)
replaced by its lumped (diagonal) version, stiffness K_ij = (c grad phi_j,
c grad phi_i).  With an elementwise constant coefficient c_e^2 (one-point
centroid quadrature of the random field, which the paper evaluates "at the
quadrature nodes") the element stiffness is c_e^2 |T_e| grad(lambda_a) .
grad(lambda_b) exactly.  Nodal (vertex) quadrature of the mass gives
m_i = sum over elements containing i of |T_e| / 3.

Gradients here come from inverting the affine map of each triangle; the
stiffness is assembled by a plain scatter over the elements (scipy's COO ->
CSR sum of duplicates).  Dirichlet nodes are eliminated: the free system is
the restriction of M and K to the free nodes (u = 0 on Dirichlet nodes).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def barycentric_gradients(xy: np.ndarray, tri: np.ndarray):
    """(area[e], grad[e, a, :]) of the barycentric functions lambda_a on e.

    lambda = B^{-1} (x - x0) with B = [x1 - x0, x2 - x0]; rows of B^{-1} are
    the gradients of lambda_1 and lambda_2, lambda_0 = 1 - lambda_1 - lambda_2.
    """
    X = xy[tri]                                   # [n_tri, 3, 2]
    B = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]], axis=2)  # columns
    det = B[:, 0, 0] * B[:, 1, 1] - B[:, 0, 1] * B[:, 1, 0]
    if np.any(det <= 0):
        raise ValueError("triangles must be counter-clockwise with positive area")
    Binv = np.empty_like(B)
    Binv[:, 0, 0] = B[:, 1, 1] / det
    Binv[:, 0, 1] = -B[:, 0, 1] / det
    Binv[:, 1, 0] = -B[:, 1, 0] / det
    Binv[:, 1, 1] = B[:, 0, 0] / det
    g1, g2 = Binv[:, 0, :], Binv[:, 1, :]
    grad = np.stack([-g1 - g2, g1, g2], axis=1)   # [n_tri, 3, 2]
    return 0.5 * det, grad


def lumped_mass(xy: np.ndarray, tri: np.ndarray) -> np.ndarray:
    """Diagonal of the lumped mass matrix, m_i = sum_{e ni i} |T_e| / 3."""
    area, _ = barycentric_gradients(xy, tri)
    m = np.zeros(xy.shape[0])
    for a in range(3):
        np.add.at(m, tri[:, a], area / 3.0)
    return m


def coefficient(psi: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """Element values c_e^2 = exp(sum_k xi_k psi_{e,k}) of the log-field."""
    return np.exp(psi @ xi)


def stiffness(xy: np.ndarray, tri: np.ndarray, c2: np.ndarray) -> sp.csr_matrix:
    """K_ij = sum_e c_e^2 |T_e| grad(lambda_j) . grad(lambda_i) (full, all nodes)."""
    area, grad = barycentric_gradients(xy, tri)
    rows, cols, vals = [], [], []
    for a in range(3):
        for b in range(3):
            rows.append(tri[:, a])
            cols.append(tri[:, b])
            vals.append(c2 * area * (grad[:, a, :] * grad[:, b, :]).sum(axis=1))
    n = xy.shape[0]
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    K.sum_duplicates()
    return K


def free_system(xy, tri, dirichlet, c2):
    """(free index array, lumped mass on free nodes, K restricted to free nodes)."""
    free = np.nonzero(~dirichlet.astype(bool))[0]
    m = lumped_mass(xy, tri)[free]
    K = stiffness(xy, tri, c2)[free][:, free].tocsr()
    return free, m, K
