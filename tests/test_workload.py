"""Checks of the seeded input generators (meshes, masks, QoI weights, draws)."""
import numpy as np
import pytest

from workload import (CONFIG_BATCHED, CONFIG_PLAIN, box_qoi_weights, coarse_dt,
                      level_problem, square_mesh, xi_uniform)


def _edges(tri):
    e = np.sort(np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]]), axis=1)
    return np.unique(e, axis=0, return_counts=True)


@pytest.mark.parametrize("n,p", [(8, 1), (8, 2), (16, 4), (32, 8)])
def test_mesh_conforming_and_oriented(n, p):
    box = (0.3, 0.7, 0.3, 0.7) if n <= 8 else (0.45, 0.55, 0.45, 0.55)
    m = square_mesh(n, box=box, p=p)
    V = m.xy[m.tri]
    area = 0.5 * ((V[:, 1, 0] - V[:, 0, 0]) * (V[:, 2, 1] - V[:, 0, 1])
                  - (V[:, 2, 0] - V[:, 0, 0]) * (V[:, 1, 1] - V[:, 0, 1]))
    assert area.min() > 0
    assert area.sum() == pytest.approx(1.0, rel=1e-13)
    u, c = _edges(m.tri)
    assert c.max() == 2
    bnd = u[c == 1]
    onb = m.dirichlet.astype(bool)
    assert onb[bnd].all(), "a boundary edge off the square boundary means a hanging node"
    # every node is used
    assert np.unique(m.tri).size == m.n_nodes
    # no duplicated coordinates
    assert np.unique(np.round(m.xy * n * p).astype(np.int64), axis=0).shape[0] == m.n_nodes


def test_refinement_mask_rule():
    m = square_mesh(16, box=(0.4, 0.6, 0.4, 0.6), p=4)
    ref = m.refined.astype(bool)
    v1 = np.zeros(m.n_nodes, bool)
    v1[m.tri[ref].ravel()] = True
    touching = v1[m.tri].any(axis=1)
    expect = np.zeros(m.n_nodes, bool)
    expect[m.tri[touching].ravel()] = True
    expect &= ~m.dirichlet.astype(bool)
    assert (m.P.astype(bool) == expect).all()
    # every small element is refined; refined elements lie in the box or its ring
    V = m.xy[m.tri]
    emin = np.min([np.linalg.norm(V[:, i] - V[:, (i + 1) % 3], axis=1) for i in range(3)], axis=0)
    assert ref[emin < 0.99 * m.H].all()
    x0, x1, y0, y1 = m.box
    c = V[ref].mean(axis=1)
    assert ((c[:, 0] > x0 - m.H) & (c[:, 0] < x1 + m.H) & (c[:, 1] > y0 - m.H) & (c[:, 1] < y1 + m.H)).all()


def test_qoi_weights_exact_for_linear_functions():
    for n, p in ((16, 1), (16, 4)):
        m = square_mesh(n, box=(0.4, 0.6, 0.4, 0.6), p=p)
        for box in ((0.7, 0.8, 0.7, 0.8), (0.63, 0.81, 0.22, 0.57)):
            idx, g = box_qoi_weights(m, box)
            assert g.sum() == pytest.approx(1.0, rel=1e-13)
            u = 1.5 + 2.0 * m.xy[:, 0] - 0.5 * m.xy[:, 1]
            cx, cy = (box[0] + box[1]) / 2, (box[2] + box[3]) / 2
            assert g @ u[idx] == pytest.approx(1.5 + 2 * cx - 0.5 * cy, rel=1e-13)


def test_qoi_weights_against_monte_carlo_integral():
    """Independent check: average of the P1 interpolant at random box points."""
    m = square_mesh(12, box=(0.4, 0.6, 0.4, 0.6), p=2)
    box = (0.63, 0.81, 0.22, 0.57)
    idx, g = box_qoi_weights(m, box)
    rng = np.random.default_rng(5)
    u = rng.standard_normal(m.n_nodes)
    u[m.dirichlet.astype(bool)] = 0
    pts = np.column_stack([rng.uniform(box[0], box[1], 200000), rng.uniform(box[2], box[3], 200000)])
    # locate points by brute force over candidate triangles near the box
    V = m.xy[m.tri]
    lo, hi = V.min(1), V.max(1)
    cand = np.nonzero((hi[:, 0] >= box[0]) & (lo[:, 0] <= box[1]) & (hi[:, 1] >= box[2]) & (lo[:, 1] <= box[3]))[0]
    vals = np.full(pts.shape[0], np.nan)
    for e in cand:
        T = V[e]
        Mx = np.array([[T[1, 0] - T[0, 0], T[2, 0] - T[0, 0]], [T[1, 1] - T[0, 1], T[2, 1] - T[0, 1]]])
        l = np.linalg.solve(Mx, (pts - T[0]).T).T
        lam = np.column_stack([1 - l.sum(1), l])
        ins = (lam >= -1e-12).all(1)
        vals[ins] = lam[ins] @ u[m.tri[e]]
    assert not np.isnan(vals).any()
    assert g @ u[idx] == pytest.approx(vals.mean(), abs=3e-3 * np.abs(u).max())


def test_xi_rows_independent_of_batch_split():
    a = xi_uniform(7, 2, 10, 8)
    b = xi_uniform(7, 2, 4, 8, offset=6)
    np.testing.assert_array_equal(a[6:], b)
    assert a.min() >= -1 and a.max() <= 1
    assert not np.allclose(xi_uniform(7, 3, 10, 8), a)


def test_level_hierarchy_keeps_box_and_halves_h():
    l0 = level_problem(CONFIG_PLAIN, 0)
    l1 = level_problem(CONFIG_PLAIN, 1)
    assert l0["mesh"].box == l1["mesh"].box
    assert l1["mesh"].H == l0["mesh"].H / 2
    assert l1["n_steps"] >= 2 * l0["n_steps"] - 1
    dt, n = coarse_dt(1 / 128, 8, 1.0)
    assert n == 432 and dt * n == pytest.approx(1.0)
    assert CONFIG_BATCHED.levels == 5
