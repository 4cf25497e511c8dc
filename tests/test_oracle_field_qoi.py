"""Pins of the L2(D)-valued QoI oracle (oracle/field_qoi.py) against what the
mathematics fixes: nodal interpolation reproduces linear functions exactly
and copies shared nodes, its rows are a partition of unity; on nested
meshes it embeds the coarse space (the L2 norm is kept); the consistent mass
matrix integrates products of P1 functions exactly (area, first and second
moments of the unit square and of the L-shape) and its row sums are the
lumped mass of oracle/fem.py; the V-norm variance of Eq. Vell_est equals the
definition (1/(N-1)) sum ||dU_i - mean||^2; the MLMC field estimate
telescopes to the finest level's mean when every level uses the same draws."""
import math

import numpy as np
import pytest

from oracle.fem import lumped_mass
from oracle.field_qoi import (field_bias_estimate, field_mean_and_variance, field_sums,
                              interpolation_matrix, l2_norm2, mass_matrix, mlmc_field_estimate)
from workload import lshape_graded_mesh, square_mesh


def _lin(xy, a=0.3, b=-1.7, c=2.2):
    return a + b * xy[:, 0] + c * xy[:, 1]


@pytest.mark.parametrize("coarse,fine", [
    (dict(n=4), dict(n=8)),
    (dict(n=8, box=(0.375, 0.625, 0.375, 0.625), p=2), dict(n=16, box=(0.375, 0.625, 0.375, 0.625), p=2)),
    (dict(n=5), dict(n=7)),                       # not nested
])
def test_interpolation_is_exact_for_linear_functions(coarse, fine):
    mc, mf = square_mesh(**coarse), square_mesh(**fine)
    I = interpolation_matrix(mc.xy, mc.tri, mf.xy)
    np.testing.assert_allclose(I @ _lin(mc.xy), _lin(mf.xy), rtol=0, atol=1e-13)
    np.testing.assert_allclose(np.asarray(I.sum(axis=1)).ravel(), 1.0, rtol=0, atol=1e-13)
    assert I.data.min() >= -1e-10 and I.data.max() <= 1 + 1e-10
    # nodes present on both meshes copy the coarse value
    key = {tuple(np.round(x, 12)): i for i, x in enumerate(mc.xy)}
    u = np.random.default_rng(1).normal(size=mc.n_nodes)
    v = I @ u
    for j, x in enumerate(mf.xy):
        i = key.get(tuple(np.round(x, 12)))
        if i is not None:
            assert v[j] == pytest.approx(u[i], abs=1e-13)


def test_nested_meshes_keep_the_l2_norm():
    mc, mf = square_mesh(6), square_mesh(12)
    I = interpolation_matrix(mc.xy, mc.tri, mf.xy)
    u = np.random.default_rng(2).normal(size=mc.n_nodes)
    assert l2_norm2(mass_matrix(mf.xy, mf.tri), I @ u) == pytest.approx(
        l2_norm2(mass_matrix(mc.xy, mc.tri), u), rel=1e-12)


def test_mass_matrix_integrates_p1_products_exactly():
    m = square_mesh(9, box=(0.3, 0.7, 0.3, 0.7), p=3)
    M = mass_matrix(m.xy, m.tri)
    one, x, y = np.ones(m.n_nodes), m.xy[:, 0], m.xy[:, 1]
    assert one @ (M @ one) == pytest.approx(1.0, rel=1e-13)          # area
    assert one @ (M @ x) == pytest.approx(0.5, rel=1e-13)            # int x
    assert x @ (M @ x) == pytest.approx(1.0 / 3.0, rel=1e-13)        # int x^2
    assert x @ (M @ y) == pytest.approx(0.25, rel=1e-13)             # int x y
    np.testing.assert_allclose(np.asarray(M.sum(axis=1)).ravel(), lumped_mass(m.xy, m.tri), rtol=1e-13)
    L = lshape_graded_mesh(6, 2.0, 2)
    ML = mass_matrix(L.xy, L.tri)
    one = np.ones(L.n_nodes)
    assert one @ (ML @ one) == pytest.approx(3.0, rel=1e-12)         # |[-1,1]^2 minus a quarter|
    # int x over the L-shape: squares [-1,0]x[-1,1] (-1), [0,1]x[0,1] (+1/2)
    assert one @ (ML @ L.xy[:, 0]) == pytest.approx(-0.5, rel=1e-12)


def test_vell_est_equals_the_sample_variance_in_the_norm():
    m = square_mesh(5)
    M = mass_matrix(m.xy, m.tri)
    dU = np.random.default_rng(3).normal(size=(11, m.n_nodes))
    s1, s2 = field_sums(dU, M)
    mean, V = field_mean_and_variance(s1, s2, dU.shape[0], M)
    direct = math.fsum(l2_norm2(M, u - dU.mean(axis=0)) for u in dU) / (dU.shape[0] - 1)
    np.testing.assert_allclose(mean, dU.mean(axis=0), rtol=1e-13)
    assert V == pytest.approx(direct, rel=1e-11)


def test_mlmc_field_estimate_telescopes_on_shared_draws():
    """With the same draws on every level, sum_l I_{l->L} mean(u_l - I u_{l-1})
    equals the mean of u_L (nested meshes, fields of the draws)."""
    meshes = [square_mesh(4 * 2**l) for l in range(3)]
    rng = np.random.default_rng(4)
    w = rng.normal(size=(7, 3))

    def field(m, wk):  # a smooth random field sampled at the nodes
        x, y = m.xy[:, 0], m.xy[:, 1]
        return wk[0] * np.sin(np.pi * x) * np.sin(np.pi * y) + wk[1] * x * y + wk[2]

    Ip = [None] + [interpolation_matrix(meshes[l - 1].xy, meshes[l - 1].tri, meshes[l].xy) for l in (1, 2)]
    means = []
    for l, m in enumerate(meshes):
        M = mass_matrix(m.xy, m.tri)
        U = np.array([field(m, wk) for wk in w])
        dU = U if l == 0 else U - np.array([Ip[l] @ field(meshes[l - 1], wk) for wk in w])
        s1, s2 = field_sums(dU, M)
        means.append(field_mean_and_variance(s1, s2, len(w), M)[0])
    to_finest = [Ip[2] @ Ip[1], Ip[2], None]
    est = mlmc_field_estimate(means, to_finest)
    np.testing.assert_allclose(est, np.mean([field(meshes[2], wk) for wk in w], axis=0), rtol=0, atol=1e-13)
    ML = mass_matrix(meshes[2].xy, meshes[2].tri)
    b = field_bias_estimate(means[2], ML, 2.0)
    assert b == pytest.approx(math.sqrt(l2_norm2(ML, means[2])) / 3.0, rel=1e-15)


def test_alg1_field_reduces_to_the_scalar_driver():
    """V = R (one node, M = [1]): the field driver takes the scalar driver's
    decisions and returns its estimate."""
    import scipy.sparse as sp

    from oracle.field_qoi import alg1_field
    from oracle.mlmc import alg1

    rng = np.random.default_rng(7)
    table = {l: rng.normal(2.0**(-2 * l), 2.0**(-1.5 * l), size=20000) for l in range(6)}

    def sample(l, off, n):
        return table[l][off:off + n]

    kw = dict(eps=2e-3, cost=lambda l: 4.0**l, N_init=lambda l: 32, alpha=2.0, L_max=5)
    a = alg1(sample, **kw)
    b = alg1_field(lambda l, off, n: sample(l, off, n)[:, None], mass=lambda l: sp.identity(1, format="csr"),
                   to_finest=lambda l, L: None, **kw)
    assert b["L"] == a["L"] and b["N"] == a["N"]
    assert b["estimate"][0] == pytest.approx(a["estimate"], rel=1e-13, abs=1e-15)
    np.testing.assert_allclose(b["V"], a["V"], rtol=1e-10)


def test_alg1_field_meets_its_tolerance_on_a_known_mean():
    """Nested meshes, u_l = nodal values of f(x) + w1 g(x) + 4^-l w2 h(x) with
    E w = 0: E[u_L] = f at the nodes of mesh L; the driver's estimate lies
    within three of its own RMSE estimates of it in the L2 norm."""
    from oracle.field_qoi import alg1_field

    meshes = [square_mesh(4 * 2**l) for l in range(5)]
    Ms = [mass_matrix(m.xy, m.tri) for m in meshes]
    Ip = {}

    def to_finest(l, L):
        if l == L:
            return None
        if (l, L) not in Ip:
            Ip[(l, L)] = interpolation_matrix(meshes[l].xy, meshes[l].tri, meshes[L].xy)
        return Ip[(l, L)]

    def u(m, l, w):
        x, y = m.xy[:, 0], m.xy[:, 1]
        return (np.sin(np.pi * x) * np.sin(np.pi * y) + w[0] * x * (1 - x)
                + 4.0**(-l) * w[1] * np.cos(3 * x) * y)

    W = np.random.default_rng(11).normal(size=(5, 4000, 2))

    def sample(l, off, n):
        m = meshes[l]
        rows = []
        for i in range(off, off + n):
            d = u(m, l, W[l, i])
            if l > 0:
                d = d - to_finest(l - 1, l) @ u(meshes[l - 1], l - 1, W[l, i])
            rows.append(d)
        return np.array(rows)

    r = alg1_field(sample, eps=0.05, cost=lambda l: 4.0**l, N_init=lambda l: 16,
                   mass=lambda l: Ms[l], to_finest=to_finest, alpha=2.0, L_max=4)
    L = r["L"]
    x, y = meshes[L].xy[:, 0], meshes[L].xy[:, 1]
    err = math.sqrt(l2_norm2(Ms[L], r["estimate"] - np.sin(np.pi * x) * np.sin(np.pi * y)))
    assert r["mse"] <= 0.05**2 * 1.5
    assert err <= 3 * math.sqrt(r["mse"])
