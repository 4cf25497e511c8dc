"""Pins of the oracle's P1 geometry, lumped mass and stiffness (no GPU)."""
import numpy as np
import pytest

from oracle.fem import barycentric_gradients, coefficient, lumped_mass, stiffness
from workload import psi_sine, square_mesh


def test_reference_triangle_gradients():
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2]])
    area, g = barycentric_gradients(xy, tri)
    assert area[0] == 0.5
    np.testing.assert_allclose(g[0], [[-1, -1], [1, 0], [0, 1]], atol=0)
    K = stiffness(xy, tri, np.ones(1)).toarray()
    # textbook element matrix of the reference triangle
    np.testing.assert_allclose(K, 0.5 * np.array([[2, -1, -1], [-1, 1, 0], [-1, 0, 1]]), atol=1e-15)


def test_clockwise_triangle_rejected():
    xy = np.array([[0.0, 0.0], [0.0, 1.0], [1.0, 0.0]])
    with pytest.raises(ValueError):
        barycentric_gradients(xy, np.array([[0, 1, 2]]))


@pytest.mark.parametrize("p", [1, 2, 4])
def test_mass_and_stiffness_invariants(p):
    m = square_mesh(12, box=(0.35, 0.65, 0.35, 0.65), p=p)
    mass = lumped_mass(m.xy, m.tri)
    assert mass.sum() == pytest.approx(1.0, rel=1e-13)     # |D| = 1
    c2 = coefficient(psi_sine(m, 4), np.array([0.3, -0.7, 0.9, -0.2]))
    K = stiffness(m.xy, m.tri, c2)
    assert abs(K - K.T).max() < 1e-13 * abs(K).max()
    # constants are in the kernel (row sums vanish)
    assert np.abs(K @ np.ones(m.n_nodes)).max() < 1e-12 * abs(K).max()
    # linear functions: K u vanishes at interior nodes when c is constant
    Kc = stiffness(m.xy, m.tri, np.ones(m.n_tri))
    u = 2.0 * m.xy[:, 0] - 3.0 * m.xy[:, 1]
    r = Kc @ u
    interior = ~m.dirichlet.astype(bool)
    assert np.abs(r[interior]).max() < 1e-11
    # energy of a linear function: u^T K u = |grad u|^2 |D|
    assert u @ (Kc @ u) == pytest.approx(13.0, rel=1e-12)


def test_coefficient_is_exp_of_field():
    psi = np.array([[0.0, 0.0], [1.0, 0.5], [-1.0, 2.0]])
    xi = np.array([0.25, -0.5])
    np.testing.assert_allclose(coefficient(psi, xi), [1.0, np.exp(0.0), np.exp(-1.25)], rtol=1e-15)
