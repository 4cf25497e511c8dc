"""The random-width channel workload (Sec. 4.3): the reference mesh, the vertex
map of Eq. MeshTransform and the oracle on the mapped meshes, pinned by what
geometry and the method fix: the mesh tiles the domain exactly, the map
moves only |x| < 0.1 and puts the walls at +-b/2, the line mean is exact for
linear functions, the solution on a mapped mesh conserves the lumped mass
integral (Neumann boundary, v0 = 0: 1^T K = 0), and LF-LTS with the
substeps the narrowest draw needs agrees with tiny-step leapfrog."""
import numpy as np
import pytest

from oracle.lts import solve_sample
from workload.channel import (B_BAR, CONFIG_CHANNEL, bump_pulse, channel_level, channel_mesh,
                              displacement_mode, line_mean_weights, warped_xy, xi_width)


def _areas(xy, tri):
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    return 0.5 * ((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1]))


@pytest.mark.parametrize("n0,level", [(20, 0), (60, 0)])
def test_channel_mesh_tiles_the_domain(n0, level):
    m = channel_mesh(n0, level)
    A = _areas(m.xy, m.tri)
    assert (A > 0).all()
    # two 0.95 x 1 rectangles and a 0.1 x bbar channel
    assert abs(A.sum() - (2 * 0.95 + 0.1 * B_BAR)) < 1e-12
    e = np.sort(np.concatenate([m.tri[:, [0, 1]], m.tri[:, [1, 2]], m.tri[:, [2, 0]]]), axis=1)
    edges, count = np.unique(e, axis=0, return_counts=True)
    assert count.max() == 2  # conforming: no edge in three triangles
    mid = m.xy[edges[count == 1]].mean(axis=1)
    x, y = np.abs(mid[:, 0]), np.abs(mid[:, 1])
    on_boundary = ((np.abs(x - 1) < 1e-12) | (np.abs(y - 0.5) < 1e-12)
                   | ((np.abs(x - 0.05) < 1e-12) & (y >= 0.5 * B_BAR - 1e-12))
                   | ((np.abs(y - 0.5 * B_BAR) < 1e-12) & (x <= 0.05 + 1e-12)))
    assert on_boundary.all()  # every unshared edge lies on the domain's boundary
    assert m.dirichlet.sum() == 0 and m.P.sum() > 0


@pytest.mark.parametrize("b", [0.001, 0.0025, 0.004, 0.007])
def test_map_moves_the_walls_and_nothing_far_away(b):
    m = channel_mesh(20, 0)
    D = displacement_mode(m)
    xi = 0.5 * (b - B_BAR)
    w = warped_xy(m, D, xi)
    far = np.abs(m.xy[:, 0]) >= 0.1
    assert np.array_equal(w[far], m.xy[far])
    assert np.array_equal(w[:, 0], m.xy[:, 0])
    wall = (np.abs(m.xy[:, 0]) <= 0.05) & (np.abs(np.abs(m.xy[:, 1]) - 0.5 * B_BAR) < 1e-12)
    assert wall.any() and np.allclose(np.abs(w[wall, 1]), 0.5 * b, rtol=0, atol=1e-15)
    A = _areas(w, m.tri)
    assert (A > 0).all()  # no element folds over
    cen = m.xy[m.tri].mean(axis=1)
    channel = (np.abs(cen[:, 0]) < 0.05)
    assert abs(A[channel].sum() - 0.1 * b) < 1e-15
    assert abs(A.sum() - _areas(m.xy, m.tri).sum() - 0.1 * (b - B_BAR)) < 1e-10 or b == B_BAR


def test_line_mean_is_exact_for_linear_functions():
    m = channel_mesh(20, 1)
    idx, w = line_mean_weights(m, -0.4)
    u = 0.7 + 1.3 * m.xy[:, 0] - 2.1 * m.xy[:, 1]
    # mean over y in [-0.5, 0.5] of 0.7 + 1.3 x - 2.1 y at x = -0.4
    assert abs(w @ u[idx] - (0.7 - 0.52)) < 1e-14


def test_width_draws_are_uniform_and_prefix_stable():
    xi = xi_width(6, 0, 20000)
    b = 2 * xi[:, 0] + B_BAR
    assert b.min() >= 0.001 and b.max() <= 0.007
    assert abs(b.mean() - 0.004) < 5 * 0.006 / np.sqrt(12 * 20000)  # five standard errors
    assert np.array_equal(xi_width(6, 0, 50), xi[:50])


@pytest.fixture(scope="module")
def small():
    lev = channel_level(CONFIG_CHANNEL, 0, n0=20)
    return lev


def _solve(lev, xy, scheme="lts", dt=None, n=None, p=None):
    m = lev["mesh"]
    return solve_sample(xy, m.tri, m.dirichlet, m.P, lev["psi"], np.zeros(1), lev["u0"],
                        lev["dt"] if dt is None else dt, lev["n_steps"] if n is None else n,
                        lev["p"] if p is None else p, lev["nu"], scheme=scheme)


@pytest.mark.parametrize("b", [0.001, 0.007])
def test_oracle_conserves_the_mass_integral_on_a_mapped_mesh(small, b):
    """Neumann boundary and v0 = 0: sum_i m_i u_i(t) stays sum_i m_i u0_i, the
    m_i being the lumped masses of the draw's own (mapped) mesh."""
    m = small["mesh"]
    xy = warped_xy(m, displacement_mode(m), 0.5 * (b - B_BAR))
    uN = _solve(small, xy)
    A = _areas(xy, m.tri)
    mass = np.zeros(m.n_nodes)
    for a in range(3):
        np.add.at(mass, m.tri[:, a], A / 3.0)
    # rounding of about 3,200 substeps of FP64 sums (measured 3e-10 relative);
    # masses of the unmapped mesh miss by 1e-4 and more
    assert abs(mass @ uN - mass @ small["u0"]) < 1e-9 * (mass @ np.abs(small["u0"]))
    assert np.abs(uN).max() < 2.0 * np.abs(small["u0"]).max()  # stable with p = 100 at b = 0.001


def test_oracle_lts_agrees_with_tiny_step_leapfrog_on_the_narrowest_draw(small):
    """Brute force on b = 0.001 over a quarter of the horizon: leapfrog with
    dt / (4 p) everywhere against LF-LTS with p = 100 substeps, at the coarse
    step and at half of it: the difference is the second-order time error of
    LF-LTS (8 % at this coarse mesh's CFL step, 1.8 % at half the step)."""
    m = small["mesh"]
    xy = warped_xy(m, displacement_mode(m), 0.5 * (0.001 - B_BAR))
    n = small["n_steps"] // 4
    u_ref = _solve(small, xy, scheme="lf", dt=small["dt"] / (4 * small["p"]), n=n * 4 * small["p"])
    e1 = np.linalg.norm(_solve(small, xy, n=n) - u_ref) / np.linalg.norm(u_ref)
    e2 = np.linalg.norm(_solve(small, xy, dt=small["dt"] / 2, n=2 * n) - u_ref) / np.linalg.norm(u_ref)
    assert e1 < 0.1 and e2 < e1 / 3.5


def test_unmapped_draw_is_the_reference_problem(small):
    m = small["mesh"]
    xy = warped_xy(m, displacement_mode(m), 0.0)
    assert np.array_equal(xy, m.xy)
    assert abs(bump_pulse(m).max() - 1.0) < 1e-12 or bump_pulse(m).max() <= 1.0
