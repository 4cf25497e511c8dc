"""The graded L-shape workload (inputs) and the oracle on it (no GPU)."""
import numpy as np
import pytest

from oracle.lts import solve_sample
from workload import CONFIG_LSHAPE, lshape_level, lshape_steps, xi_gaussian
from workload.mesh import lshape_graded_mesh


@pytest.mark.parametrize("m,s,q", [(4, 1.0, 1), (10, 2.0, 2), (12, 2.0, 4)])
def test_graded_mesh_structure(m, s, q):
    mesh = lshape_graded_mesh(m, s, q)
    V = mesh.xy[mesh.tri]
    area = 0.5 * ((V[:, 1, 0] - V[:, 0, 0]) * (V[:, 2, 1] - V[:, 0, 1])
                  - (V[:, 2, 0] - V[:, 0, 0]) * (V[:, 1, 1] - V[:, 0, 1]))
    assert mesh.n_tri == 6 * m * m
    assert area.min() > 0 and area.sum() == pytest.approx(3.0, rel=1e-13)
    e = np.sort(np.concatenate([mesh.tri[:, [0, 1]], mesh.tri[:, [1, 2]], mesh.tri[:, [2, 0]]]), axis=1)
    u, c = np.unique(e, axis=0, return_counts=True)
    assert c.max() == 2 and mesh.dirichlet.astype(bool)[u[c == 1]].all()
    # layer k of every spoke sits at distance (k/m)^s from the corner
    r = np.linalg.norm(mesh.xy, axis=1)
    on_axis = np.abs(mesh.xy[:, 1]) < 1e-14
    rs = np.sort(r[on_axis & (mesh.xy[:, 0] >= 0)])
    np.testing.assert_allclose(rs, (np.arange(m + 1) / m) ** s, rtol=0, atol=1e-15)
    # refined tiers touch the corner, P contains their vertices
    assert mesh.P[mesh.tri[mesh.refined.astype(bool)]].astype(bool)[~mesh.dirichlet[mesh.tri[mesh.refined.astype(bool)]].astype(bool)].all()


def test_lshape_lts_agrees_with_tiny_step_leapfrog():
    """LF-LTS with the per-draw step vs leapfrog with a step 8p times smaller,
    Ricker source and graded mesh: the difference is the O(dt^2) LTS error."""
    lev = lshape_level(CONFIG_LSHAPE, 0, m0=4)
    lev = dict(lev, T=0.4)
    xi = xi_gaussian(3, 0, 1, CONFIG_LSHAPE.K, CONFIG_LSHAPE.sigma)
    n = int(lshape_steps(lev, xi)[0])
    m = lev["mesh"]
    args = (m.xy, m.tri, m.dirichlet, m.P, lev["psi"], xi[0], lev["u0"])
    u_lts = solve_sample(*args, lev["T"] / n, n, lev["p"], lev["nu"], source=lev["source"])
    k = 8 * lev["p"]
    u_ref = solve_sample(*args, lev["T"] / (n * k), n * k, 1, 0.0, scheme="lf", source=lev["source"])
    u_lts2 = solve_sample(*args, lev["T"] / (2 * n), 2 * n, lev["p"], lev["nu"], source=lev["source"])
    e1 = np.abs(u_lts - u_ref).max() / np.abs(u_ref).max()
    e2 = np.abs(u_lts2 - u_ref).max() / np.abs(u_ref).max()
    assert np.abs(u_ref).max() > 0
    assert e1 < 0.05 and e2 < e1 / 3
