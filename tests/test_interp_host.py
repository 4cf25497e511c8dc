"""lflts_interp_weights (host only, no GPU) against the oracle's nodal
interpolation (oracle/field_qoi.py): the same values of coarse P1 functions
at the fine nodes on nested and non-nested square meshes, on meshes with a
refined box and on graded L-shapes; weights are barycentric (sum 1, within
[0, 1] up to rounding); nodes outside the coarse mesh and bad vertex ids are
refused."""
import numpy as np
import pytest

from oracle.field_qoi import interpolation_matrix
from workload import lshape_graded_mesh, square_mesh


@pytest.fixture(scope="module")
def lib():
    from paper_2106_11117_gb300 import build, lflts
    build.build()
    return lflts


CASES = [
    (lambda: square_mesh(4), lambda: square_mesh(8)),
    (lambda: square_mesh(5), lambda: square_mesh(7)),
    (lambda: square_mesh(8, box=(0.375, 0.625, 0.375, 0.625), p=2),
     lambda: square_mesh(16, box=(0.375, 0.625, 0.375, 0.625), p=2)),
    (lambda: square_mesh(8, box=(0.375, 0.625, 0.375, 0.625), p=4), lambda: square_mesh(13)),
    (lambda: lshape_graded_mesh(4, 2.0, 1), lambda: lshape_graded_mesh(8, 2.0, 2)),
]


@pytest.mark.parametrize("k", range(len(CASES)))
def test_interp_weights_match_the_oracle(lib, k):
    mc, mf = CASES[k][0](), CASES[k][1]()
    vert, w = lib.lflts_interp_weights(mc.xy, mc.tri, mf.xy)
    np.testing.assert_allclose(w.sum(axis=1), 1.0, rtol=0, atol=1e-13)
    assert w.min() >= -1e-10 and w.max() <= 1 + 1e-10
    u = np.random.default_rng(k).normal(size=mc.n_nodes)
    got = (w * u[vert]).sum(axis=1)
    ref = interpolation_matrix(mc.xy, mc.tri, mf.xy) @ u
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
    lin = 0.4 - 1.1 * mc.xy[:, 0] + 2.3 * mc.xy[:, 1]
    np.testing.assert_allclose((w * lin[vert]).sum(axis=1), 0.4 - 1.1 * mf.xy[:, 0] + 2.3 * mf.xy[:, 1],
                               rtol=0, atol=1e-13)


def test_interp_weights_refuse_outside_nodes_and_bad_ids(lib):
    mc = square_mesh(4)
    with pytest.raises(lib.LfltsError):
        lib.lflts_interp_weights(mc.xy, mc.tri, np.array([[0.5, 0.5], [1.2, 0.5]]))
    bad = mc.tri.copy()
    bad[0, 0] = mc.n_nodes
    with pytest.raises(lib.LfltsError):
        lib.lflts_interp_weights(mc.xy, bad, np.array([[0.5, 0.5]]))
