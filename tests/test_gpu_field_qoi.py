"""L2(D)-valued QoI on the GPU (needs a GB300): lflts_run_field_pair forms,
for every draw of a level pair, dU = u_l(., T) - I u_{l-1}(., T) on the fine
mesh and the FP64 sums of the V-valued estimator (sum_s dU_s per node,
||dU_s||^2 in L2(D) per draw and summed).  Checked element by element
against the FP64 oracle (oracle/field_qoi.py: brute-force interpolation
matrix, consistent mass matrix, math.fsum), each quantity relative to its
own largest value: FP64 1e-12, FP32 1e-5."""
import math

import numpy as np
import pytest

from gpu_common import draws, oracle_run, small_level

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_11117_gb300 import build, lflts
    build.build()
    return lflts


def _levels():
    return [small_level(n=n, p=3, K=4, box=(0.375, 0.625, 0.375, 0.625), T=0.5) for n in (8, 16)]


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 1e-5)])
@pytest.mark.parametrize("level", [0, 1])
def test_field_pair_against_oracle(lf, precision, tol, level):
    from oracle.field_qoi import field_sums, interpolation_matrix, l2_norm2, mass_matrix
    levs = _levels()
    S = 6
    xi = draws(S, 4, seed=31 + level)
    ctx = lf.Context(0)
    try:
        hs = [ctx.add_level(lv) for lv in levs]
        mf, mc = levs[level]["mesh"], levs[level - 1]["mesh"] if level else None
        job = lf.PairJob()
        job.fine = hs[level].desc(precision)
        iid = -1
        if level:
            job.coarse = hs[level - 1].desc(precision)
            job.has_coarse = 1
            vert, w = lf.lflts_interp_weights(mc.xy, mc.tri, mf.xy)
            iid = lf.lflts_field_interp_add(ctx.h, hs[level].mesh_id, hs[level - 1].mesh_id, vert, w)
        x = np.ascontiguousarray(xi)
        dQ, Qf, sums = np.zeros(S), np.zeros(S), np.zeros(4)
        job.xi, job.S = x.ctypes.data, S
        job.dQ, job.Qf, job.sums = dQ.ctypes.data, Qf.ctypes.data, sums.ctypes.data
        s1 = np.zeros(mf.n_nodes)
        n2 = np.zeros(S)
        sn = np.zeros(1)
        for _ in range(2):   # repeated calls reuse the buffers (and graphs)
            lf.lflts_run_field_pair(ctx.h, job, iid, s1, n2, sn)
    finally:
        ctx.close()
    # oracle: states of both levels, brute-force interpolation, consistent mass
    Qo, Uf = oracle_run(levs[level], xi)
    dU = Uf.T.copy()
    if level:
        Qc, Uc = oracle_run(levs[level - 1], xi)
        I = interpolation_matrix(mc.xy, mc.tri, mf.xy)
        dU -= (I @ Uc).T
        Qo = Qo - Qc
    M = mass_matrix(mf.xy, mf.tri)
    s1_ref, s2_ref = field_sums(dU, M)
    n2_ref = np.array([l2_norm2(M, u) for u in dU])
    assert _rel(s1, s1_ref) <= tol, _rel(s1, s1_ref)
    assert _rel(n2, n2_ref) <= tol, _rel(n2, n2_ref)
    assert abs(sn[0] - s2_ref) <= tol * abs(s2_ref)
    assert sn[0] == pytest.approx(math.fsum(n2), rel=1e-15)
    # the scalar QoI of the same solves
    assert _rel(dQ, Qo) <= 2 * tol
    assert sums[0] == pytest.approx(math.fsum(dQ), rel=1e-14, abs=1e-300)


def test_field_pair_needs_a_matching_interpolation(lf):
    levs = _levels()
    ctx = lf.Context(0)
    try:
        hs = [ctx.add_level(lv) for lv in levs]
        job = lf.PairJob()
        job.fine = hs[1].desc(64)
        job.coarse = hs[0].desc(64)
        job.has_coarse = 1
        x = np.ascontiguousarray(draws(2, 4))
        job.xi, job.S = x.ctypes.data, 2
        s1, sn = np.zeros(levs[1]["mesh"].n_nodes), np.zeros(1)
        with pytest.raises(lf.LfltsError) as e:
            lf.lflts_run_field_pair(ctx.h, job, -1, s1, None, sn)
        assert e.value.code == lf.LFLTS_ERR_ARG
        mf, mc = levs[1]["mesh"], levs[0]["mesh"]
        vert, w = lf.lflts_interp_weights(mc.xy, mc.tri, mf.xy)
        wrong = lf.lflts_field_interp_add(ctx.h, hs[0].mesh_id, hs[0].mesh_id,
                                          np.zeros((mc.xy.shape[0], 3), np.int32), np.zeros((mc.xy.shape[0], 3)))
        with pytest.raises(lf.LfltsError):
            lf.lflts_run_field_pair(ctx.h, job, wrong, s1, None, sn)
        with pytest.raises(lf.LfltsError):   # a vertex outside the coarse mesh
            lf.lflts_field_interp_add(ctx.h, hs[1].mesh_id, hs[0].mesh_id, vert + mc.xy.shape[0], w)
    finally:
        ctx.close()
