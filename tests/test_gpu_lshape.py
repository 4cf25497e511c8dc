"""Uneven batching on the graded L-shape (needs a GB300): every draw has its
own time step (Gaussian xi, no a-priori c_max), draws are bucketed by the
(fine, coarse) step counts and all buckets of two level pairs go to the GPU
in one lflts_run_pairs call (merged per mesh and step, concurrent streams);
each dQ matches the oracle run with that draw's step."""
import numpy as np
import pytest

from gpu_common import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_11117_gb300 import build, lflts
    build.build()
    return lflts


# Relative to the batch's largest |Q| (fine and coarse): FP32 1e-5 (the
# required FP32 bound of the QoI); FP64 1e-11.  On the graded L-shape the QoI (a box mean
# far from the point source) is 10 to 40 times smaller than the state's
# largest value, and two algebraically equivalent FP64 forms of Alg. 2 (the
# oracle's z-form on full values and the u-form on increments that the
# kernels use) already differ by up to 1.3e-12 of that scale when both run
# in numpy; the kernels measured up to 4.5e-12 (1e-12 on the square
# meshes, where the QoI and the state are of one size).  dQ is checked
# against the oracle's dQ at dQ's own scale (the largest |dQ| of the checked
# draws): the estimator sums dQ, and on fine pairs |dQ| is much smaller
# than |Q|.
@pytest.mark.parametrize("precision,tol", [(64, 1e-11), (32, 1e-5)])
def test_lshape_buckets_match_oracle(lf, precision, tol):
    from oracle.lts import solve_qoi
    from workload import CONFIG_LSHAPE, lshape_level, lshape_steps, xi_gaussian
    cfg = CONFIG_LSHAPE
    levs = [dict(lshape_level(cfg, l, m0=4), T=0.8) for l in range(3)]
    ctx = lf.Context(0)
    try:
        hs = [ctx.add_level(dict(lv, dt=lv["T"], n_steps=1)) for lv in levs]
        jobs, meta = [], []
        for l in (1, 2):
            xi = xi_gaussian(cfg.seed, l, 24, cfg.K, cfg.sigma)
            nf, nc = lshape_steps(levs[l], xi), lshape_steps(levs[l - 1], xi)
            for key in sorted(set(zip(nf.tolist(), nc.tolist()))):
                sel = np.nonzero((nf == key[0]) & (nc == key[1]))[0]
                x = np.ascontiguousarray(xi[sel])
                dQ, Qf, sums = np.zeros(len(sel)), np.zeros(len(sel)), np.zeros(4)
                j = lf.PairJob()
                j.fine = hs[l].desc(precision)
                j.fine.dt, j.fine.n_steps = levs[l]["T"] / key[0], key[0]
                j.coarse = hs[l - 1].desc(precision)
                j.coarse.dt, j.coarse.n_steps = levs[l - 1]["T"] / key[1], key[1]
                j.has_coarse = 1
                j.xi, j.S = x.ctypes.data, len(sel)
                j.dQ, j.Qf, j.sums = dQ.ctypes.data, Qf.ctypes.data, sums.ctypes.data
                jobs.append(j)
                meta.append((l, key, x, dQ, Qf, sums))  # the jobs point into these arrays
        assert len(jobs) > 2  # uneven: several buckets per level pair
        lf.lflts_run_pairs(ctx.h, jobs)
        eq, edq, dq_ref = [], [], []
        for l, (kf, kc), x, dQ, Qf, _ in meta:
            for i in range(min(3, x.shape[0])):
                qf = solve_qoi(dict(levs[l], dt=levs[l]["T"] / kf, n_steps=kf), x[i])
                qc = solve_qoi(dict(levs[l - 1], dt=levs[l - 1]["T"] / kc, n_steps=kc), x[i])
                # the batch's QoI scale, fine and coarse (Qc = Qf - dQ)
                scale = max(np.abs(Qf).max(), np.abs(Qf - dQ).max(), 1e-300)
                eq.append(abs(Qf[i] - qf) / scale)
                edq.append(abs(dQ[i] - (qf - qc)))
                dq_ref.append(qf - qc)
        dq_scale = max(np.abs(dq_ref).max(), 1e-300)
        edq = np.array(edq) / dq_scale
        assert max(eq) <= tol, f"QoI errors per draw: {np.array(eq)}"
        assert edq.max() <= tol, f"dQ errors per draw (dQ scale {dq_scale:.3e}): {edq}"
    finally:
        ctx.close()
