"""Parity of the CUDA LF-LTS path with the FP64 oracle (needs a GB300).

Tolerances (relative to the batch's largest |value|):
  FP64 path: QoI <= 1e-12, state u_N <= 1e-11
  FP32 path: QoI <= 1e-5,  state u_N <= 1e-4
All calls go through the C ABI (ctypes binding)."""
import math

import numpy as np
import pytest

from gpu_common import draws, oracle_run, rel_err, small_level

pytestmark = pytest.mark.gpu

TOL_Q = {64: 1e-12, 32: 1e-5}
TOL_U = {64: 1e-11, 32: 1e-4}


@pytest.fixture(scope="module")
def lf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_11117_gb300 import build, lflts
    build.build()
    return lflts


@pytest.fixture(scope="module")
def ctx(lf):
    c = lf.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("p", [2, 3, 5])
def test_lts_state_and_qoi_match_oracle(lf, ctx, precision, p):
    lev = small_level(n=12, p=p, K=4)
    xi = draws(37, 4, seed=p)            # 37: one full and one ragged 32-sample slab
    Qo, Uo = oracle_run(lev, xi)
    h = ctx.add_level(lev)
    assert h.info["n_R"] > h.info["n_P"] > 0
    Q, U = ctx.solve(h, xi, precision=precision, state=True)
    assert rel_err(U, Uo) <= TOL_U[precision], rel_err(U, Uo)
    assert rel_err(Q, Qo) <= TOL_Q[precision], rel_err(Q, Qo)


@pytest.mark.parametrize("precision", [64, 32])
def test_plain_leapfrog_paths(lf, ctx, precision):
    """p = 1 with the mask, and P = 0 with p = 4: both are leapfrog (Sec. 3.3).
    Plain leapfrog on the locally refined mesh needs the fine step dt/p."""
    lev = small_level(n=12, p=4, K=4)
    lev = dict(lev, dt=lev["dt"] / 4, n_steps=lev["n_steps"] * 4)
    xi = draws(9, 4, seed=11)
    Qo, Uo = oracle_run(lev, xi, scheme="lf")
    h = ctx.add_level(lev)
    Q1, U1 = ctx.solve(h, xi, precision=precision, state=True, p=1)
    assert rel_err(U1, Uo) <= TOL_U[precision]
    h0 = ctx.add_level(lev, P=False)
    assert h0.info["n_P"] == 0 and h0.info["n_R"] == 0
    Q0, U0 = ctx.solve(h0, xi, precision=precision, state=True)
    assert rel_err(U0, Uo) <= TOL_U[precision]
    assert rel_err(Q0, Qo) <= TOL_Q[precision]


def test_single_sample_and_initial_velocity(lf, ctx):
    """S = 1 (one sample per launch, the plain FP64 path) and v0 != 0."""
    from workload import gaussian_bump
    lev = small_level(n=16, p=4, K=4)
    m = lev["mesh"]
    v0 = gaussian_bump(m, (0.5, 0.6), 60.0)
    xi = draws(1, 4, seed=5)
    Qo, Uo = oracle_run(lev, xi, v0=v0)
    h = ctx.add_level(lev)
    vf = lf.lflts_field_add(ctx.h, h.mesh_id, v0)
    d = h.desc(64)
    d.v0_field = vf
    Q = np.zeros(1)
    U = np.zeros((m.n_nodes, 1))
    lf.lflts_solve(ctx.h, d, xi, 1, Q, U)
    assert rel_err(U, Uo) <= TOL_U[64]
    assert rel_err(Q, Qo) <= TOL_Q[64]


@pytest.mark.parametrize("S", [1, 3, 31, 33, 130])
def test_batch_split_invariance(lf, ctx, S):
    """A sample's result does not depend on the batch it is solved in."""
    lev = small_level(n=10, p=2, K=4)
    h = ctx.add_level(lev)
    xi = draws(S, 4, seed=S)
    for prec in (32, 64):
        Qb = ctx.solve(h, xi, precision=prec)
        Qs = np.array([ctx.solve(h, xi[i:i + 1], precision=prec)[0] for i in range(0, S, max(1, S // 4))])
        np.testing.assert_array_equal(Qb[::max(1, S // 4)], Qs)


def test_device_memory_path_matches_host_path(lf, ctx):
    import torch
    lev = small_level(n=12, p=3, K=4)
    h = ctx.add_level(lev)
    xi = draws(40, 4, seed=3)
    Qh = ctx.solve(h, xi, precision=32)
    xi_d = torch.from_numpy(xi).cuda()
    Q_d = torch.zeros(40, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    lf.lflts_solve(ctx.h, h.desc(32), xi_d, 40, Q_d, None, lf.LFLTS_MEM_DEVICE, st)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Q_d.cpu().numpy(), Qh)


def test_level_sums_against_fsum(lf, ctx):
    from oracle.mlmc import level_sums
    rng = np.random.default_rng(4)
    for S in (1, 7, 256, 10001):
        Qf = rng.standard_normal(S) * 1e-3 + 0.25
        Qc = Qf + rng.standard_normal(S) * 1e-6
        out = np.zeros(4)
        lf.lflts_level_sums(ctx.h, Qf, Qc, S, out)
        ref = level_sums(Qf, Qc)
        for a, b in zip(out, ref):
            assert a == pytest.approx(b, rel=1e-15, abs=1e-300)
        lf.lflts_level_sums(ctx.h, Qf, None, S, out)
        ref = level_sums(Qf)
        assert out[0] == pytest.approx(ref[0], rel=1e-15)


def test_run_pairs_merges_and_matches_separate_solves(lf, ctx):
    """Level pairs share draws; the coarse solve of pair l and the fine solve
    of pair l-1 run on one mesh and are merged into one batch."""
    from oracle.mlmc import level_sums
    levs = [small_level(n=8 * 2**l, p=2, K=4, box=(0.375, 0.625, 0.375, 0.625)) for l in range(3)]
    hs = [ctx.add_level(l) for l in levs]
    S = [20, 9, 5]
    xis = [draws(S[l], 4, seed=40 + l) for l in range(3)]
    for prec in (64, 32):
        jobs, outs = [], []
        for l in range(3):
            dQ, Qf, sums = np.zeros(S[l]), np.zeros(S[l]), np.zeros(4)
            outs.append((dQ, Qf, sums))
            j = lf.PairJob()
            j.fine = hs[l].desc(prec)
            if l > 0:
                j.coarse = hs[l - 1].desc(prec)
                j.has_coarse = 1
            j.xi = xis[l].ctypes.data
            j.S = S[l]
            j.dQ, j.Qf, j.sums = dQ.ctypes.data, Qf.ctypes.data, sums.ctypes.data
            jobs.append(j)
        lf.lflts_run_pairs(ctx.h, jobs)
        for l in range(3):
            dQ, Qf, sums = outs[l]
            qf = ctx.solve(hs[l], xis[l], precision=prec)
            qc = ctx.solve(hs[l - 1], xis[l], precision=prec) if l > 0 else None
            np.testing.assert_array_equal(Qf, qf)
            np.testing.assert_array_equal(dQ, qf - qc if qc is not None else qf)
            ref = level_sums(qf, qc)
            np.testing.assert_allclose(sums, ref, rtol=1e-14)
        if prec == 64:
            Qo = [oracle_run(levs[l], xis[2])[0] for l in (1, 2)]
            assert rel_err(outs[2][0], Qo[1] - Qo[0]) <= 1e-10


def test_plain_config_levels_match_oracle(lf, ctx):
    """The per-sample FP64 workload (32x32 base, p = 4, K = 4), levels 0-1."""
    from workload import CONFIG_PLAIN, level_problem
    for l, S in ((0, 6), (1, 2)):
        lev = level_problem(CONFIG_PLAIN, l)
        xi = draws(S, CONFIG_PLAIN.K, seed=90 + l)
        Qo, _ = oracle_run(lev, xi)
        h = ctx.add_level(lev)
        Q64 = np.array([ctx.solve(h, xi[i:i + 1], precision=64)[0] for i in range(S)])
        assert rel_err(Q64, Qo) <= TOL_Q[64], rel_err(Q64, Qo)
        Q32 = ctx.solve(h, xi, precision=32)
        assert rel_err(Q32, Qo) <= TOL_Q[32], rel_err(Q32, Qo)


def test_unstable_step_reported(lf, ctx):
    """A time step far above the CFL limit blows up; the library reports the
    first non-finite sample instead of returning garbage."""
    lev = small_level(n=12, p=2, K=4)
    lev = dict(lev, dt=lev["dt"] * 40, n_steps=400)
    h = ctx.add_level(lev)
    with pytest.raises(lf.LfltsError) as e:
        ctx.solve(h, draws(3, 4), precision=32)
    assert e.value.code == lf.LFLTS_ERR_UNSTABLE
    assert "first sample 0" in str(e.value)


def test_bad_arguments_rejected(lf, ctx):
    lev = small_level(n=8, p=2, K=4)
    h = ctx.add_level(lev)
    bad = h.desc(32)
    bad.p = 0
    with pytest.raises(lf.LfltsError):
        lf.lflts_solve(ctx.h, bad, draws(2, 4), 2, np.zeros(2))
    bad = h.desc(16)
    with pytest.raises(lf.LfltsError):
        lf.lflts_solve(ctx.h, bad, draws(2, 4), 2, np.zeros(2))
    bad = h.desc(32)
    bad.qoi_id = 999
    with pytest.raises(lf.LfltsError):
        lf.lflts_solve(ctx.h, bad, draws(2, 4), 2, np.zeros(2))


@pytest.mark.parametrize("fused", [0, 2])
def test_profiling_counters(lf, ctx, fused):
    """Per-class launch counts: p - 1 inner launches per step, or one with the
    fused inner kernel; init 3 kernels, QoI 2."""
    lev = small_level(n=12, p=4, K=4)
    h = ctx.add_level(lev)
    lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_FUSED_INNER, fused)
    try:
        lf.lflts_profile_reset(ctx.h)
        lf.lflts_profile_enable(ctx.h, True)
        n0 = lf.lflts_launch_count(ctx.h)
        ctx.solve(h, draws(8, 4), precision=32)
        lf.lflts_profile_enable(ctx.h, False)
        co = lf.lflts_profile_read(ctx.h, "coarse")
        inn = lf.lflts_profile_read(ctx.h, "inner")
        per_step = 3 if fused == 0 else 1
        assert co["launches"] == h.n_steps
        assert inn["launches"] == h.n_steps * per_step
        assert co["ms"] > 0 and inn["alg_bytes"] > 0
        assert lf.lflts_launch_count(ctx.h) - n0 == 3 + h.n_steps * (1 + per_step) + 2
    finally:
        lf.lflts_set_option(ctx.h, lf.LFLTS_OPT_FUSED_INNER, 1)


@pytest.mark.parametrize("precision", [64, 32])
def test_ricker_point_source_matches_oracle(lf, ctx, precision):
    """Forcing f = r(t) delta(x - x_s) (Ricker wavelet), entering Alg. 2 through
    w_n and frozen over the inner substeps."""
    from workload import point_source
    lev = small_level(n=12, p=3, K=4)
    nodes, w = point_source(lev["mesh"], (0.5, 0.47))
    lev = dict(lev, source={"nodes": nodes, "weights": w, "f0": 6.0, "t0": 0.2, "amp": 2.0},
               u0=0.0 * lev["u0"])
    xi = draws(6, 4, seed=17)
    Qo, Uo = oracle_run(lev, xi, source=lev["source"])
    h = ctx.add_level(lev)
    Q, U = ctx.solve(h, xi, precision=precision, state=True)
    assert np.abs(Uo).max() > 1e-3
    assert rel_err(U, Uo) <= TOL_U[precision]
    assert rel_err(Q, Qo) <= TOL_Q[precision]
