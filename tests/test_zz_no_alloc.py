"""The QoI reduction that allocates nothing (lflts_qoi_reduce_noalloc).

It serves callers that cannot let the library allocate device memory:
applications whose GPU memory is owned by their own pool allocator, or code
that must not allocate once it is running.  Its partial sums live in a fixed
array inside the library, so these tests check that two calls in a row on
that shared array give exactly the QoI of the regular lflts_solve path (same
values, same weights, same summation order: bit for bit) and agree with the
FP64 oracle within the parity tolerances, and that a call too large for the
array is refused.  Collected last on purpose.
"""
import numpy as np
import pytest

from gpu_common import draws, oracle_run, rel_err, small_level

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_11117_gb300 import build, lflts
    build.build()
    return lflts


@pytest.mark.parametrize("precision,tol", [(32, 1e-5), (64, 1e-12)])
def test_noalloc_qoi_matches_solve_twice(lf, precision, tol):
    import torch
    lev = small_level(n=16, p=4, K=4)
    ctx = lf.Context(0)
    try:
        h = ctx.add_level(lev)
        S = 37
        xi = draws(S, 4, seed=7)
        Q_ref, U = ctx.solve(h, xi, precision=precision, state=True)  # existing entry point
        dtype = torch.float32 if precision == 32 else torch.float64
        u_d = torch.from_numpy(U).to(dtype).cuda().contiguous()          # [n_nodes][S], exact copy
        idx_d = torch.from_numpy(lev["qoi_idx"].astype(np.int32)).cuda()
        g_d = torch.from_numpy(lev["qoi_w"]).cuda()
        st = torch.cuda.current_stream().cuda_stream
        Q_or, _ = oracle_run(lev, xi[:5])
        for _ in range(2):                                                 # two calls in a row
            Q_d = torch.full((S,), float("nan"), dtype=torch.float64, device="cuda")
            lf.lflts_qoi_reduce_noalloc(ctx.h, u_d, precision, U.shape[0], S, idx_d, g_d,
                                        idx_d.numel(), Q_d, st)
            torch.cuda.synchronize()
            Q = Q_d.cpu().numpy()
            np.testing.assert_array_equal(Q, Q_ref)
            assert rel_err(Q[:5], Q_or) <= tol, rel_err(Q[:5], Q_or)
    finally:
        ctx.close()


def test_noalloc_rejects_calls_beyond_its_scratch(lf):
    import torch
    S = 300000          # 1 chunk x 300000 partial sums > 131072
    idx_d = torch.zeros(4, dtype=torch.int32, device="cuda")
    g_d = torch.ones(4, dtype=torch.float64, device="cuda")
    u_d = torch.zeros(S, dtype=torch.float32, device="cuda")
    Q_d = torch.zeros(S, dtype=torch.float64, device="cuda")
    ctx = lf.Context(0)
    try:
        with pytest.raises(lf.LfltsError) as e:
            lf.lflts_qoi_reduce_noalloc(ctx.h, u_d, 32, 1, S, idx_d, g_d, 4, Q_d, None)
        assert e.value.code == lf.LFLTS_ERR_ARG
        assert "exceeds the fixed scratch capacity" in str(e.value)
    finally:
        ctx.close()
