"""Level-pair runs in time slices (needs a GB300): lflts_run_pairs_slice cuts
the time loop of every merged batch into n parts; calls 0..n-1 must give
exactly the results of one lflts_run_pairs call (dQ, Qf and the level sums,
bit for bit), with device and with host buffers, for uniform and ragged
batches, with per-launch profiling on (every batch then runs on the caller's
stream); calls that do not continue the run in progress are refused."""
import numpy as np
import pytest

from gpu_common import draws, small_level

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_11117_gb300 import build, lflts
    build.build()
    return lflts


def _hierarchy(lf, ctx, p=3):
    """Three nested square levels (8, 16, 32 base cells), refined box, p."""
    hs = []
    for n in (8, 16, 32):
        lev = small_level(n=n, p=p, K=4, box=(0.375, 0.625, 0.375, 0.625), T=0.4)
        hs.append(ctx.add_level(lev))
    return hs


class Jobs:
    """Pair jobs of levels 0..2 (level l > 0 pairs with l - 1) with their
    buffers, kept alive with the job array."""

    def __init__(self, lf, hs, prec, sizes, device, seed=0, ragged=False):
        import torch
        self.keep, jobs = [], []
        for l, S in enumerate(sizes):
            x = draws(S, 4, seed=seed + l)
            j = lf.PairJob()
            j.fine = hs[l].desc(prec)
            if l:
                j.coarse = hs[l - 1].desc(prec)
                j.has_coarse = 1
            if ragged and l == 1:  # a second step count on the middle mesh
                j.fine.dt, j.fine.n_steps = j.fine.dt * j.fine.n_steps / (j.fine.n_steps + 3), j.fine.n_steps + 3
            if device:
                xd = torch.from_numpy(x).cuda()
                o = [torch.zeros(S, dtype=torch.float64, device="cuda") for _ in range(2)]
                o.append(torch.zeros(4, dtype=torch.float64, device="cuda"))
                j.xi = xd.data_ptr()
                j.dQ, j.Qf, j.sums = (t.data_ptr() for t in o)
                self.keep.append((xd, o))
            else:
                o = [np.zeros(S), np.zeros(S), np.zeros(4)]
                j.xi = x.ctypes.data
                j.dQ, j.Qf, j.sums = (a.ctypes.data for a in o)
                self.keep.append((x, o))
            j.S = S
            jobs.append(j)
        self.arr = (lf.PairJob * len(jobs))(*jobs)

    def results(self):
        out = []
        for _, o in self.keep:
            out.append([t.cpu().numpy().copy() if hasattr(t, "cpu") else t.copy() for t in o])
        return out


def _run(lf, ctx, jobs, n_slices, mem, profile=False):
    import torch
    st = torch.cuda.current_stream().cuda_stream
    if profile:
        lf.lflts_profile_reset(ctx.h)
        lf.lflts_profile_enable(ctx.h, True)
    try:
        if n_slices == 0:
            lf.lflts_run_pairs(ctx.h, list(jobs.arr), mem, st)
        else:
            for k in range(n_slices):
                lf.lflts_run_pairs_slice(ctx.h, jobs.arr, k, n_slices, mem, st)
        torch.cuda.synchronize()
    finally:
        if profile:
            lf.lflts_profile_enable(ctx.h, False)
    return jobs.results()


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("device", [True, False])
@pytest.mark.parametrize("ragged", [False, True])
def test_slices_equal_one_call(lf, prec, device, ragged):
    mem = lf.LFLTS_MEM_DEVICE if device else lf.LFLTS_MEM_HOST
    ctx = lf.Context(0)
    try:
        hs = _hierarchy(lf, ctx)
        sizes = (40, 12, 6)
        ref = _run(lf, ctx, Jobs(lf, hs, prec, sizes, device, ragged=ragged), 0, mem)
        for n in (1, 2, 3, 7):
            got = _run(lf, ctx, Jobs(lf, hs, prec, sizes, device, ragged=ragged), n, mem)
            for a, b in zip(got, ref):
                for x, y in zip(a, b):
                    np.testing.assert_array_equal(x, y)
        got = _run(lf, ctx, Jobs(lf, hs, prec, sizes, device, ragged=ragged), 4, mem, profile=True)
        for a, b in zip(got, ref):
            for x, y in zip(a, b):
                np.testing.assert_array_equal(x, y)
        assert np.all(np.isfinite(ref[0][0])) and np.abs(ref[0][1]).max() > 0
    finally:
        ctx.close()


def test_slices_out_of_order_are_refused(lf):
    import torch
    st = torch.cuda.current_stream().cuda_stream
    ctx = lf.Context(0)
    try:
        hs = _hierarchy(lf, ctx)
        a = Jobs(lf, hs, 32, (8, 4, 4), True)
        b = Jobs(lf, hs, 32, (8, 4, 4), True, seed=5)
        with pytest.raises(lf.LfltsError) as e:   # no run in progress
            lf.lflts_run_pairs_slice(ctx.h, a.arr, 1, 3, lf.LFLTS_MEM_DEVICE, st)
        assert e.value.code == lf.LFLTS_ERR_ARG
        lf.lflts_run_pairs_slice(ctx.h, a.arr, 0, 3, lf.LFLTS_MEM_DEVICE, st)
        for bad in ((a, 2, 3), (b, 1, 3), (a, 1, 4), (a, 3, 3), (a, -1, 3)):
            with pytest.raises(lf.LfltsError) as e:
                lf.lflts_run_pairs_slice(ctx.h, bad[0].arr, bad[1], bad[2], lf.LFLTS_MEM_DEVICE, st)
            assert e.value.code == lf.LFLTS_ERR_ARG
        # an error drops the run: continuing it is refused as well
        with pytest.raises(lf.LfltsError):
            lf.lflts_run_pairs_slice(ctx.h, a.arr, 1, 3, lf.LFLTS_MEM_DEVICE, st)
        # a new run starts at slice 0 and completes
        for k in range(3):
            lf.lflts_run_pairs_slice(ctx.h, a.arr, k, 3, lf.LFLTS_MEM_DEVICE, st)
        torch.cuda.synchronize()
        assert np.all(np.isfinite(a.results()[2][0]))
    finally:
        ctx.close()
