"""Adaptive MLMC driver (Alg. 1) on top of the CUDA level-pair solver.

Sec. 2.2 of the paper:
  * estimator  Q^ML = sum_l N_l^{-1} sum_i dQ_l(w^{(i,l)})          (Eq. MLMCestimator)
  * variance   V_l ~ (sum dQ_l^2 - (sum dQ_l)^2 / N_l) / (N_l - 1)  (Eq. Vell_est)
  * samples    N_l = ceil(2/eps^2 sqrt(V_l/C_l) sum_l' sqrt(V_l' C_l'))  (Eq. optimal_Nl)
  * bias       |E[Q - Q_L]| ~ |E dQ_L| / (2^alpha - 1), test < eps^2/2   (Eq. bias_est)
  * Alg. 1     L = 2 and initial N_l; repeat: compute the missing samples of
               every level, update V_l and N_l, add a level when the bias
               test fails; stop when no N_l grew.

Each Alg. 1 iteration evaluates all levels' missing draws in one
``lflts_run_pairs`` call (all levels' batches scheduled together; the
solves that share a mesh are merged by the library).  The per-level sums
come back from the GPU in FP64 (compensated within a call) and are
accumulated across iterations with compensated summation on the host.

``plain=True`` evaluates one draw per call with the FP64 path, the per-sample
baseline the batched path is compared with (time to reach RMSE eps).

The level evaluator is pluggable (``LevelPairs`` protocol: ``run(requests)``
-> per-level (dQ, sums)), so the driver logic runs on the CPU in tests with a
synthetic evaluator.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np


# ------------------------------------------------------------ formulas
def _csum(xs):
    """Compensated sum of a sequence of floats."""
    return math.fsum(xs)


def estimator(sum_dQ, N):
    return _csum(s / n for s, n in zip(sum_dQ, N))


def level_variance(s1, s2, N):
    if N < 2:
        return float("nan")
    return (s2 - s1 * s1 / N) / (N - 1)


def optimal_samples(V, C, eps):
    tot = _csum(math.sqrt(max(v, 0.0) * c) for v, c in zip(V, C))
    return [int(math.ceil(2.0 / (eps * eps) * math.sqrt(max(v, 0.0) / c) * tot)) for v, c in zip(V, C)]


def bias(mean_dQ_L, alpha):
    return abs(mean_dQ_L) / (2.0 ** alpha - 1.0)


# ------------------------------------------------------------ evaluators
class GpuLevelPairs:
    """Evaluates dQ_l = Q_l - Q_{l-1} on shared draws with lflts_run_pairs.

    handles[l] is a LevelHandle of level l (same K on every level)."""

    def __init__(self, lflts, ctx, handles, precision=32, plain=False):
        self.lf = lflts
        self.ctx = ctx
        self.h = handles
        self.precision = 64 if plain else precision
        self.plain = plain
        self.calls = 0

    def _job(self, l, xi, dQ, Qf, sums):
        j = self.lf.PairJob()
        j.fine = self.h[l].desc(self.precision)
        if l > 0:
            j.coarse = self.h[l - 1].desc(self.precision)
            j.has_coarse = 1
        j.xi = xi.ctypes.data
        j.S = xi.shape[0]
        j.dQ, j.Qf, j.sums = dQ.ctypes.data, Qf.ctypes.data, sums.ctypes.data
        return j

    def run(self, requests):
        """requests: {l: xi [n, K]} -> {l: (dQ [n], [sum dQ, sum dQ^2, sum Qf, sum Qf^2])}"""
        out = {}
        if self.plain:
            for l, xi in requests.items():
                dqs, parts = [], []
                for i in range(xi.shape[0]):
                    x = np.ascontiguousarray(xi[i:i + 1])
                    dQ, Qf, sums = np.zeros(1), np.zeros(1), np.zeros(4)
                    self.lf.lflts_run_pairs(self.ctx.h, [self._job(l, x, dQ, Qf, sums)])
                    self.calls += 1
                    dqs.append(dQ[0])
                    parts.append(sums.copy())
                P = np.array(parts)
                out[l] = (np.array(dqs), [_csum(P[:, k]) for k in range(4)])
            return out
        jobs, bufs = [], {}
        for l, xi in requests.items():
            xi = np.ascontiguousarray(xi, dtype=np.float64)
            dQ, Qf, sums = np.zeros(xi.shape[0]), np.zeros(xi.shape[0]), np.zeros(4)
            bufs[l] = (xi, dQ, Qf, sums)
            jobs.append(self._job(l, xi, dQ, Qf, sums))
        if jobs:
            self.lf.lflts_run_pairs(self.ctx.h, jobs)
            self.calls += 1
        for l, (xi, dQ, Qf, sums) in bufs.items():
            out[l] = (dQ, list(sums))
        return out


class ShardedLevelPairs:
    """Splits every level's draws across ranks (contiguous blocks, no data
    exchange) and combines the per-level sums of all ranks.

    Draws are independent (the MLMC sample is an independent sample,
    Sec. 2.2), so rank r evaluates rows [n r / world, n (r+1) / world) of each
    request with its own evaluator.  The only exchange is the level sums, in
    one FP64 all-reduce: every rank writes its (sum, compensation) pairs of
    the 4 sums of every requested level into its own slot of a
    [world, levels, 4, 2] array that is zero elsewhere, the all-reduce adds
    the arrays (adding zeros is exact, so every rank receives every pair
    unchanged, whatever the reduction order), and each level sum is then the
    compensated sum (math.fsum) of all pairs in rank order -- the same value
    on every rank, so all ranks take identical Alg. 1 decisions.
    ``allreduce(array) -> array`` is the collective (sum; e.g. a wrapper of
    torch.distributed.all_reduce, see ``torch_allreduce``); dQ stays local."""

    def __init__(self, evaluator, rank, world, allreduce):
        self.ev = evaluator
        self.rank = rank
        self.world = world
        self.allreduce = allreduce
        self.calls = 0

    def run(self, requests):
        local = {}
        for l, xi in requests.items():
            n = xi.shape[0]
            lo, hi = n * self.rank // self.world, n * (self.rank + 1) // self.world
            local[l] = xi[lo:hi]
        nonempty = {l: x for l, x in local.items() if x.shape[0] > 0}
        res = self.ev.run(nonempty) if nonempty else {}
        self.calls += 1
        levels = sorted(requests)
        buf = np.zeros((self.world, len(levels), 4, 2))
        for k, l in enumerate(levels):
            if l in res:
                for j, v in enumerate(res[l][1]):
                    buf[self.rank, k, j] = pairs(v)
        tot = np.asarray(self.allreduce(buf), dtype=np.float64).reshape(buf.shape)
        out = {}
        for k, l in enumerate(levels):
            sums = [_csum(x for r in range(self.world) for x in tot[r, k, j]) for j in range(4)]
            out[l] = (res[l][0] if l in res else np.zeros(0), sums)
        return out


def pairs(v):
    """(sum, compensation) of a value: a float, or a pair already."""
    if isinstance(v, (tuple, list, np.ndarray)) and len(v) == 2:
        return float(v[0]), float(v[1])
    return float(v), 0.0


def torch_allreduce(group=None, device="cpu"):
    """Sum all-reduce of a numpy FP64 array over torch.distributed (gloo on
    CPU tensors, NCCL on CUDA tensors)."""
    import torch
    import torch.distributed as dist

    def red(a):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        return t.cpu().numpy()
    return red


# ------------------------------------------------------------ Alg. 1
@dataclass
class MLMCResult:
    estimate: float
    L: int
    N: list
    V: list
    mean_dQ: list
    bias: float
    mse: float
    iterations: int
    seconds: float
    cost: float
    history: list = field(default_factory=list)


def alg1(evaluator, draw, eps, cost, N_init, alpha=2.0, L_start=2, L_max=None,
         max_iterations=100) -> MLMCResult:
    """Adaptive MLMC, Alg. 1.

    evaluator.run({l: xi}) -> {l: (dQ, sums4)}; draw(l, offset, n) -> xi [n, K];
    cost(l) -> C_l (work of one dQ_l sample); N_init(l) -> initial N_l."""
    t0 = time.perf_counter()
    L = L_start
    N = [int(N_init(l)) for l in range(L + 1)]
    done = [0] * (L + 1)
    parts1 = [[] for _ in range(L + 1)]
    parts2 = [[] for _ in range(L + 1)]
    history = []
    it = 0
    increased = True
    while increased and it < max_iterations:
        it += 1
        increased = False
        req = {l: draw(l, done[l], N[l] - done[l]) for l in range(L + 1) if N[l] > done[l]}
        res = evaluator.run(req)
        for l, (_, sums) in res.items():
            parts1[l].append(sums[0])
            parts2[l].append(sums[1])
            done[l] = N[l]
        s1 = [_csum(p) for p in parts1]
        s2 = [_csum(p) for p in parts2]
        V = [level_variance(s1[l], s2[l], done[l]) for l in range(L + 1)]
        C = [cost(l) for l in range(L + 1)]
        Nopt = optimal_samples([v if math.isfinite(v) else 0.0 for v in V], C, eps)
        for l in range(L + 1):
            if Nopt[l] > N[l]:
                N[l] = Nopt[l]
                increased = True
        mean_L = s1[L] / done[L]
        history.append({"iteration": it, "L": L, "N": list(N), "V": V})
        if bias(mean_L, alpha) ** 2 >= eps * eps / 2 and (L_max is None or L < L_max):
            L += 1
            N.append(int(N_init(L)))
            done.append(0)
            parts1.append([])
            parts2.append([])
            increased = True
    s1 = [_csum(p) for p in parts1]
    s2 = [_csum(p) for p in parts2]
    V = [level_variance(s1[l], s2[l], done[l]) for l in range(L + 1)]
    b = bias(s1[L] / done[L], alpha)
    mse = _csum(v / n for v, n in zip(V, done)) + b * b
    return MLMCResult(estimate=estimator(s1, done), L=L, N=done, V=V,
                      mean_dQ=[s / n for s, n in zip(s1, done)], bias=b, mse=mse, iterations=it,
                      seconds=time.perf_counter() - t0,
                      cost=_csum(n * cost(l) for l, n in enumerate(done)), history=history)
