"""Benchmark: MLMC level-pair batch of stabilised LF-LTS solves on GB300.

Workload square128-p8-K8-L5-fp32: 5 levels, 128^2 .. 2048^2 base cells,
refined box 8x (p = 8), K = 8 log-field terms, 8192/2048/512/128/32 samples
per level as fine/coarse pairs on a shared draw; per-sample coefficients,
Alg. 2 time loop to T = 1 on every mesh, QoI, dQ and FP64 level sums.
Solves on one mesh from the two pairs that use it run as one batch, meshes
run on concurrent streams.

One bench step is one time slice of that whole batch (lflts_run_pairs_slice):
step j advances every mesh's batch through the outer steps
[floor(N k / n), floor(N (k+1) / n)), k = j mod n (n = --slices, default
20), so n consecutive steps are exactly one complete MLMC batch; slice 0
also forms the coefficients and start values, slice n-1 the QoI, dQ and
level sums.  The timed K steps hold the units of their own slices.

Metric: sample*DOF*substep/s = sum over solves of S * steps * (n_free + p*|R|)
(each free DOF updated once per coarse step plus every DOF of the inner set
R once per substep) divided by the time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --impl reference the FP64 CPU oracle runs a bounded sample of the same
workload (level-0 solves of the same draws, one per host core) per step.
Under torchrun every rank runs the full batch with its own draws (weak
scaling, no data-path collective); times are maxed over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sample·DOF·substep/s and MLMC time-to-RMSE ε: batched FP32 vs plain FP64"
UNIT = "sample·DOF·substep/s"
FALLBACK_HBM_GBS = 6800.0


# ----------------------------------------------------------------- helpers
def _cfg(name):
    from workload import CONFIG_BANDWIDTH, CONFIG_BATCHED, CONFIG_PLAIN
    return {"batched": CONFIG_BATCHED, "plain": CONFIG_PLAIN, "bandwidth": CONFIG_BANDWIDTH}[name]


def _workload_desc(cfg):
    return (f"{cfg.name}: unit square, P1 lumped, {cfg.levels} levels with "
            f"{cfg.n0}^2..{cfg.n0 * 2 ** (cfg.levels - 1)}^2 base cells, box {cfg.box} refined "
            f"p={cfg.p}, c^2=exp(sum_k xi_k sin(k pi x) sin(k pi y)/k^2) K={cfg.K} xi~U(-1,1), "
            f"u0=exp(-200|x-(0.3,0.3)|^2), T={cfg.T}, QoI=mean over {cfg.qoi_box}, nu={cfg.nu}, "
            f"samples {'/'.join(map(str, cfg.samples))} as fine/coarse pairs")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        return parse_clock_rows(lines)


def parse_clock_rows(lines):
    """Summary of nvidia-smi samples in the FIELDS order (csv, noheader,
    nounits): median SM clock, the largest max SM clock, and every throttle
    reason of the four watched ones that was active in any sample."""
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) >= 9:
            rows.append(parts)
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------- CPU oracle
_ORACLE_LEVEL = {}


def _oracle_sample(args):
    cfg_name, level, xi = args
    from oracle.lts import solve_qoi
    from workload import level_problem
    key = (cfg_name, level)
    if key not in _ORACLE_LEVEL:
        _ORACLE_LEVEL[key] = level_problem(_cfg(cfg_name), level)
    lev = _ORACLE_LEVEL[key]
    t = time.perf_counter()
    solve_qoi(lev, xi)
    return time.perf_counter() - t


def oracle_units_per_sample(cfg, level):
    """Work units of one oracle solve: N_steps * (n_free + p |R|) with R = the
    vertices of elements touching P (the same count the GPU path reports)."""
    import numpy as np
    from workload import level_problem
    lev = level_problem(cfg, level)
    m = lev["mesh"]
    free = ~m.dirichlet.astype(bool)
    P = m.P.astype(bool) & free
    R = np.zeros(m.n_nodes, bool)
    R[m.tri[P[m.tri].any(axis=1)].ravel()] = True
    R &= free
    return lev["n_steps"] * (int(free.sum()) + cfg.p * int(R.sum()))


class OraclePool:
    """Spawned worker processes (safe to start after CUDA is initialised)."""

    def __init__(self, cores):
        import multiprocessing as mp
        self.cores = cores
        self.pool = mp.get_context("spawn").Pool(cores)

    def step(self, cfg_name, level, xis):
        t = time.perf_counter()
        self.pool.map(_oracle_sample, [(cfg_name, level, x) for x in xis], chunksize=1)
        return time.perf_counter() - t

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(cfg_name, cores, n_rounds=1, pool=None):
    """Oracle throughput on the host cores: `cores` level-0 samples per round."""
    from workload import xi_uniform
    cfg = _cfg(cfg_name)
    units = oracle_units_per_sample(cfg, 0)
    own = pool is None
    pool = pool or OraclePool(cores)
    try:
        xis = xi_uniform(cfg.seed, 0, cores * n_rounds, cfg.K)
        pool.step(cfg_name, 0, xis[:1])  # worker start-up and level build, untimed
        el = pool.step(cfg_name, 0, list(xis))
    finally:
        if own:
            pool.close()
    n = cores * n_rounds
    return {"value": units * n / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} level-0 solves (128^2 base, p={cfg.p}, {units:.3e} units each) of the "
                      f"same workload, one per process, FP64 numpy/scipy, {el:.1f} s"}


# ------------------------------------------------------------------- GPU
def slice_steps(N, n_slices):
    """Outer steps of each slice of an N-step time loop: slice k runs
    [floor(N k / n), floor(N (k + 1) / n)) (the library's rule)."""
    return [N * (k + 1) // n_slices - N * k // n_slices for k in range(n_slices)]


def setup_gpu(cfg, rank, n_slices, autotune=True):
    import torch
    from paper_2106_11117_gb300 import build, lflts
    from workload import level_problem, xi_uniform
    build.build()
    ctx = lflts.Context(torch.cuda.current_device())
    if not autotune:
        # for a launch list under a profiler (whose serialisation would skew
        # the autotuner's timings): the inner kernels the autotuner picks for
        # this hierarchy on GB300, paired substeps where |R| >= 200,000
        # (levels 2-4 of square128-p8-K8-L5), default shapes otherwise
        lflts.lflts_set_option(ctx.h, lflts.LFLTS_OPT_AUTOTUNE, 0)
        lflts.lflts_set_option(ctx.h, lflts.LFLTS_OPT_PAIRED_INNER, 2)
        lflts.lflts_set_option(ctx.h, lflts.LFLTS_OPT_PAIR_MIN_R, 200000)
    hs = []
    for l in range(cfg.levels):
        lev = level_problem(cfg, l)
        hs.append(ctx.add_level(lev))
        del lev["mesh"]  # free host memory of large meshes
    prec = cfg.precision
    xis_h, xis_d, outs_d, outs_h = [], [], [], []
    for l, S in enumerate(cfg.samples):
        x = xi_uniform(cfg.seed + 1000 * rank, l, S, cfg.K)
        xh = torch.from_numpy(x).pin_memory()
        xis_h.append(xh)
        xis_d.append(xh.cuda())
        outs_d.append([torch.zeros(S, dtype=torch.float64, device="cuda") for _ in range(2)]
                      + [torch.zeros(4, dtype=torch.float64, device="cuda")])
        outs_h.append([torch.zeros(S, dtype=torch.float64).pin_memory() for _ in range(2)]
                      + [torch.zeros(4, dtype=torch.float64).pin_memory()])

    def jobs(device_mem):
        js = []
        for l, S in enumerate(cfg.samples):
            j = lflts.PairJob()
            j.fine = hs[l].desc(prec)
            if l > 0:
                j.coarse = hs[l - 1].desc(prec)
                j.has_coarse = 1
            o = outs_d[l] if device_mem else outs_h[l]
            j.xi = (xis_d[l] if device_mem else xis_h[l]).data_ptr()
            j.S = S
            j.dQ, j.Qf, j.sums = o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr()
            js.append(j)
        return (lflts.PairJob * len(js))(*js)

    # solves per mesh: the fine solve of pair l and the coarse solve of pair
    # l + 1 share mesh l and run as one batch
    solves = {}
    for l, S in enumerate(cfg.samples):
        solves[l] = solves.get(l, 0) + S
        if l > 0:
            solves[l - 1] = solves.get(l - 1, 0) + S
    units_slice = [0] * n_slices
    for l, S in solves.items():
        info = hs[l].info
        per_step = S * (info["n_free"] + cfg.p * info["n_R"])
        for k, n in enumerate(slice_steps(hs[l].n_steps, n_slices)):
            units_slice[k] += per_step * n
    h2d = sum(S * cfg.K * 8 for S in cfg.samples)             # xi, copied by slice 0
    d2h = sum(S * 8 * 2 + 32 for S in cfg.samples)            # dQ, Qf, sums, by the last slice
    return {"ctx": ctx, "hs": hs, "jobs_d": jobs(True), "jobs_h": jobs(False),
            "units_slice": units_slice, "units_run": sum(units_slice), "outs_d": outs_d,
            "outs_h": outs_h, "xis": (xis_h, xis_d), "h2d": h2d, "d2h": d2h, "solves": solves,
            "lflts": lflts}


class SliceRunner:
    """Bench steps: step j runs slice (j mod n) of the level-pair run, so n
    consecutive steps are one complete MLMC batch of the workload (the
    coefficients at slice 0, every outer step of every level once, the QoI,
    dQ and level sums at slice n - 1)."""

    def __init__(self, lf, ctx, jobs, n_slices, mem, stream, units_slice):
        self.lf, self.ctx, self.jobs, self.n, self.mem, self.st = lf, ctx, jobs, n_slices, mem, stream
        self.units_slice = units_slice
        self.phase = 0
        self.starts = self.ends = 0

    def step(self):
        k = self.phase
        self.lf.lflts_run_pairs_slice(self.ctx.h, self.jobs, k, self.n, self.mem, self.st)
        self.starts += k == 0
        self.ends += k == self.n - 1
        self.phase = (k + 1) % self.n
        return self.units_slice[k]


def run_ours(args):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    cfg = _cfg(args.config)
    pool = None  # the CPU baseline runs at N = 1 only (rank 0 of one process)
    if world == 1 and not args.no_cpu_baseline:
        pool = OraclePool(args.cpu_cores or os.cpu_count() or 1)
    n_sl = args.slices
    W = setup_gpu(cfg, rank, n_sl, autotune=not args.no_autotune)
    lf = W["lflts"]
    ctx = W["ctx"]
    st = torch.cuda.current_stream()
    dev = SliceRunner(lf, ctx, W["jobs_d"], n_sl, lf.LFLTS_MEM_DEVICE, st.cuda_stream, W["units_slice"])

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        if world > 1:
            t = torch.tensor([x], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            x = float(t.item())
        return x

    for _ in range(args.warmup):
        dev.step()
    torch.cuda.synchronize()
    barrier()
    clocks = Clocks(local)
    clocks.start()
    n0 = lf.lflts_launch_count(ctx.h)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    units = 0
    e0.record(st)
    for _ in range(args.steps):
        units += dev.step()
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1))
    launches = lf.lflts_launch_count(ctx.h) - n0
    clk = clocks.stop()
    value = units * world / (ms * 1e-3)

    # end to end through the public API with host buffers: each step is the
    # same slice call with pinned host xi and outputs (slice 0 copies xi in,
    # the last slice copies dQ, Qf and the sums out; every call synchronises)
    e2e = None
    if not args.no_e2e:
        host = SliceRunner(lf, ctx, W["jobs_h"], n_sl, lf.LFLTS_MEM_HOST, st.cuda_stream, W["units_slice"])
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        u_e2e = 0
        for _ in range(args.steps):
            u_e2e += host.step()
        torch.cuda.synchronize()
        barrier()
        el = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": u_e2e * world / el, "unit": UNIT,
               "h2d_bytes_per_step": W["h2d"] * host.starts * world / args.steps,
               "d2h_bytes_per_step": W["d2h"] * host.ends * world / args.steps,
               "seconds": el, "runs_started": host.starts, "runs_completed": host.ends}

    # one more slice (slice 0 of a fresh run) with CUDA events around every
    # launch, the batches one after another on one stream, for the kernel split
    # and the roofline
    lf.lflts_profile_reset(ctx.h)
    lf.lflts_profile_enable(ctx.h, True)
    SliceRunner(lf, ctx, W["jobs_d"], n_sl, lf.LFLTS_MEM_DEVICE, st.cuda_stream, W["units_slice"]).step()
    torch.cuda.synchronize()
    lf.lflts_profile_enable(ctx.h, False)
    prof = {k: lf.lflts_profile_read(ctx.h, k) for k in ("init", "coarse", "inner", "inner_pair", "qoi", "sums")}
    roof = _roofline(prof, ("coarse", "inner", "inner_pair"),
                     {"coarse": "k_coarse", "inner": INNER_NAME, "inner_pair": PAIR_NAME})

    tte = None
    if world == 1 and not args.no_time_to_eps:
        tte = time_to_eps(args.eps)

    cpu = None
    if pool is not None:
        cpu = cpu_baseline(args.config, pool.cores, pool=pool, n_rounds=args.cpu_rounds)
        pool.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if cfg.precision == 32 else "f64", "data": "synthetic",
                "config": {"workload": _workload_desc(cfg),
                           "step": f"one time slice of the whole level-pair batch: outer steps "
                                   f"[floor(N k/{n_sl}), floor(N (k+1)/{n_sl})) of every mesh's batch, "
                                   f"k = step mod {n_sl}; {n_sl} consecutive steps are one complete MLMC "
                                   f"batch (coefficients at k = 0, QoI, dQ and FP64 level sums at "
                                   f"k = {n_sl - 1})",
                           "slices_per_batch": n_sl,
                           "solves_per_step": {f"mesh{l}": S for l, S in sorted(W["solves"].items())},
                           "units_timed": units * world, "units_per_batch": W["units_run"] * world,
                           "l2": "inputs larger than L2 (per-mesh state >= 1 GB), no flush",
                           "parallelism": f"samples sharded, dp{world}",
                           "timing": "timed steps without per-launch events (mesh batches on concurrent "
                                     "streams); roofline and kernel_classes from one further slice with "
                                     "CUDA events around every launch, batches one after another"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, "time_to_eps": tte, "kernel_classes": _classes_json(prof)}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def time_to_eps(eps=2e-3):
    """MLMC (Alg. 1) to RMSE eps on the plain workload square32-p4-K4
    (3 levels used, a 4th available): batched FP32 path vs the per-draw FP64
    path (one draw per launch), same draws, wall time of the whole Alg. 1."""
    from paper_2106_11117_gb300 import lflts, mlmc
    from workload import CONFIG_PLAIN, level_problem, xi_uniform
    cfg = CONFIG_PLAIN
    ctx = lflts.Context(0)
    try:
        hs = [ctx.add_level(level_problem(cfg, l)) for l in range(4)]

        def w(h):
            return h.n_steps * (h.info["n_free"] + h.p * h.info["n_R"])

        def cost(l):
            return float(w(hs[l]) + (w(hs[l - 1]) if l else 0))

        def draw(l, off, n):
            return xi_uniform(cfg.seed, l, n, cfg.K, offset=off)

        def n_init(l):
            return cfg.samples[l] if l < len(cfg.samples) else 16

        out = {"eps": eps, "workload": cfg.name}
        for name, plain in (("batched_fp32", False), ("plain_fp64", True)):
            ev = mlmc.GpuLevelPairs(lflts, ctx, hs, precision=32, plain=plain)
            r = mlmc.alg1(ev, draw, eps, cost, n_init, L_max=3)
            out[name] = {"seconds": r.seconds, "estimate": r.estimate, "L": r.L, "N": r.N,
                         "rmse_estimate": math.sqrt(r.mse), "calls": ev.calls}
        out["speedup"] = out["plain_fp64"]["seconds"] / out["batched_fp32"]["seconds"]
        out["estimate_diff"] = abs(out["plain_fp64"]["estimate"] - out["batched_fp32"]["estimate"])
        return out
    finally:
        ctx.close()


# Names of the inner kernel classes in the roofline record.
INNER_NAME = "k_inner (one launch per substep) / k_inner_fused"
PAIR_NAME = "k_inner_pair (two substeps per launch)"

# DRAM traffic of one captured launch per kernel class (ncu, dram__bytes_read.sum +
# dram__bytes_write.sum, --set full, one launch of level 3 of square128-p8-K8 with
# 32 draws: profiles/k_inner_square128-L3-S32.md, profiles/k_coarse_square128-L3-S32.md,
# profiles/k_inner_pair_square128-L3-S32.md)
# with its algorithmic bytes, and the hash of the kernel sources it was taken
# with: a changed source makes the figure stale and the record's traffic null.
CAPTURED = {
    "inner": {"src": ["kernels.cuh"], "sha16": "bba516a503aa701b",
              "dram_bytes": 553.56032e6 + 90.601728e6, "alg_bytes": 16.0 * 805987 * 32},
    "coarse": {"src": ["kernels.cuh"], "sha16": "bba516a503aa701b",
               "dram_bytes": 925.441024e6 + 336.92416e6, "alg_bytes": 12.0 * 1838369 * 32},
    # the second pair launch of a step (profiles/k_inner_pair_square128-L3-S32.md);
    # its traffic also depends on the block plan (mesh_prep.cpp)
    "inner_pair": {"src": ["kernels.cuh", "inner_pair.cuh", "mesh_prep.cpp"], "sha16": "f38aa14cabab141a",
                   "dram_bytes": 635.711232e6 + 193.946368e6, "alg_bytes": 20.0 * 805987 * 32},
}


def _src_sha16(src):
    """First 16 hex digits of the SHA-256 of the named kernel sources, concatenated."""
    import hashlib
    h = hashlib.sha256()
    for name in src:
        with open(os.path.join(ROOT, "paper_2106_11117_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _timed_passes(lf, ctx, step, st, warmup, steps, profile_steps=1, local=0):
    """W warm-up steps, K timed steps (CUDA events on `st`, no per-launch
    events, so graphs run where the solves fit one), then `profile_steps`
    steps with per-launch events for the kernel-class split."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    n0 = lf.lflts_launch_count(ctx.h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = lf.lflts_launch_count(ctx.h) - n0
    clk = clocks.stop()
    if profile_steps < 1:
        return ms, launches, clk, None
    lf.lflts_profile_reset(ctx.h)
    lf.lflts_profile_enable(ctx.h, True)
    for _ in range(profile_steps):
        step()
    torch.cuda.synchronize()
    lf.lflts_profile_enable(ctx.h, False)
    prof = {k: lf.lflts_profile_read(ctx.h, k) for k in lf.KERNEL_CLASSES}
    return ms, launches, clk, prof


def _roofline(prof, classes, names):
    """Roofline record of the kernel class with the most device time:
    achieved = algorithmic bytes / time over its launches (the library books
    3 values per free node and coarse launch, 4 per node of R and inner
    substep, 5 per node of R for two substeps in one launch (7 when they end
    the step), 3 per node of R for a launch of all substeps; per-draw edge
    weights not counted), against the measured HBM copy bandwidth.  traffic:
    DRAM bytes per launch, the captured launch's DRAM/algorithmic ratio times
    this class's algorithmic bytes per launch (traffic grows with the draws
    and nodes a launch covers), null without a capture of the current kernel
    source; dram_achieved / dram_frac: that traffic over the live launch
    time, the rate of the bytes the kernel actually moves."""
    peak, peak_kind = _peaks()
    total = sum(v["ms"] for v in prof.values()) or 1.0
    dom = max(classes, key=lambda k: prof[k]["ms"])
    pd = prof[dom]
    achieved = pd["alg_bytes"] / (pd["ms"] * 1e-3) / 1e9 if pd["ms"] > 0 else 0.0
    per = pd["alg_bytes"] / max(pd["launches"], 1)
    cap = CAPTURED.get(dom)
    traffic = None
    if cap and cap["sha16"] == _src_sha16(cap["src"]):
        traffic = cap["dram_bytes"] / cap["alg_bytes"] * per
    avg_s = pd["ms"] * 1e-3 / max(pd["launches"], 1)
    dram = traffic / avg_s / 1e9 if traffic and avg_s > 0 else None
    return {"bound": "hbm", "kernel": names[dom], "achieved": round(achieved, 1), "peak": peak,
            "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
            "traffic_over_alg": traffic / per if traffic else None,
            "dram_achieved": round(dram, 1) if dram else None,
            "dram_frac": round(dram / peak, 4) if dram else None,
            "alg_bytes_per_launch": per, "launches": pd["launches"],
            "avg_launch_ms": pd["ms"] / max(pd["launches"], 1),
            "share_of_kernel_time": round(pd["ms"] / total, 4)}


def _classes_json(prof):
    return {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                "alg_GBps": round(v["alg_bytes"] / (v["ms"] * 1e-3) / 1e9, 1) if v["ms"] > 0 else None}
            for k, v in prof.items() if v["launches"]}


def _alg1_run(lflts, mlmc, ctx, hs, cfg, eps, plain, L_max, n_init, seed_off=0, draw=None):
    """Alg. 1 on the given level handles with the workload's draws (or
    draw(l, offset, n)); wall time."""
    from workload import xi_uniform

    def w(h):
        return h.n_steps * (h.info["n_free"] + h.p * h.info["n_R"])

    def cost(l):
        return float(w(hs[l]) + (w(hs[l - 1]) if l else 0))

    if draw is None:
        def draw(l, off, n):
            return xi_uniform(cfg.seed + seed_off, l, n, cfg.K, offset=off)

    ev = mlmc.GpuLevelPairs(lflts, ctx, hs, precision=32, plain=plain)
    r = mlmc.alg1(ev, draw, eps, cost, lambda l: n_init, L_max=L_max)
    return {"seconds": r.seconds, "estimate": r.estimate, "L": r.L, "N": r.N,
            "rmse_estimate": math.sqrt(r.mse), "V": r.V, "bias": r.bias, "calls": ev.calls,
            "dtype": "f64" if plain else "f32", "work_units": r.cost}


def run_tte(args):
    """MLMC (Alg. 1) to RMSE eps on the batched hierarchies (Sec. 2.2, Alg. 1,
    Eq. optimal_Nl): (1) the bandwidth hierarchy square1024-p4-K8 (128^2 ..
    1024^2 base cells, p = 4) to eps = --eps-bw with the batched FP32 path;
    (2) the first levels of square128-p8-K8 (128^2 .. 512^2 base cells, p = 8)
    to eps = --eps-cls with the batched FP32 path and with the plain per-draw
    FP64 path (one draw per call) on the same draws.  Wall time of the whole
    Alg. 1 (mesh setup excluded), estimates and their difference."""
    import torch
    from paper_2106_11117_gb300 import build, lflts, mlmc
    from workload import CONFIG_BANDWIDTH, CONFIG_BATCHED, level_problem
    build.build()
    torch.cuda.set_device(0)
    out = {"mode": "time_to_eps", "metric": "MLMC time to RMSE eps (Alg. 1)", "unit": "s",
           "higher_is_better": False, "n_gpus": 1, "data": "synthetic"}
    ctx = lflts.Context(0)
    try:
        if not args.tte_skip_bw:
            hs = [ctx.add_level(level_problem(CONFIG_BANDWIDTH, l)) for l in range(CONFIG_BANDWIDTH.levels)]
            r = _alg1_run(lflts, mlmc, ctx, hs, CONFIG_BANDWIDTH, args.eps_bw, False,
                          CONFIG_BANDWIDTH.levels - 1, args.tte_n_init)
            out["bandwidth_hierarchy"] = {"workload": CONFIG_BANDWIDTH.name + " (128^2..1024^2, p=4, K=8)",
                                          "eps": args.eps_bw, "batched_fp32": r}
        cfg = CONFIG_BATCHED
        L_max = args.tte_levels - 1
        hs = [ctx.add_level(level_problem(cfg, l)) for l in range(args.tte_levels)]
        res = {}
        for name, plain in (("batched_fp32", False), ("plain_fp64", True)):
            if plain and args.tte_skip_plain:
                continue
            res[name] = _alg1_run(lflts, mlmc, ctx, hs, cfg, args.eps_cls, plain, L_max, args.tte_n_init)
        blk = {"workload": f"{cfg.name} levels 0..{L_max} (128^2..{128 * 2 ** L_max}^2, p=8, K=8)",
               "eps": args.eps_cls, **res}
        if "plain_fp64" in res:
            blk["speedup"] = res["plain_fp64"]["seconds"] / res["batched_fp32"]["seconds"]
            blk["estimate_diff"] = abs(res["plain_fp64"]["estimate"] - res["batched_fp32"]["estimate"])
            blk["estimate_diff_over_eps"] = blk["estimate_diff"] / args.eps_cls
        out["batched_hierarchy"] = blk
    finally:
        ctx.close()
    print(json.dumps(out), flush=True)


def run_lshape(args):
    """Uneven batching on the graded L-shape (lshape-graded-s2-K16-ricker):
    4 levels (m = 58..464 layers, p = 3, 5, 9, 17), Gaussian draws with their
    own time steps bucketed by (fine, coarse) step counts, Ricker source; all
    buckets of all level pairs in one lflts_run_pairs call (merged per mesh
    and step count, concurrent streams, autotuned shapes incl. the fused
    inner kernel).  FP32 state, FP64 QoI and sums."""
    import numpy as np
    import torch
    from paper_2106_11117_gb300 import build, lflts
    from workload import CONFIG_LSHAPE as cfg, lshape_level, lshape_steps, xi_gaussian
    build.build()
    torch.cuda.set_device(0)
    ctx = lflts.Context(0)
    levs = [lshape_level(cfg, l) for l in range(cfg.levels)]
    hs = [ctx.add_level(dict(lv, dt=lv["T"], n_steps=1)) for lv in levs]

    def w(h):
        return h.info["n_free"] + h.p * h.info["n_R"]

    jobs, keep, units, buckets, h2d = [], [], 0, 0, 0
    for l in range(cfg.levels):
        xi = xi_gaussian(cfg.seed, l, cfg.samples[l], cfg.K, cfg.sigma)
        nf = lshape_steps(levs[l], xi)
        nc = lshape_steps(levs[l - 1], xi) if l else np.zeros_like(nf)
        for kf, kc in sorted(set(zip(nf.tolist(), nc.tolist()))):
            sel = np.nonzero((nf == kf) & (nc == kc))[0]
            x = torch.from_numpy(np.ascontiguousarray(xi[sel])).cuda()
            o = [torch.zeros(len(sel), dtype=torch.float64, device="cuda") for _ in range(2)]
            o.append(torch.zeros(4, dtype=torch.float64, device="cuda"))
            j = lflts.PairJob()
            j.fine = hs[l].desc(cfg.precision)
            j.fine.dt, j.fine.n_steps = cfg.T / kf, kf
            if l:
                j.coarse = hs[l - 1].desc(cfg.precision)
                j.coarse.dt, j.coarse.n_steps = cfg.T / kc, kc
                j.has_coarse = 1
            j.xi, j.S = x.data_ptr(), len(sel)
            j.dQ, j.Qf, j.sums = o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr()
            jobs.append(j)
            keep.append((x, o))
            units += len(sel) * (kf * w(hs[l]) + (kc * w(hs[l - 1]) if l else 0))
            buckets += 1
            h2d += x.numel() * 8
    st = torch.cuda.current_stream()

    def step():
        lflts.lflts_run_pairs(ctx.h, jobs, lflts.LFLTS_MEM_DEVICE, st.cuda_stream)

    ms, launches, clk, prof = _timed_passes(lflts, ctx, step, st, args.warmup, args.steps)
    value = units * args.steps / (ms * 1e-3)
    names = {"coarse": "k_coarse", "inner": "k_inner / k_inner_fused"}
    line = {"mode": "lshape", "metric": UNIT + " (uneven batching, graded L-shape)", "value": value,
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{cfg.name}: L-shape [-1,1]^2 minus [0,1]x[-1,0], graded s={cfg.s}, "
                                   f"m={cfg.m0}*2^l layers, p=2q+1 with q={cfg.q_levels}, K={cfg.K}, "
                                   f"xi~N(0,{cfg.sigma}^2), Ricker f0={cfg.f0} at {cfg.source_xy}, "
                                   f"samples {'/'.join(map(str, cfg.samples))}, per-draw steps bucketed",
                       "buckets": buckets, "units_per_step": units,
                       "mesh_nodes": [h.info["n_nodes"] for h in hs], "n_R": [h.info["n_R"] for h in hs],
                       "l2": "largest meshes' state above L2, no flush"},
            "roofline": _roofline(prof, ("coarse", "inner"), names), "gpu_launches": launches,
            "clocks": clk, "stats": lflts.lflts_get_stats(ctx.h), "kernel_classes": _classes_json(prof),
            "h2d_bytes_per_step": h2d}
    ctx.close()
    print(json.dumps(line), flush=True)


def run_channel(args):
    """The narrow channel of random width (channel60-p25-b-uniform, Sec. 4.3):
    3 levels of the reference mesh (H = 1/60, 1/120, 1/240; channel box
    refined 25x; p = 100 substeps because the narrowest channel squeezes its
    cells 4x), 256/64/16 level pairs, every draw's vertices moved by
    Eq. MeshTransform and its stiffness and lumped mass formed on the GPU,
    c = 1, Neumann boundary, QoI the mean of u(., 1) along x = -0.4.  One step
    is the whole level-pair batch in one lflts_run_pairs call.  FP32 state,
    FP64 QoI and sums."""
    import numpy as np
    import torch
    from paper_2106_11117_gb300 import build, lflts
    from workload.channel import CONFIG_CHANNEL as cfg, channel_level, xi_width
    build.build()
    torch.cuda.set_device(0)
    ctx = lflts.Context(0)
    hs = [ctx.add_level(channel_level(cfg, l)) for l in range(cfg.levels)]

    def w(h):
        return h.info["n_free"] + h.p * h.info["n_R"]

    jobs, keep, units, h2d = [], [], 0, 0
    for l in range(cfg.levels):
        S = cfg.samples[l]
        x = torch.from_numpy(xi_width(cfg.seed, l, S)).cuda()
        o = [torch.zeros(S, dtype=torch.float64, device="cuda") for _ in range(2)]
        o.append(torch.zeros(4, dtype=torch.float64, device="cuda"))
        j = lflts.PairJob()
        j.fine = hs[l].desc(cfg.precision)
        if l:
            j.coarse = hs[l - 1].desc(cfg.precision)
            j.has_coarse = 1
        j.xi, j.S = x.data_ptr(), S
        j.dQ, j.Qf, j.sums = o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr()
        jobs.append(j)
        keep.append((x, o))
        units += S * (hs[l].n_steps * w(hs[l]) + (hs[l - 1].n_steps * w(hs[l - 1]) if l else 0))
        h2d += x.numel() * 8
    jobs = (lflts.PairJob * len(jobs))(*jobs)
    st = torch.cuda.current_stream()

    def step():
        lflts.lflts_run_pairs(ctx.h, jobs, lflts.LFLTS_MEM_DEVICE, st.cuda_stream)

    ms, launches, clk, prof = _timed_passes(lflts, ctx, step, st, args.warmup, args.steps)
    value = units * args.steps / (ms * 1e-3)
    names = {"coarse": "k_coarse", "inner": INNER_NAME, "inner_pair": PAIR_NAME}
    tte = None
    if not args.no_time_to_eps:  # Alg. 1 on the three levels, draws of their own
        from paper_2106_11117_gb300 import mlmc
        torch.cuda.synchronize()
        tte = _alg1_run(lflts, mlmc, ctx, hs, cfg, args.eps_channel, False, cfg.levels - 1, 64,
                        draw=lambda l, off, n: xi_width(cfg.seed + 77, l, n, offset=off))
        tte["eps"] = args.eps_channel
    line = {"mode": "channel", "metric": UNIT + " (random-geometry channel)", "value": value,
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{cfg.name}: two 0.95 x 1 rectangles joined by a 0.1 x b(w) channel, "
                                   f"b ~ U(0.001, 0.007) mapped from the reference width 0.004 by moving "
                                   f"the vertices, H = 1/{cfg.n0}..1/{cfg.n0 * 2 ** (cfg.levels - 1)}, "
                                   f"channel box refined {cfg.p_mesh}x, p = {cfg.p_lts}, c = 1, Neumann, "
                                   f"T = {cfg.T}, QoI mean of u along x = -0.4, samples "
                                   f"{'/'.join(map(str, cfg.samples))} as fine/coarse pairs",
                       "units_per_step": units, "mesh_nodes": [h.info["n_nodes"] for h in hs],
                       "n_R": [h.info["n_R"] for h in hs], "n_steps": [h.n_steps for h in hs],
                       "l2": "largest state below L2 (a few MB per array), no flush"},
            "roofline": _roofline(prof, ("coarse", "inner", "inner_pair"), names), "gpu_launches": launches,
            "clocks": clk, "kernel_classes": _classes_json(prof), "h2d_bytes_per_step": h2d,
            "sums": [keep[l][1][2].cpu().tolist() for l in range(cfg.levels)], "time_to_eps": tte}
    ctx.close()
    print(json.dumps(line), flush=True)


def run_adjoint(args):
    """dQ/dxi of every draw on square256-p8-K16 (256^2 base cells, box refined
    8x, 16 field terms, 1024 draws, 2000 outer steps of the CFL step, so
    T = 2000 dt): forward with checkpoints every 64 steps, segment
    recomputation, the adjoint recursion and the contraction with dK/dxi;
    FP32 and FP64.  Throughput counts the forward work units of the solve
    (S N (n_free + p |R|)) per gradient evaluation."""
    import torch
    from paper_2106_11117_gb300 import build, lflts
    from workload import CONFIG_ADJOINT as cfg, level_problem, xi_uniform
    build.build()
    torch.cuda.set_device(0)
    N, ckpt = 2000, 64
    lev = level_problem(cfg, 0)
    lev = dict(lev, n_steps=N, T=N * lev["dt"])
    ctx = lflts.Context(0)
    h = ctx.add_level(lev)
    S = cfg.samples[0]
    xi = torch.from_numpy(xi_uniform(cfg.seed, 0, S, cfg.K)).cuda()
    units = S * N * (h.info["n_free"] + cfg.p * h.info["n_R"])
    st = torch.cuda.current_stream()
    out = {"mode": "adjoint", "metric": UNIT + " of dQ/dxi (forward + adjoint)", "unit": UNIT,
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
           "data": "synthetic",
           "config": {"workload": f"{cfg.name}: unit square, {cfg.n0}^2 base cells, box {cfg.box} refined "
                                  f"p={cfg.p}, K={cfg.K}, xi~U(-1,1), S={S}, N={N} outer steps "
                                  f"(dt={lev['dt']:.4e}, T={lev['T']:.4f}), checkpoints every {ckpt}",
                      "n_free": h.info["n_free"], "n_R": h.info["n_R"], "n_edges": h.info["n_edges"],
                      "units_per_gradient": units}}
    names = {"coarse": "k_coarse", "inner": "k_inner", "adj_inner": "k_adj_inner (+ recomputed r)",
             "adj_edges": "k_adj_edges", "grad": "k_grad_contract"}
    for prec in (32, 64):
        Q = torch.zeros(S, dtype=torch.float64, device="cuda")
        G = torch.zeros(S, cfg.K, dtype=torch.float64, device="cuda")
        d = h.desc(prec)

        def step():
            lflts.lflts_grad_xi(ctx.h, d, xi, S, ckpt, Q, G, lflts.LFLTS_MEM_DEVICE, st.cuda_stream)

        # the FP64 gradient takes minutes: timed only, no extra profiled pass
        ms, launches, clk, prof = _timed_passes(lflts, ctx, step, st, args.warmup, args.steps,
                                                profile_steps=1 if prec == 32 else 0)
        out[f"fp{prec}"] = {"value": units * args.steps / (ms * 1e-3), "ms_per_gradient": ms / args.steps,
                            "gpu_launches": launches, "clocks": clk,
                            "roofline": _roofline(prof, tuple(names), names) if prof else None,
                            "kernel_classes": _classes_json(prof) if prof else None,
                            "grad_finite": bool(torch.isfinite(G).all().item()),
                            "grad_abs_max": float(G.abs().max().item())}
    out["value"] = out["fp32"]["value"]
    out["dtype"] = "f32"
    ctx.close()
    print(json.dumps(out), flush=True)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from workload import xi_uniform
    cfg = _cfg(args.config)
    cores = args.cpu_cores or os.cpu_count() or 1
    units = oracle_units_per_sample(cfg, 0)
    pool = OraclePool(cores)
    try:
        xis = xi_uniform(cfg.seed, 0, cores * (args.warmup + args.steps + 1), cfg.K)
        pool.step(args.config, 0, xis[:1])
        k = 0
        for _ in range(args.warmup):
            pool.step(args.config, 0, list(xis[k:k + cores]))
            k += cores
        el = 0.0
        for _ in range(args.steps):
            el += pool.step(args.config, 0, list(xis[k:k + cores]))
            k += cores
    finally:
        pool.close()
    value = units * cores * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": _workload_desc(cfg),
                       "sample": f"each step: {cores} level-0 solves (one per host core)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{cores} level-0 solves per step, {args.steps} timed steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_lts_vs_lf(args):
    """LF-LTS vs standard leapfrog (global step dt/p, the same mesh without P)
    on the first levels of the batched workload: measured solve times against
    the cost model (Eqs. cost_waveeq_LF / cost_waveeq_LTS) and the MLMC
    speed-up S of Prop. 3.2 with the variances of the batch."""
    import numpy as np
    import torch
    from paper_2106_11117_gb300 import build, costmodel, lflts
    from workload import level_problem, xi_uniform
    build.build()
    cfg = _cfg(args.config)
    levels = list(range(min(args.lts_vs_lf_levels, cfg.levels)))
    ctx = lflts.Context(0)
    st = torch.cuda.Stream()
    out = {"mode": "lts_vs_lf", "workload": cfg.name, "levels": []}
    Q = {}
    for l in levels:
        lev = level_problem(cfg, l)
        h_lts = ctx.add_level(lev)
        lev_lf = dict(lev, dt=lev["dt"] / cfg.p, n_steps=lev["n_steps"] * cfg.p)
        h_lf = ctx.add_level(lev_lf, P=False)
        # the batch of mesh l: fine draws of pair l, then the coarse draws of pair l+1
        parts = [xi_uniform(cfg.seed, l, cfg.samples[l], cfg.K)]
        if l + 1 < cfg.levels:
            parts.append(xi_uniform(cfg.seed, l + 1, cfg.samples[l + 1], cfg.K))
        xi_np = np.concatenate(parts)
        S = xi_np.shape[0]
        xi = torch.from_numpy(xi_np).cuda()
        row = {"level": l, "S": S, "n_free": h_lts.info["n_free"], "n_R": h_lts.info["n_R"], "p": cfg.p}
        for name, h in (("lts", h_lts), ("lf", h_lf)):
            q = torch.zeros(S, dtype=torch.float64, device="cuda")
            d = h.desc(cfg.precision)
            with torch.cuda.stream(st):
                lflts.lflts_solve(ctx.h, d, xi, S, q, None, lflts.LFLTS_MEM_DEVICE, st.cuda_stream)  # tune, capture
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                lflts.lflts_solve(ctx.h, d, xi, S, q, None, lflts.LFLTS_MEM_DEVICE, st.cuda_stream)
                e1.record(st)
            torch.cuda.synchronize()
            row["t_" + name] = e0.elapsed_time(e1) * 1e-3
            row["units_" + name] = S * costmodel.solve_work(h.n_steps if name == "lts" else h_lts.n_steps,
                                                             h.info["n_free"], h_lts.info["n_R"], cfg.p, name)
            Q[(l, name)] = q.cpu().numpy()
        row["work_ratio_lf_over_lts"] = row["units_lf"] / row["units_lts"]
        row["time_ratio_lf_over_lts"] = row["t_lf"] / row["t_lts"]
        row["mean_abs_dQ_lf_vs_lts"] = float(np.abs(Q[(l, "lf")] - Q[(l, "lts")]).mean())
        out["levels"].append(row)
    # MLMC speed-up (Prop. 3.2) with V_l from the batch and per-sample pair costs
    V, Ct, Cu = {"lf": [], "lts": []}, {"lf": [], "lts": []}, {"lf": [], "lts": []}
    for name in ("lf", "lts"):
        for i, row in enumerate(out["levels"]):
            l = row["level"]
            n = cfg.samples[l]
            qf = Q[(l, name)][:n]
            dq = qf - Q[(l - 1, name)][cfg.samples[l - 1]:cfg.samples[l - 1] + n] if l > 0 else qf
            V[name].append(float(np.var(dq, ddof=1)))
            ct = row["t_" + name] / row["S"] + (out["levels"][i - 1]["t_" + name] / out["levels"][i - 1]["S"] if l else 0)
            cu = row["units_" + name] / row["S"] + (out["levels"][i - 1]["units_" + name] / out["levels"][i - 1]["S"] if l else 0)
            Ct[name].append(ct)
            Cu[name].append(cu)
    out["V_lts"], out["V_lf"] = V["lts"], V["lf"]
    out["S_prop32_measured_time"] = costmodel.speedup_S(V["lts"], Ct["lf"], Ct["lts"])
    out["S_prop32_work_units"] = costmodel.speedup_S(V["lts"], Cu["lf"], Cu["lts"])
    ctx.close()
    print(json.dumps(out), flush=True)


def run_profile_case(args):
    """Small case for ncu captures: a few steps of one batched FP32 mesh solve
    with the benchmark's launch configuration (level args.profile_case); with
    --config lshape a few steps of one graded L-shape level with the fused
    inner kernel; with --config adjoint one gradient of a few steps."""
    import torch
    from paper_2106_11117_gb300 import build, lflts
    from workload import level_problem, xi_uniform
    build.build()
    if args.config == "lshape":
        from workload import CONFIG_LSHAPE as lc, lshape_level, xi_gaussian
        l = args.profile_case
        lev = lshape_level(lc, l)
        S = args.profile_samples or lc.samples[l]
        ctx = lflts.Context(0)
        lflts.lflts_set_option(ctx.h, lflts.LFLTS_OPT_AUTOTUNE, 0)
        lflts.lflts_set_option(ctx.h, lflts.LFLTS_OPT_FUSED_INNER, 2)
        h = ctx.add_level(dict(lev, dt=lev["T"] / 200000, n_steps=args.profile_steps))
        xi = torch.from_numpy(xi_gaussian(lc.seed, l, S, lc.K, lc.sigma)).cuda()
        Q = torch.zeros(S, dtype=torch.float64, device="cuda")
        lflts.lflts_solve(ctx.h, h.desc(lc.precision), xi, S, Q, None, lflts.LFLTS_MEM_DEVICE,
                          torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": f"{lc.name} level {l}", "S": S, "n_steps": args.profile_steps, **h.info}))
        ctx.close()
        return
    if args.config == "adjoint":
        from workload import CONFIG_ADJOINT as ac
        S = args.profile_samples or ac.samples[0]
        ctx = lflts.Context(0)
        h = ctx.add_level(dict(level_problem(ac, 0), n_steps=args.profile_steps))
        xi = torch.from_numpy(xi_uniform(ac.seed, 0, S, ac.K)).cuda()
        Q = torch.zeros(S, dtype=torch.float64, device="cuda")
        G = torch.zeros(S, ac.K, dtype=torch.float64, device="cuda")
        lflts.lflts_grad_xi(ctx.h, h.desc(32), xi, S, 64, Q, G, lflts.LFLTS_MEM_DEVICE,
                            torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": f"{ac.name} gradient", "S": S, "n_steps": args.profile_steps, **h.info}))
        ctx.close()
        return
    cfg = _cfg(args.config)
    l = args.profile_case
    S = cfg.samples[l] + (cfg.samples[l + 1] if l + 1 < cfg.levels else 0)
    if args.profile_samples:
        S = args.profile_samples
    ctx = lflts.Context(0)
    if args.no_autotune:
        lflts.lflts_set_option(ctx.h, lflts.LFLTS_OPT_AUTOTUNE, 0)
    if args.inner != "auto":  # one launch per substep, the tiled kernel or paired substeps, forced
        lflts.lflts_set_option(ctx.h, lflts.LFLTS_OPT_FUSED_INNER, 0)
        lflts.lflts_set_option(ctx.h, lflts.LFLTS_OPT_TILED_INNER, 2 if args.inner == "tiled" else 0)
        lflts.lflts_set_option(ctx.h, lflts.LFLTS_OPT_PAIRED_INNER, 2 if args.inner == "paired" else 0)
    if args.pair_block:
        lflts.lflts_set_option(ctx.h, lflts.LFLTS_OPT_PAIR_BLOCK, args.pair_block)
    h = ctx.add_level(level_problem(cfg, l))
    xi = torch.from_numpy(xi_uniform(cfg.seed, l, S, cfg.K)).cuda()
    Q = torch.zeros(S, dtype=torch.float64, device="cuda")
    d = h.desc(cfg.precision)
    d.n_steps = args.profile_steps
    lflts.lflts_solve(ctx.h, d, xi, S, Q, None, lflts.LFLTS_MEM_DEVICE, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    info = h.info
    print(json.dumps({"profile_case": f"{cfg.name} level {l}", "S": S, "n_steps": d.n_steps, **info}))
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--slices", type=int, default=20,
                    help="time slices per level-pair batch (one bench step = one slice)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=["batched", "plain", "bandwidth", "lshape", "adjoint", "tte", "channel"],
                    default="batched")
    ap.add_argument("--eps-bw", type=float, default=1e-3, help="RMSE target on the bandwidth hierarchy")
    ap.add_argument("--eps-cls", type=float, default=2e-3, help="RMSE target, batched vs plain comparison")
    ap.add_argument("--eps-channel", type=float, default=2e-5, help="RMSE target on the channel hierarchy")
    ap.add_argument("--tte-levels", type=int, default=3, help="levels of square128-p8-K8 in the comparison")
    ap.add_argument("--tte-n-init", type=int, default=64, help="initial samples per level of Alg. 1")
    ap.add_argument("--tte-skip-plain", action="store_true")
    ap.add_argument("--tte-skip-bw", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="fixed launch shapes (the autotuner's timings are not valid under a profiler): "
                         "the inner kernels the autotuner picks on GB300, default shapes otherwise")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-cores", type=int, default=0)
    ap.add_argument("--cpu-rounds", type=int, default=8,
                    help="level-0 oracle solves per host core in the CPU baseline")
    ap.add_argument("--no-time-to-eps", action="store_true")
    ap.add_argument("--eps", type=float, default=2e-3)
    ap.add_argument("--profile-case", type=int, default=-1,
                    help="run only a few steps of one mesh solve (for ncu captures)")
    ap.add_argument("--profile-steps", type=int, default=4)
    ap.add_argument("--profile-samples", type=int, default=0)
    ap.add_argument("--inner", choices=["auto", "substep", "tiled", "paired"], default="auto",
                    help="inner-substep kernel of a --profile-case run")
    ap.add_argument("--pair-block", type=int, default=0,
                    help="nodes of R per block of the paired substeps (--profile-case)")
    ap.add_argument("--lts-vs-lf", action="store_true", help="compare LF-LTS with standard leapfrog")
    ap.add_argument("--lts-vs-lf-levels", type=int, default=2)
    args = ap.parse_args()
    if args.lts_vs_lf:
        run_lts_vs_lf(args)
    elif args.profile_case >= 0:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.config == "channel":
        run_channel(args)
    elif args.config == "lshape":
        run_lshape(args)
    elif args.config == "adjoint":
        run_adjoint(args)
    elif args.config == "tte":
        run_tte(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
