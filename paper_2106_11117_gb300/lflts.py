"""Thin ctypes binding of liblflts.so (include/lflts.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
Each C entry point ``lflts_X`` has a Python function of the same name taking
the same arguments, with numpy arrays for host buffers and integers (device
addresses, e.g. ``torch.Tensor.data_ptr()``) or torch CUDA tensors for device
buffers.  ``Context`` wraps them for convenience.

If the shared library is missing or cannot be loaded, importing the names
works but every call raises ``LibraryNotBuilt``: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblflts.so")

LFLTS_OK = 0
LFLTS_ERR_ARG = -1
LFLTS_ERR_OOM = -2
LFLTS_ERR_CUDA = -3
LFLTS_ERR_UNSTABLE = -4
LFLTS_ERR_TIMEOUT = -5
LFLTS_ERR_MESH = -6
LFLTS_MEM_HOST = 0
LFLTS_MEM_DEVICE = 1
KERNEL_CLASSES = {"init": 0, "coarse": 1, "inner": 2, "qoi": 3, "sums": 4,
                  "adj_inner": 5, "adj_edges": 6, "grad": 7, "inner_pair": 8}

EXPORTED = [
    "lflts_version", "lflts_create", "lflts_destroy", "lflts_last_error", "lflts_mesh_add",
    "lflts_mesh_info", "lflts_mesh_order", "lflts_lts_constants", "lflts_field_add",
    "lflts_qoi_add", "lflts_solve", "lflts_level_sums", "lflts_run_pairs",
    "lflts_profile_enable", "lflts_profile_reset", "lflts_profile_read", "lflts_launch_count",
    "lflts_qoi_reduce_noalloc", "lflts_grad_xi", "lflts_set_option", "lflts_get_stats",
    "lflts_source_add", "lflts_interp_weights", "lflts_run_pairs_slice", "lflts_field_interp_add",
    "lflts_run_field_pair", "lflts_graph_cache_size", "lflts_mesh_add_moving",
]
LFLTS_OPT_GRAPHS = 1
LFLTS_OPT_AUTOTUNE = 2
LFLTS_OPT_FUSED_INNER = 5
LFLTS_OPT_TILED_INNER = 6
LFLTS_OPT_TILE_CAP = 7
LFLTS_OPT_GRAPH_CACHE = 8
LFLTS_OPT_PAIRED_INNER = 9
LFLTS_OPT_PAIR_BLOCK = 10
LFLTS_OPT_PAIR_MIN_R = 11
LFLTS_OPT_COARSE_RC = 12


class LibraryNotBuilt(RuntimeError):
    pass


class LfltsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lflts error {code}: {msg}")
        self.code = code


class SolveDesc(C.Structure):
    _fields_ = [("mesh_id", C.c_int), ("qoi_id", C.c_int), ("u0_field", C.c_int),
                ("v0_field", C.c_int), ("precision", C.c_int), ("p", C.c_int),
                ("nu", C.c_double), ("dt", C.c_double), ("n_steps", C.c_int64),
                ("source_id", C.c_int), ("src_f0", C.c_double), ("src_t0", C.c_double),
                ("src_amp", C.c_double)]

    def __init__(self, *args, **kw):
        super().__init__(*args, **kw)
        if len(args) < 10 and "source_id" not in kw:
            self.source_id = -1


class PairJob(C.Structure):
    """lflts_pair_job: raw pointers (numpy ``ctypes.data`` or torch
    ``data_ptr()``), so every array a job points to must stay alive until
    lflts_run_pairs has returned (host buffers) or its stream has finished
    (device buffers)."""
    _fields_ = [("fine", SolveDesc), ("coarse", SolveDesc), ("has_coarse", C.c_int),
                ("xi", C.c_void_p), ("S", C.c_int64), ("dQ", C.c_void_p), ("Qf", C.c_void_p),
                ("sums", C.c_void_p)]


_lib = None


def load(path: str | None = None):
    """Load (once) and type the shared library."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise LibraryNotBuilt(f"{p} not found: run paper_2106_11117_gb300.build.build() first")
    try:
        lib = C.CDLL(p)
    except OSError as e:
        raise LibraryNotBuilt(f"cannot load {p}: {e}") from e
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
    sig = {
        "lflts_version": (i32, []),
        "lflts_create": (i32, [C.POINTER(vp), i32]),
        "lflts_destroy": (i32, [vp]),
        "lflts_last_error": (C.c_char_p, [vp]),
        "lflts_mesh_add": (i32, [vp, vp, i64, vp, i64, vp, vp, vp, i32, C.POINTER(i32)]),
        "lflts_mesh_add_moving": (i32, [vp, vp, i64, vp, i64, vp, vp, vp, i32, C.POINTER(i32)]),
        "lflts_mesh_info": (i32, [vp, i32, vp]),
        "lflts_mesh_order": (i32, [vp, i32, vp]),
        "lflts_lts_constants": (i32, [i32, C.c_double, C.c_double, vp]),
        "lflts_field_add": (i32, [vp, i32, vp, C.POINTER(i32)]),
        "lflts_qoi_add": (i32, [vp, i32, vp, vp, i64, C.POINTER(i32)]),
        "lflts_solve": (i32, [vp, C.POINTER(SolveDesc), vp, i64, vp, vp, i32, vp]),
        "lflts_level_sums": (i32, [vp, vp, vp, i64, vp, i32, vp]),
        "lflts_run_pairs": (i32, [vp, C.POINTER(PairJob), i32, i32, vp]),
        "lflts_run_pairs_slice": (i32, [vp, C.POINTER(PairJob), i32, i32, i32, i32, vp]),
        "lflts_field_interp_add": (i32, [vp, i32, i32, vp, vp, C.POINTER(i32)]),
        "lflts_run_field_pair": (i32, [vp, C.POINTER(PairJob), i32, vp, vp, vp, i32, vp]),
        "lflts_profile_enable": (i32, [vp, i32]),
        "lflts_profile_reset": (i32, [vp]),
        "lflts_profile_read": (i32, [vp, i32, C.POINTER(i64), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "lflts_launch_count": (i32, [vp, C.POINTER(i64)]),
        "lflts_graph_cache_size": (i32, [vp, C.POINTER(i64)]),
        "lflts_qoi_reduce_noalloc": (i32, [vp, vp, i32, i64, i64, vp, vp, i64, vp, vp]),
        "lflts_grad_xi": (i32, [vp, C.POINTER(SolveDesc), vp, i64, i32, vp, vp, i32, vp]),
        "lflts_set_option": (i32, [vp, i32, i64]),
        "lflts_source_add": (i32, [vp, i32, vp, vp, i64, C.POINTER(i32)]),
        "lflts_get_stats": (i32, [vp, vp]),
        "lflts_interp_weights": (i32, [vp, i64, vp, i64, vp, i64, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(x):
    """Address of a numpy array, a torch tensor, an int address or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_contiguous") and not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


def _check(ctx, rc):
    if rc != LFLTS_OK:
        msg = load().lflts_last_error(ctx).decode() if ctx else ""
        raise LfltsError(rc, msg)
    return rc


# ---------------------------------------------------------------- C names
def lflts_version():
    return load().lflts_version()


def lflts_create(device: int = 0):
    h = C.c_void_p()
    rc = load().lflts_create(C.byref(h), int(device))
    if rc != LFLTS_OK:
        raise LfltsError(rc, f"lflts_create(device={device}) failed")
    return h.value


def lflts_destroy(ctx):
    return load().lflts_destroy(ctx)


def lflts_last_error(ctx):
    return load().lflts_last_error(ctx).decode()


def lflts_mesh_add(ctx, xy, tri, dirichlet, P, psi):
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    dirichlet = np.ascontiguousarray(dirichlet, dtype=np.uint8)
    P = None if P is None else np.ascontiguousarray(P, dtype=np.uint8)
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    if psi.ndim != 2 or psi.shape[0] != tri.shape[0]:
        raise ValueError("psi must be [n_tri, K]")
    mid = C.c_int()
    _check(ctx, load().lflts_mesh_add(ctx, _ptr(xy), xy.shape[0], _ptr(tri), tri.shape[0],
                                      _ptr(dirichlet), _ptr(P), _ptr(psi), psi.shape[1], C.byref(mid)))
    return mid.value


def lflts_mesh_add_moving(ctx, xy, tri, dirichlet, P, disp):
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    dirichlet = np.ascontiguousarray(dirichlet, dtype=np.uint8)
    P = None if P is None else np.ascontiguousarray(P, dtype=np.uint8)
    disp = np.ascontiguousarray(disp, dtype=np.float64)
    if disp.ndim != 3 or disp.shape[1:] != (xy.shape[0], 2):
        raise ValueError("disp must be [K, n_nodes, 2]")
    mid = C.c_int()
    _check(ctx, load().lflts_mesh_add_moving(ctx, _ptr(xy), xy.shape[0], _ptr(tri), tri.shape[0],
                                             _ptr(dirichlet), _ptr(P), _ptr(disp), disp.shape[0],
                                             C.byref(mid)))
    return mid.value


def lflts_mesh_info(ctx, mesh_id):
    info = np.zeros(8, dtype=np.int64)
    _check(ctx, load().lflts_mesh_info(ctx, mesh_id, _ptr(info)))
    keys = ["n_nodes", "n_free", "n_R", "n_P", "n_tri", "K", "n_edges", "n_edges_P"]
    return {k: int(v) for k, v in zip(keys, info)}


def lflts_mesh_order(ctx, mesh_id):
    n = lflts_mesh_info(ctx, mesh_id)["n_nodes"]
    out = np.zeros(n, dtype=np.int32)
    _check(ctx, load().lflts_mesh_order(ctx, mesh_id, _ptr(out)))
    return out


def lflts_interp_weights(xy_c, tri_c, xy_f):
    """(vert [n_f, 3] int32, w [n_f, 3]): the coarse triangle's vertices and
    barycentric coordinates at every fine node (host only)."""
    xy_c = np.ascontiguousarray(xy_c, dtype=np.float64)
    tri_c = np.ascontiguousarray(tri_c, dtype=np.int32)
    xy_f = np.ascontiguousarray(xy_f, dtype=np.float64)
    vert = np.zeros((xy_f.shape[0], 3), dtype=np.int32)
    w = np.zeros((xy_f.shape[0], 3), dtype=np.float64)
    rc = load().lflts_interp_weights(_ptr(xy_c), xy_c.shape[0], _ptr(tri_c), tri_c.shape[0], _ptr(xy_f),
                                     xy_f.shape[0], _ptr(vert), _ptr(w))
    if rc != LFLTS_OK:
        raise LfltsError(rc, "interp_weights: " + ("a fine node lies outside the coarse mesh"
                                                   if rc == LFLTS_ERR_MESH else "bad arguments"))
    return vert, w


def lflts_lts_constants(p, nu, dt):
    out = np.zeros(4 + 2 * max(p - 1, 0), dtype=np.float64)
    rc = load().lflts_lts_constants(int(p), float(nu), float(dt), _ptr(out))
    if rc != LFLTS_OK:
        raise LfltsError(rc, "lts_constants: bad arguments")
    return {"delta": out[0], "omega": out[1], "c0": out[2], "gamma": out[3],
            "beta": {m: out[4 + 2 * (m - 1)] for m in range(1, p)},
            "c": {m: out[5 + 2 * (m - 1)] for m in range(1, p)}}


def lflts_field_add(ctx, mesh_id, values):
    v = np.ascontiguousarray(values, dtype=np.float64)
    fid = C.c_int()
    _check(ctx, load().lflts_field_add(ctx, mesh_id, _ptr(v), C.byref(fid)))
    return fid.value


def lflts_source_add(ctx, mesh_id, nodes, weights):
    nodes = np.ascontiguousarray(nodes, dtype=np.int32)
    weights = np.ascontiguousarray(weights, dtype=np.float64)
    sid = C.c_int()
    _check(ctx, load().lflts_source_add(ctx, mesh_id, _ptr(nodes), _ptr(weights), nodes.shape[0], C.byref(sid)))
    return sid.value


def lflts_qoi_add(ctx, mesh_id, idx, g):
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    g = np.ascontiguousarray(g, dtype=np.float64)
    qid = C.c_int()
    _check(ctx, load().lflts_qoi_add(ctx, mesh_id, _ptr(idx), _ptr(g), idx.shape[0], C.byref(qid)))
    return qid.value


def lflts_solve(ctx, desc: SolveDesc, xi, S, Q, uN=None, mem=LFLTS_MEM_HOST, stream=None):
    return _check(ctx, load().lflts_solve(ctx, C.byref(desc), _ptr(xi), int(S), _ptr(Q), _ptr(uN),
                                          int(mem), stream))


def lflts_grad_xi(ctx, desc: SolveDesc, xi, S, ckpt_every, Q, dQdxi, mem=LFLTS_MEM_HOST, stream=None):
    return _check(ctx, load().lflts_grad_xi(ctx, C.byref(desc), _ptr(xi), int(S), int(ckpt_every), _ptr(Q),
                                            _ptr(dQdxi), int(mem), stream))


def lflts_level_sums(ctx, Qf, Qc, S, sums, mem=LFLTS_MEM_HOST, stream=None):
    return _check(ctx, load().lflts_level_sums(ctx, _ptr(Qf), _ptr(Qc), int(S), _ptr(sums), int(mem), stream))


def lflts_run_pairs(ctx, jobs, mem=LFLTS_MEM_HOST, stream=None):
    arr = (PairJob * len(jobs))(*jobs)
    return _check(ctx, load().lflts_run_pairs(ctx, arr, len(jobs), int(mem), stream))


def lflts_run_pairs_slice(ctx, jobs, slice, n_slices, mem=LFLTS_MEM_HOST, stream=None):
    """Slice ``slice`` of ``n_slices`` of the level-pair run of ``jobs``.  The
    caller keeps one ``(PairJob * n)`` array (or list) and every buffer the jobs
    point to alive for the whole run."""
    arr = jobs if isinstance(jobs, C.Array) else (PairJob * len(jobs))(*jobs)
    return _check(ctx, load().lflts_run_pairs_slice(ctx, arr, len(arr), int(mem), int(slice), int(n_slices),
                                                    stream))


def lflts_field_interp_add(ctx, mesh_f, mesh_c, vert, w):
    vert = np.ascontiguousarray(vert, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    iid = C.c_int()
    _check(ctx, load().lflts_field_interp_add(ctx, int(mesh_f), int(mesh_c), _ptr(vert), _ptr(w), C.byref(iid)))
    return iid.value


def lflts_run_field_pair(ctx, job, interp_id, sum_dU, norm2, sum_norm2, mem=LFLTS_MEM_HOST, stream=None):
    return _check(ctx, load().lflts_run_field_pair(ctx, C.byref(job), int(interp_id), _ptr(sum_dU), _ptr(norm2),
                                                   _ptr(sum_norm2), int(mem), stream))


def lflts_profile_enable(ctx, on=True):
    return _check(ctx, load().lflts_profile_enable(ctx, int(bool(on))))


def lflts_profile_reset(ctx):
    return _check(ctx, load().lflts_profile_reset(ctx))


def lflts_profile_read(ctx, kernel_class):
    cls = KERNEL_CLASSES[kernel_class] if isinstance(kernel_class, str) else int(kernel_class)
    n, ms, b = C.c_int64(), C.c_double(), C.c_double()
    _check(ctx, load().lflts_profile_read(ctx, cls, C.byref(n), C.byref(ms), C.byref(b)))
    return {"launches": n.value, "ms": ms.value, "alg_bytes": b.value}


def lflts_set_option(ctx, option, value):
    return _check(ctx, load().lflts_set_option(ctx, int(option), int(value)))


def lflts_get_stats(ctx):
    out = np.zeros(4, dtype=np.int64)
    _check(ctx, load().lflts_get_stats(ctx, _ptr(out)))
    return {"launches": int(out[0]), "graph_launches": int(out[1]), "tune_launches": int(out[2]),
            "tuned_shapes": int(out[3])}


def lflts_graph_cache_size(ctx):
    n = C.c_int64()
    _check(ctx, load().lflts_graph_cache_size(ctx, C.byref(n)))
    return n.value


def lflts_launch_count(ctx):
    n = C.c_int64()
    _check(ctx, load().lflts_launch_count(ctx, C.byref(n)))
    return n.value


def lflts_qoi_reduce_noalloc(ctx, u, precision, n_rows, S, idx, g, nnz, Q, stream=None):
    """QoI reduction without allocation; all arrays are device buffers."""
    return _check(ctx, load().lflts_qoi_reduce_noalloc(ctx, _ptr(u), int(precision), int(n_rows), int(S),
                                                       _ptr(idx), _ptr(g), int(nnz), _ptr(Q), stream))


# ------------------------------------------------------------ convenience
@dataclass
class LevelHandle:
    mesh_id: int
    qoi_id: int
    u0_field: int
    dt: float
    n_steps: int
    p: int
    nu: float
    info: dict
    source: tuple = (-1, 0.0, 0.0, 0.0)  # (source_id, f0, t0, amplitude)

    def desc(self, precision: int, p: int | None = None) -> SolveDesc:
        return SolveDesc(self.mesh_id, self.qoi_id, self.u0_field, -1, int(precision),
                         int(self.p if p is None else p), float(self.nu), float(self.dt),
                         int(self.n_steps), *self.source)


class Context:
    """Owns one lflts context (one device)."""

    def __init__(self, device: int = 0):
        self.h = lflts_create(device)
        self.device = device

    def close(self):
        if self.h:
            lflts_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_level(self, level: dict, P=True) -> LevelHandle:
        """Register a level built by the workload generators (mesh, psi, u0, QoI)."""
        m = level["mesh"]
        if level.get("modes") is not None:  # vertices moved per draw by xi . modes
            mid = lflts_mesh_add_moving(self.h, m.xy, m.tri, m.dirichlet, m.P if P else None, level["modes"])
        else:
            mid = lflts_mesh_add(self.h, m.xy, m.tri, m.dirichlet, m.P if P else None, level["psi"])
        qid = lflts_qoi_add(self.h, mid, level["qoi_idx"], level["qoi_w"])
        fid = lflts_field_add(self.h, mid, level["u0"])
        src = (-1, 0.0, 0.0, 0.0)
        if level.get("source") is not None:
            s_ = level["source"]
            sid = lflts_source_add(self.h, mid, s_["nodes"], s_["weights"])
            src = (sid, float(s_["f0"]), float(s_["t0"]), float(s_["amp"]))
        return LevelHandle(mid, qid, fid, level["dt"], level["n_steps"], level["p"], level["nu"],
                           lflts_mesh_info(self.h, mid), src)

    def grad(self, lv: LevelHandle, xi, precision=64, ckpt_every=16):
        """Host convenience: xi [S, K] -> (Q [S], dQ/dxi [S, K])."""
        xi = np.ascontiguousarray(xi, dtype=np.float64)
        S, K = xi.shape
        Q, G = np.zeros(S), np.zeros((S, K))
        lflts_grad_xi(self.h, lv.desc(precision), xi, S, ckpt_every, Q, G, LFLTS_MEM_HOST, None)
        return Q, G

    def solve(self, lv: LevelHandle, xi, precision=32, state=False, p=None):
        """Host convenience: xi [S, K] numpy -> Q [S] (and u_N [n_nodes, S])."""
        xi = np.ascontiguousarray(xi, dtype=np.float64)
        S = xi.shape[0]
        Q = np.zeros(S)
        uN = np.zeros((lv.info["n_nodes"], S)) if state else None
        lflts_solve(self.h, lv.desc(precision, p), xi, S, Q, uN, LFLTS_MEM_HOST, None)
        return (Q, uN) if state else Q
