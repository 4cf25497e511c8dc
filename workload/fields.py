"""Random-field basis, random draws, initial data, QoI weights and the
workload configurations (inputs only).

Workloads.  The paper's experiments (Sec. 4) use no public dataset; every
input here is synthetic and seeded.  The square workloads follow the
configurations this library is measured on:

* coefficient  c^2(x, w) = exp( sum_k xi_k(w) psi_k(x) ),
  psi_k(x, y) = sin(k pi x) sin(k pi y) / k^2, xi_k i.i.d. U(-1, 1)
  (a KL-style log-field; the paper's Sec. 4.1 field is an affine KL sum);
  psi_k is evaluated at the element centroid (one-point rule, the element
  coefficient is constant per triangle);
* initial data u0 = exp(-200 |x - (0.3, 0.3)|^2) interpolated at the nodes,
  v0 = 0 (Sec. 2.1 model problem with f = 0);
* QoI: the mean of u(., T) over the box [0.7, 0.8]^2, represented by weights
  g_i = |B|^-1 * integral over B of phi_i (exact P1 integrals over the
  clipped triangles), so Q = sum_i g_i u_i;
* time step: leapfrog on the "/"-split uniform grid is stable for
  dt <= H / (sqrt(2) c_max); with |xi_k| <= 1 the a-priori bound
  c_max = exp(0.5 * sum_k 1/k^2) holds for every sample, so all samples of a
  level step in lockstep with dt = T / ceil(T / (0.9 H / (sqrt(2) c_max))).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .mesh import Mesh, lshape_graded_mesh, square_mesh


# --------------------------------------------------------------------------
# random field basis and draws
# --------------------------------------------------------------------------
def centroids(mesh: Mesh) -> np.ndarray:
    return mesh.xy[mesh.tri].mean(axis=1)


def psi_sine(mesh: Mesh, K: int) -> np.ndarray:
    """psi[e, k-1] = sin(k pi x_e) sin(k pi y_e) / k^2 at the centroid of e."""
    c = centroids(mesh)
    k = np.arange(1, K + 1, dtype=np.float64)
    return (np.sin(np.pi * c[:, :1] * k) * np.sin(np.pi * c[:, 1:2] * k) / k**2).astype(np.float64)


def xi_uniform(seed: int, level: int, S: int, K: int, offset: int = 0) -> np.ndarray:
    """Draws xi[i, k] ~ U(-1, 1) for samples offset .. offset+S-1 of a level.

    Counter-based Philox stream keyed by (seed, level); sample i always gets
    the same row, whatever S and offset are."""
    ss = np.random.SeedSequence([int(seed), int(level)])
    gen = np.random.Generator(np.random.Philox(ss))
    if offset:
        gen.uniform(-1.0, 1.0, size=(offset, K))  # skip the earlier samples
    return gen.uniform(-1.0, 1.0, size=(S, K)).astype(np.float64)


def gaussian_bump(mesh: Mesh, center=(0.3, 0.3), a: float = 200.0) -> np.ndarray:
    """Nodal interpolant of exp(-a |x - center|^2), zero on Dirichlet nodes."""
    d2 = ((mesh.xy - np.asarray(center)) ** 2).sum(axis=1)
    u0 = np.exp(-a * d2)
    u0[mesh.dirichlet.astype(bool)] = 0.0
    return u0


# --------------------------------------------------------------------------
# QoI weights: exact box average of the P1 interpolant
# --------------------------------------------------------------------------
def _clip_polygon(poly, axis, value, keep_greater):
    out = []
    n = len(poly)
    for i in range(n):
        a, b = poly[i], poly[(i + 1) % n]
        ina = (a[axis] >= value) if keep_greater else (a[axis] <= value)
        inb = (b[axis] >= value) if keep_greater else (b[axis] <= value)
        if ina:
            out.append(a)
        if ina != inb:
            t = (value - a[axis]) / (b[axis] - a[axis])
            out.append(a + t * (b - a))
    return out


def _polygon_area_centroid(poly):
    P = np.asarray(poly)
    x, y = P[:, 0], P[:, 1]
    xn, yn = np.roll(x, -1), np.roll(y, -1)
    cr = x * yn - xn * y
    A = 0.5 * cr.sum()
    if abs(A) < 1e-300:
        return 0.0, np.zeros(2)
    cx = ((x + xn) * cr).sum() / (6 * A)
    cy = ((y + yn) * cr).sum() / (6 * A)
    return A, np.array([cx, cy])


def box_qoi_weights(mesh: Mesh, box=(0.7, 0.8, 0.7, 0.8)):
    """(idx int32, g float64) with Q(u) = sum g[k] u[idx[k]] = mean of u_h over box."""
    x0, x1, y0, y1 = box
    V = mesh.xy[mesh.tri]                      # [n_tri, 3, 2]
    lo, hi = V.min(axis=1), V.max(axis=1)
    inside = (lo[:, 0] >= x0) & (hi[:, 0] <= x1) & (lo[:, 1] >= y0) & (hi[:, 1] <= y1)
    touch = (hi[:, 0] > x0) & (lo[:, 0] < x1) & (hi[:, 1] > y0) & (lo[:, 1] < y1)
    partial = touch & ~inside
    w = np.zeros(mesh.n_nodes)
    # triangles inside the box: integral of phi_i = |T| / 3
    Vi = V[inside]
    area = 0.5 * np.abs((Vi[:, 1, 0] - Vi[:, 0, 0]) * (Vi[:, 2, 1] - Vi[:, 0, 1])
                        - (Vi[:, 2, 0] - Vi[:, 0, 0]) * (Vi[:, 1, 1] - Vi[:, 0, 1]))
    np.add.at(w, mesh.tri[inside].ravel(), np.repeat(area / 3.0, 3))
    # triangles cut by the box: clip, integrate the linear phi_i exactly
    for e in np.nonzero(partial)[0]:
        T = V[e]
        poly = [T[0].copy(), T[1].copy(), T[2].copy()]
        for axis, val, keep in ((0, x0, True), (0, x1, False), (1, y0, True), (1, y1, False)):
            poly = _clip_polygon(poly, axis, val, keep)
            if not poly:
                break
        if len(poly) < 3:
            continue
        A, c = _polygon_area_centroid(poly)
        if A <= 0:
            continue
        # barycentric coordinates of the clipped centroid
        M = np.array([[T[1, 0] - T[0, 0], T[2, 0] - T[0, 0]],
                      [T[1, 1] - T[0, 1], T[2, 1] - T[0, 1]]])
        l12 = np.linalg.solve(M, c - T[0])
        lam = np.array([1.0 - l12.sum(), l12[0], l12[1]])
        w[mesh.tri[e]] += A * lam
    w /= (x1 - x0) * (y1 - y0)
    w[mesh.dirichlet.astype(bool)] = 0.0
    idx = np.nonzero(w)[0].astype(np.int32)
    return idx, w[idx].astype(np.float64)


def point_source(mesh: Mesh, xs):
    """Load vector of a point source at xs: F_i = phi_i(xs), nonzero on the
    three vertices of the triangle containing xs (barycentric coordinates)."""
    xs = np.asarray(xs, dtype=np.float64)
    V = mesh.xy[mesh.tri]
    lo, hi = V.min(axis=1), V.max(axis=1)
    cand = np.nonzero((lo[:, 0] <= xs[0]) & (hi[:, 0] >= xs[0]) & (lo[:, 1] <= xs[1]) & (hi[:, 1] >= xs[1]))[0]
    for e in cand:
        T = V[e]
        M = np.array([[T[1, 0] - T[0, 0], T[2, 0] - T[0, 0]], [T[1, 1] - T[0, 1], T[2, 1] - T[0, 1]]])
        l12 = np.linalg.solve(M, xs - T[0])
        lam = np.array([1.0 - l12.sum(), l12[0], l12[1]])
        if (lam >= -1e-12).all():
            return mesh.tri[e].astype(np.int32), np.clip(lam, 0.0, 1.0)
    raise ValueError("point outside the mesh")


# --------------------------------------------------------------------------
# time step and configurations
# --------------------------------------------------------------------------
def coarse_dt(H: float, K: int, T: float, safety: float = 0.9):
    """(dt, n_steps): CFL-limited coarse step with the a-priori c_max bound."""
    cmax = math.exp(0.5 * sum(1.0 / k**2 for k in range(1, K + 1)))
    dt = safety * H / (math.sqrt(2.0) * cmax)
    n = int(math.ceil(T / dt - 1e-12))
    return T / n, n


@dataclass(frozen=True)
class SquareConfig:
    name: str
    n0: int                 # coarse cells per side on level 0
    box: tuple              # refined box, snapped on level 0 and kept fixed
    p: int                  # LTS ratio (constant over levels: h halves everywhere)
    K: int                  # random-field terms
    samples: tuple          # MLMC samples per level
    T: float = 1.0
    nu: float = 0.01        # stabilisation parameter
    seed: int = 1
    qoi_box: tuple = (0.7, 0.8, 0.7, 0.8)
    u0_center: tuple = (0.3, 0.3)
    u0_a: float = 200.0
    precision: int = 64

    @property
    def levels(self) -> int:
        return len(self.samples)


CONFIG_PLAIN = SquareConfig("square32-p4-K4-fp64", 32, (0.45, 0.55, 0.45, 0.55), 4, 4,
                            (256, 64, 16), seed=1, precision=64)
CONFIG_BATCHED = SquareConfig("square128-p8-K8-L5-fp32", 128, (0.45, 0.55, 0.45, 0.55), 8, 8,
                              (8192, 2048, 512, 128, 32), seed=2, precision=32)
CONFIG_ADJOINT = SquareConfig("square256-p8-K16-adjoint", 256, (0.45, 0.55, 0.45, 0.55), 8, 16,
                              (1024,), seed=4, precision=32)
CONFIG_BANDWIDTH = SquareConfig("square1024-p4-K8-bandwidth", 128, (0.375, 0.625, 0.375, 0.625), 4, 8,
                                (2048, 1024, 512, 256), seed=5, precision=32)


def _box_cells(cfg: SquareConfig):
    x0, x1, y0, y1 = cfg.box
    n = cfg.n0
    return (int(math.floor(x0 * n + 1e-9)), int(math.ceil(x1 * n - 1e-9)),
            int(math.floor(y0 * n + 1e-9)), int(math.ceil(y1 * n - 1e-9)))


def level_problem(cfg: SquareConfig, level: int, n0: int | None = None) -> dict:
    """Mesh and deterministic inputs of one level: the level-0 box is kept and
    H halves on every level (the LTS ratio p stays constant)."""
    base = cfg.n0 if n0 is None else n0
    scale = 2 ** level
    n = base * scale
    I0, I1, J0, J1 = _box_cells(SquareConfig(cfg.name, base, cfg.box, cfg.p, cfg.K, cfg.samples))
    mesh = square_mesh(n, p=cfg.p, box_cells=(I0 * scale, I1 * scale, J0 * scale, J1 * scale))
    dt, n_steps = coarse_dt(mesh.H, cfg.K, cfg.T)
    idx, g = box_qoi_weights(mesh, cfg.qoi_box)
    return {
        "mesh": mesh,
        "psi": psi_sine(mesh, cfg.K),
        "u0": gaussian_bump(mesh, cfg.u0_center, cfg.u0_a),
        "qoi_idx": idx,
        "qoi_w": g,
        "dt": dt,
        "n_steps": n_steps,
        "p": cfg.p,
        "nu": cfg.nu,
        "T": cfg.T,
    }


# --------------------------------------------------------------------------
# graded L-shape workload with a Ricker source and Gaussian draws
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class LShapeConfig:
    """L-shaped domain [-1,1]^2 minus [0,1]x[-1,0], mesh T_{m,s} graded toward the
    reentrant corner (Sec. 3.5), m_l = m0 2^l, s = 2; the first q_l tiers are
    refined and the LTS ratio is p_l = 2 q_l + 1 (the tier sizes grow like
    2k - 1, so the coarse step is set by tier q_l + 1).  c^2 = exp(sum_k xi_k
    psi_k), psi_k = sin(k pi (x+1)/2) sin(k pi (y+1)/2) / k^2, xi_k ~ N(0, sigma^2)
    (unbounded: each draw gets its own time step), Ricker source at (-0.5, 0.5),
    zero initial data, QoI = mean of u over [0.4, 0.6]^2 at T."""
    name: str = "lshape-graded-s2-K16-ricker"
    m0: int = 58
    s: float = 2.0
    q_levels: tuple = (1, 2, 4, 8)
    K: int = 16
    sigma: float = 0.5
    samples: tuple = (4096, 1024, 256, 64)
    T: float = 1.0
    nu: float = 0.01
    seed: int = 3
    source_xy: tuple = (-0.5, 0.5)
    f0: float = 10.0
    qoi_box: tuple = (0.4, 0.6, 0.4, 0.6)
    precision: int = 32

    @property
    def levels(self) -> int:
        return len(self.q_levels)


CONFIG_LSHAPE = LShapeConfig()


def psi_sine_lshape(mesh: Mesh, K: int) -> np.ndarray:
    c = centroids(mesh)
    k = np.arange(1, K + 1, dtype=np.float64)
    return (np.sin(np.pi * (c[:, :1] + 1) / 2 * k) * np.sin(np.pi * (c[:, 1:2] + 1) / 2 * k) / k**2)


def xi_gaussian(seed: int, level: int, S: int, K: int, sigma: float, offset: int = 0) -> np.ndarray:
    ss = np.random.SeedSequence([int(seed), int(level), 7])
    gen = np.random.Generator(np.random.Philox(ss))
    if offset:
        gen.normal(0.0, sigma, size=(offset, K))
    return gen.normal(0.0, sigma, size=(S, K)).astype(np.float64)


def lshape_level(cfg: LShapeConfig, level: int, m0: int | None = None) -> dict:
    m = (cfg.m0 if m0 is None else m0) * 2**level
    q = cfg.q_levels[level]
    mesh = lshape_graded_mesh(m, cfg.s, q)
    V = mesh.xy[mesh.tri]
    e = [np.linalg.norm(V[:, i] - V[:, (i + 1) % 3], axis=1) for i in range(3)]
    a2 = np.abs((V[:, 1, 0] - V[:, 0, 0]) * (V[:, 2, 1] - V[:, 0, 1]) - (V[:, 2, 0] - V[:, 0, 0]) * (V[:, 1, 1] - V[:, 0, 1]))
    r_in = a2 / (e[0] + e[1] + e[2])          # inradius = 2 area / perimeter
    coarse = ~mesh.refined.astype(bool)
    idx, g = box_qoi_weights(mesh, cfg.qoi_box)
    nodes, w = point_source(mesh, cfg.source_xy)
    return {"mesh": mesh, "psi": psi_sine_lshape(mesh, cfg.K), "u0": np.zeros(mesh.n_nodes),
            "qoi_idx": idx, "qoi_w": g, "p": 2 * q + 1, "nu": cfg.nu, "T": cfg.T,
            "h_min_coarse": float(2.0 * r_in[coarse].min()),
            "source": {"nodes": nodes, "weights": w, "f0": cfg.f0, "t0": 1.2 / cfg.f0, "amp": 1.0}}


def lshape_steps(level: dict, xi: np.ndarray, ladder: float = 1.25) -> np.ndarray:
    """Per-draw step counts: dt(w) = 0.5 h_min / c_max(w) with the bound
    c_max^2 <= exp(sum_k |xi_k| / k^2) of the draw, n = ceil(T / dt) rounded up
    to a geometric ladder (ratio 1.25) so that draws fall into few buckets."""
    k = np.arange(1, xi.shape[1] + 1, dtype=np.float64)
    cmax = np.exp(0.5 * (np.abs(xi) / k**2).sum(axis=1))
    n = np.ceil(level["T"] / (0.5 * level["h_min_coarse"] / cmax))
    base = np.ceil(level["T"] / (0.5 * level["h_min_coarse"]))
    j = np.ceil(np.log(n / base) / np.log(ladder) - 1e-12)
    return np.maximum(np.ceil(base * ladder ** np.maximum(j, 0)), 1).astype(np.int64)
