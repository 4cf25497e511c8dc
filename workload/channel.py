"""The two-dimensional narrow channel with a random width (Sec. 4.3; inputs only).

Domain: two 0.95 x 1 rectangles, x in [-1, -0.05] and [0.05, 1], y in
[-0.5, 0.5], joined by a channel 0.1 long and b(w) wide centred at the
origin, b ~ U(0.001, 0.007).  Every draw is solved on one reference mesh of
the domain with the reference width b_bar = 0.004 whose vertices are moved by
the map of Eq. MeshTransform, (x, y) -> (x, y + phi(x) psi(y, w)):

* phi is 1 for |x| <= 0.05, 0 for |x| >= 0.1 and smooth in between; the
  paper does not give it, here it is the C^2 quintic step
  s(t) = 6 t^5 - 15 t^4 + 10 t^3 of t = (0.1 - |x|) / 0.05;
* psi(., w) is piecewise linear in y through 0 at y = 0 and y = +-0.5 and
  +-(b - b_bar)/2 at y = +-b_bar/2.

So the displacement of a vertex is xi(w) D(x, y) with one scalar per draw,
xi = (b - b_bar) / 2 in [-0.0015, 0.0015], and one displacement mode
D = (0, phi(x) psi_hat(y)), psi_hat the hat-shaped profile that is +-1 at
+-b_bar/2.  The wave speed is c = 1, the source is zero, the boundary
condition homogeneous Neumann (no Dirichlet node), u0 the compactly supported
bump centred at (0.5, 0) with radius 0.2, v0 = 0, T = 1, and the quantity of
interest the mean of u(., T) along the vertical line x = -0.4.

Reference mesh of level l: a grid of square cells of side H = 1 / (n0 2^l)
over [-1, 1] x [-0.5, 0.5], each split by its "/" diagonal; the coarse cells
of the box |x| <= 0.1, |y| <= 1/n0 refined p-fold (h_f = H / p) and closed
by a ring of balanced fans as in ``workload.mesh.square_mesh``; then every
triangle whose centroid lies outside the domain (|x| < 0.05 and
|y| > b_bar/2) removed with the nodes it leaves unused.  With n0 = 60 and
p = 25 the channel walls y = +-0.002 are fine grid lines, the coarse size is
the paper's H_0 = 1/60 and h_f = 6.7e-4 (the paper: about 7.6e-4).  Node
coordinates come from an integer lattice, so coincident nodes are identified
exactly.  This module holds no arithmetic of the method.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .mesh import Mesh, _quad_tris, refined_mask_from_elements

B_BAR = 0.004
B_RANGE = (0.001, 0.007)


def smooth_cutoff(x: np.ndarray) -> np.ndarray:
    """phi(x): 1 for |x| <= 0.05, 0 for |x| >= 0.1, quintic step between."""
    t = np.clip((0.1 - np.abs(x)) / 0.05, 0.0, 1.0)
    return t * t * t * (t * (6.0 * t - 15.0) + 10.0)


def width_profile(y: np.ndarray, bbar: float = B_BAR) -> np.ndarray:
    """psi_hat(y): piecewise linear, 0 at y = 0 and +-0.5, +-1 at +-bbar/2."""
    y = np.asarray(y, dtype=np.float64)
    a = np.abs(y)
    inner = a / (0.5 * bbar)
    outer = (0.5 - a) / (0.5 - 0.5 * bbar)
    return np.sign(y) * np.where(a <= 0.5 * bbar, inner, np.clip(outer, 0.0, None))


def displacement_mode(mesh: Mesh, bbar: float = B_BAR) -> np.ndarray:
    """D [n_nodes, 2]: the vertex displacement per unit xi = (b - bbar) / 2."""
    D = np.zeros_like(mesh.xy)
    D[:, 1] = smooth_cutoff(mesh.xy[:, 0]) * width_profile(mesh.xy[:, 1], bbar)
    return D


def warped_xy(mesh: Mesh, D: np.ndarray, xi: float) -> np.ndarray:
    """Vertex coordinates of the mesh of one draw."""
    return mesh.xy + xi * D


def channel_mesh(n0: int = 60, level: int = 0, p: int = 25, bbar: float = B_BAR) -> Mesh:
    """Reference mesh of the channel domain (width bbar) on level `level`."""
    if n0 % 20 != 0:
        raise ValueError("n0 must be a multiple of 20 (x = +-0.05 and +-0.1 on grid lines)")
    s = 2 ** level
    nx, ny = 2 * n0 * s, n0 * s                 # coarse cells
    H = 1.0 / (n0 * s)
    L = n0 * s * p                               # lattice points per unit length
    wall = (1.0 / n0 - 0.5 * bbar) * L           # fine rows from the box bottom to the lower wall
    if abs(wall - round(wall)) > 1e-9:
        raise ValueError("the channel walls are not fine grid lines for this n0, p")
    I0, I1 = int(round(0.9 * n0 * s)), int(round(1.1 * n0 * s))   # |x| <= 0.1
    J0, J1 = (n0 * s) // 2 - s, (n0 * s) // 2 + s                  # |y| <= 1/n0

    # ---- coarse nodes outside the closed box ---------------------------------
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="ij")
    in_box = (ii >= I0) & (ii <= I1) & (jj >= J0) & (jj <= J1)
    outside = ~in_box
    order_mask = outside.T.ravel()
    n_coarse = int(order_mask.sum())
    cid = -np.ones((ny + 1) * (nx + 1), dtype=np.int64)
    cid[order_mask] = np.arange(n_coarse)
    cid = cid.reshape(ny + 1, nx + 1).T           # cid[i, j]
    X = [ii.T.ravel()[order_mask] * p]
    Y = [jj.T.ravel()[order_mask] * p]

    # ---- fine nodes of the closed box -------------------------------------
    nfx, nfy = (I1 - I0) * p, (J1 - J0) * p
    aa, bb = np.meshgrid(np.arange(nfx + 1), np.arange(nfy + 1), indexing="ij")
    fid = (n_coarse + bb * (nfx + 1) + aa).astype(np.int64)
    X.append(aa.T.ravel() + I0 * p)
    Y.append(bb.T.ravel() + J0 * p)
    bi, bj = np.nonzero(in_box)
    cid[bi, bj] = fid[(bi - I0) * p, (bj - J0) * p]
    Xall = np.concatenate(X).astype(np.int64)
    Yall = np.concatenate(Y).astype(np.int64)

    tris, refined = [], []
    ci, cj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    in_ext = (ci >= I0 - 1) & (ci <= I1) & (cj >= J0 - 1) & (cj <= J1)
    corner = ((ci == I0 - 1) | (ci == I1)) & ((cj == J0 - 1) | (cj == J1))
    regular = ~in_ext | corner
    ri, rj = ci[regular], cj[regular]
    t = _quad_tris(cid[ri, rj], cid[ri + 1, rj], cid[ri + 1, rj + 1], cid[ri, rj + 1])
    tris.append(t)
    refined.append(np.zeros(t.shape[0], dtype=np.uint8))
    fa, fb = np.meshgrid(np.arange(nfx), np.arange(nfy), indexing="ij")
    fa, fb = fa.ravel(), fb.ravel()
    t = _quad_tris(fid[fa, fb], fid[fa + 1, fb], fid[fa + 1, fb + 1], fid[fa, fb + 1])
    tris.append(t)
    refined.append(np.ones(t.shape[0], dtype=np.uint8))

    # ---- ring of balanced fans around the box -----------------------------
    def fine_id(Xc, Yc):
        return fid[Xc - I0 * p, Yc - J0 * p]

    fan, mid, cells = [], p // 2, []
    for j in range(J0, J1):
        cells.append(((I0 - 1, j), (I0, j), (I0, j + 1), (I0 - 1, j + 1)))
        cells.append(((I1 + 1, j + 1), (I1, j + 1), (I1, j), (I1 + 1, j)))
    for i in range(I0, I1):
        cells.append(((i + 1, J0 - 1), (i + 1, J0), (i, J0), (i, J0 - 1)))
        cells.append(((i, J1 + 1), (i, J1), (i + 1, J1), (i + 1, J1 + 1)))
    for A, C0, Cp, B in cells:
        a, b = cid[A[0], A[1]], cid[B[0], B[1]]
        dx, dy = Cp[0] - C0[0], Cp[1] - C0[1]
        c = [fine_id(C0[0] * p + k * dx, C0[1] * p + k * dy) for k in range(p + 1)]
        fan += [(a, c[k], c[k + 1]) for k in range(mid)]
        fan += [(b, c[k], c[k + 1]) for k in range(mid, p)]
        fan.append((a, c[mid], b))
    fan = np.asarray(fan, dtype=np.int64)
    tris.append(fan)
    refined.append(np.ones(fan.shape[0], dtype=np.uint8))
    tri = np.concatenate(tris)
    refined = np.concatenate(refined)

    # ---- cut the domain out: drop triangles outside, then unused nodes --------
    x = -1.0 + Xall / L
    y = -0.5 + Yall / L
    cx = x[tri].mean(axis=1)
    cy = y[tri].mean(axis=1)
    keep = ~((np.abs(cx) < 0.05) & (np.abs(cy) > 0.5 * bbar))
    tri, refined = tri[keep], refined[keep]
    used = np.zeros(Xall.shape[0], dtype=bool)
    used[tri.ravel()] = True
    new = -np.ones(Xall.shape[0], dtype=np.int64)
    new[used] = np.arange(int(used.sum()))
    tri = new[tri].astype(np.int32)
    xy = np.stack([x[used], y[used]], axis=1)
    n_nodes = xy.shape[0]
    dirichlet = np.zeros(n_nodes, dtype=np.uint8)   # homogeneous Neumann everywhere
    P = refined_mask_from_elements(tri, refined, n_nodes, dirichlet)
    return Mesh(xy=xy, tri=tri, dirichlet=dirichlet, P=P, refined=refined,
                H=H, h_f=H / p, p=p, box=(-0.1, 0.1, -1.0 / n0, 1.0 / n0),
                meta={"n0": n0, "level": level, "bbar": bbar, "lattice": L})


def bump_pulse(mesh: Mesh, x0=(0.5, 0.0), R: float = 0.2) -> np.ndarray:
    """u0 = exp(1 - R^2 / (R^2 - |x - x0|^2)) inside the disc of radius R, else 0."""
    r2 = (mesh.xy[:, 0] - x0[0]) ** 2 + (mesh.xy[:, 1] - x0[1]) ** 2
    out = np.zeros(mesh.n_nodes)
    inside = r2 < R * R
    out[inside] = np.exp(1.0 - R * R / (R * R - r2[inside]))
    return out


def line_mean_weights(mesh: Mesh, x_line: float = -0.4):
    """(idx, w): the mean of the P1 function along the grid line x = x_line,
    y in [-0.5, 0.5] (length 1): the trapezoidal weights of the line's nodes,
    exact for the piecewise linear trace."""
    on = np.nonzero(np.abs(mesh.xy[:, 0] - x_line) < 1e-12)[0]
    if on.size < 2:
        raise ValueError("the line is not a grid line of the mesh")
    order = on[np.argsort(mesh.xy[on, 1])]
    yy = mesh.xy[order, 1]
    if abs(yy[0] + 0.5) > 1e-12 or abs(yy[-1] - 0.5) > 1e-12:
        raise ValueError("the line does not span the domain")
    seg = np.diff(yy)
    w = np.zeros(order.size)
    w[:-1] += 0.5 * seg
    w[1:] += 0.5 * seg
    return order.astype(np.int32), w


def xi_width(seed: int, level: int, S: int, offset: int = 0, bbar: float = B_BAR) -> np.ndarray:
    """[S, 1] draws xi = (b - bbar) / 2 with b ~ U(0.001, 0.007) (Philox keyed by
    seed and level; draw k is the same whatever S is)."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 1000 + level]))
    b = rng.uniform(B_RANGE[0], B_RANGE[1], size=offset + S)[offset:]
    return (0.5 * (b - bbar)).reshape(S, 1)


@dataclass(frozen=True)
class ChannelConfig:
    name: str
    n0: int = 60            # coarse cells per unit length on level 0 (H_0 = 1/60)
    p_mesh: int = 25        # refinement of the channel box (h_f = H / p_mesh)
    samples: tuple = (256, 64, 16)
    T: float = 1.0
    nu: float = 0.01
    seed: int = 6
    precision: int = 32

    @property
    def levels(self) -> int:
        return len(self.samples)

    @property
    def p_lts(self) -> int:
        """Substeps of Alg. 2: the mesh ratio times bbar / b_min, because the
        narrowest draw compresses the channel's cells by b_min / bbar."""
        return self.p_mesh * int(math.ceil(B_BAR / B_RANGE[0] - 1e-12))


CONFIG_CHANNEL = ChannelConfig("channel60-p25-b-uniform")


def channel_level(cfg: ChannelConfig, level: int, n0: int | None = None) -> dict:
    """Reference mesh and deterministic inputs of one level (H halves with the
    level, the box refinement p_mesh stays)."""
    mesh = channel_mesh(cfg.n0 if n0 is None else n0, level, cfg.p_mesh)
    dt = 0.9 * mesh.H / math.sqrt(2.0)
    n_steps = int(math.ceil(cfg.T / dt - 1e-12))
    idx, w = line_mean_weights(mesh, -0.4)
    return {"mesh": mesh, "modes": displacement_mode(mesh)[None, :, :], "psi": np.zeros((mesh.n_tri, 1)),
            "u0": bump_pulse(mesh), "qoi_idx": idx, "qoi_w": w, "dt": cfg.T / n_steps, "n_steps": n_steps,
            "p": cfg.p_lts, "nu": cfg.nu, "T": cfg.T}
