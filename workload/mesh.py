"""Locally refined triangle meshes of the unit square (inputs only).

The paper (Sec. 3.2, Fig. 1) considers meshes whose coarse part has mesh size
H and whose small region D_fine is refined to h_f = H / p, and (Sec. 3.3)
identifies through the diagonal 0/1 matrix P the degrees of freedom of the
refined part *and of all elements adjacent to it*.  This module builds such a
conforming P1 mesh:

* a uniform n x n grid of square cells on [0,1]^2, each split by its "/"
  diagonal into two triangles;
* a box of whole coarse cells [I0,I1) x [J0,J1) refined p-fold in both
  directions (each fine cell again split by its "/" diagonal);
* one ring of coarse cells around the box closes the mesh without hanging
  nodes: a ring cell that shares an edge with the box carries the p+1 fine
  nodes of that edge and is triangulated as a balanced fan (half of the fine
  edge segments fanned from each of the two far corners plus one middle
  triangle); the four corner ring cells are ordinary coarse cells.

Fine-box and fan triangles are the *refined* elements.  The mask P marks
every vertex of a refined element and every vertex of an element that shares
a vertex with a refined element; Dirichlet nodes (the boundary of the square)
are never in P.

Node coordinates are generated on an integer lattice of spacing 1/(n p), so
coincident nodes are identified exactly.  Everything is vectorised with numpy
so that meshes with several million nodes build in seconds.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Mesh:
    """A P1 triangle mesh plus the inputs the method needs on it.

    xy         float64 [n_nodes, 2]  node coordinates
    tri        int32   [n_tri, 3]    vertex indices, counter-clockwise
    dirichlet  uint8   [n_nodes]     1 on the homogeneous Dirichlet boundary
    P          uint8   [n_nodes]     the LTS mask P (1 = refined region + adjacent)
    refined    uint8   [n_tri]       1 for elements that need the small step
    H, h_f     float                 coarse and fine mesh sizes (cell edge)
    p          int                   coarse-to-fine ratio H / h_f
    box        tuple                 refined box (x0, x1, y0, y1) after snapping
    """
    xy: np.ndarray
    tri: np.ndarray
    dirichlet: np.ndarray
    P: np.ndarray
    refined: np.ndarray
    H: float
    h_f: float
    p: int
    box: tuple | None
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.xy.shape[0])

    @property
    def n_tri(self) -> int:
        return int(self.tri.shape[0])

    @property
    def n_free(self) -> int:
        return int(self.n_nodes - int(self.dirichlet.sum()))


def refined_mask_from_elements(tri: np.ndarray, refined: np.ndarray,
                               n_nodes: int, dirichlet: np.ndarray) -> np.ndarray:
    """P = vertices of refined elements and of every element sharing a vertex
    with a refined element (Sec. 3.3: "the refined part ... and all elements
    adjacent to it"), restricted to free nodes."""
    v1 = np.zeros(n_nodes, dtype=bool)
    v1[tri[refined.astype(bool)].ravel()] = True
    touch = v1[tri].any(axis=1)
    P = np.zeros(n_nodes, dtype=bool)
    P[tri[touch].ravel()] = True
    P &= ~dirichlet.astype(bool)
    return P.astype(np.uint8)


def _snap_box(box, n):
    x0, x1, y0, y1 = box
    I0 = int(np.floor(x0 * n + 1e-9))
    I1 = int(np.ceil(x1 * n - 1e-9))
    J0 = int(np.floor(y0 * n + 1e-9))
    J1 = int(np.ceil(y1 * n - 1e-9))
    return I0, I1, J0, J1


def _quad_tris(v00, v10, v11, v01):
    """Two counter-clockwise triangles of cells split by the "/" diagonal."""
    t1 = np.stack([v00, v10, v11], axis=-1).reshape(-1, 3)
    t2 = np.stack([v00, v11, v01], axis=-1).reshape(-1, 3)
    return np.concatenate([t1, t2], axis=0)


def square_mesh(n: int, box=None, p: int = 1, box_cells=None) -> Mesh:
    """Unit square, n x n coarse cells, optional box refined p-fold.

    box        (x0, x1, y0, y1) in [0,1]; snapped outward to coarse grid lines
    box_cells  (I0, I1, J0, J1) coarse cell range; overrides ``box``.  Use it
               to keep the same physical box on a hierarchy of levels.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    refine = (box is not None or box_cells is not None) and p > 1
    if refine:
        I0, I1, J0, J1 = box_cells if box_cells is not None else _snap_box(box, n)
        if not (I0 >= 2 and J0 >= 2 and I1 <= n - 2 and J1 <= n - 2 and I1 > I0 and J1 > J0):
            raise ValueError("refined box and its ring must lie strictly inside the square")
    else:
        p = 1
    L = n * p  # integer lattice: coordinate X means x = X / L

    # ---- coarse nodes outside the closed box -------------------------------
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    if refine:
        in_box = (ii >= I0) & (ii <= I1) & (jj >= J0) & (jj <= J1)
    else:
        in_box = np.zeros_like(ii, dtype=bool)
    outside = ~in_box
    # row-major (y outer, x inner) numbering of the coarse nodes
    order_mask = outside.T.ravel()  # index j*(n+1)+i
    n_coarse = int(order_mask.sum())
    cid = -np.ones((n + 1) * (n + 1), dtype=np.int64)
    cid[order_mask] = np.arange(n_coarse)
    cid = cid.reshape(n + 1, n + 1).T  # cid[i, j]
    X = [ (ii.T.ravel()[order_mask]) * p ]
    Y = [ (jj.T.ravel()[order_mask]) * p ]

    # ---- fine nodes in the closed box ---------------------------------------
    if refine:
        nfx, nfy = (I1 - I0) * p, (J1 - J0) * p
        aa, bb = np.meshgrid(np.arange(nfx + 1), np.arange(nfy + 1), indexing="ij")
        fid = (n_coarse + bb * (nfx + 1) + aa).astype(np.int64)  # fid[a, b]
        X.append((aa.T.ravel() + I0 * p))
        Y.append((bb.T.ravel() + J0 * p))
        # coarse nodes on/in the closed box are fine nodes
        bi, bj = np.nonzero(in_box)
        cid[bi, bj] = fid[(bi - I0) * p, (bj - J0) * p]
    Xall = np.concatenate(X).astype(np.int64)
    Yall = np.concatenate(Y).astype(np.int64)
    n_nodes = Xall.shape[0]
    xy = np.stack([Xall / L, Yall / L], axis=1).astype(np.float64)

    tris, refined_flags = [], []
    # ---- ordinary coarse cells ----------------------------------------------
    ci, cj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    if refine:
        in_ext = (ci >= I0 - 1) & (ci <= I1) & (cj >= J0 - 1) & (cj <= J1)
        corner = ((ci == I0 - 1) | (ci == I1)) & ((cj == J0 - 1) | (cj == J1))
        regular = ~in_ext | corner
    else:
        regular = np.ones_like(ci, dtype=bool)
    ri, rj = ci[regular], cj[regular]
    t = _quad_tris(cid[ri, rj], cid[ri + 1, rj], cid[ri + 1, rj + 1], cid[ri, rj + 1])
    tris.append(t)
    refined_flags.append(np.zeros(t.shape[0], dtype=np.uint8))

    if refine:
        # ---- fine cells of the box -----------------------------------------
        fa, fb = np.meshgrid(np.arange(nfx), np.arange(nfy), indexing="ij")
        fa, fb = fa.ravel(), fb.ravel()
        t = _quad_tris(fid[fa, fb], fid[fa + 1, fb], fid[fa + 1, fb + 1], fid[fa, fb + 1])
        tris.append(t)
        refined_flags.append(np.ones(t.shape[0], dtype=np.uint8))

        # ---- transition ring: balanced fans ---------------------------------
        def fine_id(Xc, Yc):
            return fid[(Xc - I0 * p), (Yc - J0 * p)]

        def corner_id(Xc, Yc):
            return cid[Xc // p, Yc // p]

        fan = []
        mid = p // 2
        # each ring cell: corners (A, C0, Cp, B) counter-clockwise with the fine
        # edge running from C0 to Cp; direction (dx, dy) is one fine step.
        cells = []
        for j in range(J0, J1):   # left ring: fine edge BR -> TR
            i = I0 - 1
            cells.append(((i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)))
        for j in range(J0, J1):   # right ring: fine edge TL -> BL
            i = I1
            cells.append(((i + 1, j + 1), (i, j + 1), (i, j), (i + 1, j)))
        for i in range(I0, I1):   # bottom ring: fine edge TR -> TL
            j = J0 - 1
            cells.append(((i + 1, j), (i + 1, j + 1), (i, j + 1), (i, j)))
        for i in range(I0, I1):   # top ring: fine edge BL -> BR
            j = J1
            cells.append(((i, j + 1), (i, j), (i + 1, j), (i + 1, j + 1)))
        for A, C0, Cp, B in cells:
            a = corner_id(A[0] * p, A[1] * p)
            b = corner_id(B[0] * p, B[1] * p)
            dx, dy = (Cp[0] - C0[0]), (Cp[1] - C0[1])
            c = [fine_id(C0[0] * p + k * dx, C0[1] * p + k * dy) for k in range(p + 1)]
            for k in range(mid):
                fan.append((a, c[k], c[k + 1]))
            for k in range(mid, p):
                fan.append((b, c[k], c[k + 1]))
            fan.append((a, c[mid], b))
        fan = np.asarray(fan, dtype=np.int64)
        tris.append(fan)
        refined_flags.append(np.ones(fan.shape[0], dtype=np.uint8))

    tri = np.concatenate(tris).astype(np.int32)
    refined = np.concatenate(refined_flags)
    dirichlet = ((Xall == 0) | (Xall == L) | (Yall == 0) | (Yall == L)).astype(np.uint8)
    if refine:
        P = refined_mask_from_elements(tri, refined, n_nodes, dirichlet)
        snapped = (I0 / n, I1 / n, J0 / n, J1 / n)
    else:
        P = np.zeros(n_nodes, dtype=np.uint8)
        snapped = None
    return Mesh(xy=xy, tri=tri, dirichlet=dirichlet, P=P, refined=refined,
                H=1.0 / n, h_f=1.0 / L, p=p, box=snapped,
                meta={"n": n, "box_cells": (I0, I1, J0, J1) if refine else None})


def lshape_graded_mesh(m: int, s: float = 2.0, q: int = 1) -> Mesh:
    """Graded mesh T_{m,s} of the L-shaped domain [-1,1]^2 minus [0,1]x[-1,0]
    (Sec. 3.5): six triangles of equal area share the reentrant corner C =
    (0,0); on every edge from C the m+1 layer points lie at |e| (k/m)^s,
    k = 0..m, and the k+1 points of layer k inside each triangle are spread
    uniformly, so each of the six triangles holds m^2 elements in m tiers.
    The first q tiers (the elements touching layers < q) are the refined
    region; P follows the same rule as for the square meshes."""
    C = np.array([0.0, 0.0])
    outer = [(0.0, -1.0), (-1.0, -1.0), (-1.0, 0.0), (-1.0, 1.0), (0.0, 1.0), (1.0, 1.0), (1.0, 0.0)]
    t = (np.arange(m + 1) / m) ** s
    pts, tris, tier = [], [], []
    index = {}

    def node(p):
        key = (float(p[0]), float(p[1]))
        if key not in index:
            index[key] = len(pts)
            pts.append(key)
        return index[key]

    for a, b in zip(outer[:-1], outer[1:]):
        A, B = np.array(a), np.array(b)
        ids = {}
        for k in range(m + 1):
            for j in range(k + 1):
                w = (j / k) if k else 0.0
                ids[(k, j)] = node(C + t[k] * ((1.0 - w) * (A - C) + w * (B - C)))
        for k in range(1, m + 1):
            for j in range(k):
                tris.append((ids[(k - 1, min(j, k - 1))], ids[(k, j)], ids[(k, j + 1)]))
                tier.append(k)
            for j in range(k - 1):
                tris.append((ids[(k - 1, j)], ids[(k, j + 1)], ids[(k - 1, j + 1)]))
                tier.append(k)
    xy = np.array(pts, dtype=np.float64)
    tri = np.array(tris, dtype=np.int64)
    V = xy[tri]
    area2 = ((V[:, 1, 0] - V[:, 0, 0]) * (V[:, 2, 1] - V[:, 0, 1])
             - (V[:, 2, 0] - V[:, 0, 0]) * (V[:, 1, 1] - V[:, 0, 1]))
    flip = area2 < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    tri = tri.astype(np.int32)
    x, y = xy[:, 0], xy[:, 1]
    eps = 1e-12
    on_outer = (np.abs(x + 1) < eps) | (np.abs(x - 1) < eps) | (np.abs(y + 1) < eps) | (np.abs(y - 1) < eps)
    on_notch = ((np.abs(x) < eps) & (y <= eps)) | ((np.abs(y) < eps) & (x >= -eps))
    dirichlet = (on_outer | on_notch).astype(np.uint8)
    tier = np.asarray(tier)
    refined = (tier <= q).astype(np.uint8)
    P = refined_mask_from_elements(tri, refined, xy.shape[0], dirichlet) if q > 0 else np.zeros(xy.shape[0], np.uint8)
    h1 = (1.0 / m) ** s  # radial size of the first tier (on the unit spokes)
    return Mesh(xy=xy, tri=tri, dirichlet=dirichlet, P=P, refined=refined, H=1.0 / m, h_f=h1, p=2 * q + 1,
                box=None, meta={"m": m, "s": s, "q": q, "tier": tier})
