"""Host-side checks of liblflts (no GPU): the library builds, loads and
exports every symbol include/lflts.h declares; its host-only functions (LTS
constants, mesh preparation on a host-only context) agree with the oracle
and with the mask rule."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2106_11117_gb300 import build, lflts
    build.build()
    return lflts


def _declared():
    src = open(os.path.join(ROOT, "include", "lflts.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lflts_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    lib.load()
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (lflts_[a-z_]+)", out))
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [d for d in declared if d not in exported]
    assert not missing, missing
    assert set(lib.EXPORTED) == set(declared)


def test_binding_constants_match_header(lib):
    """Status codes, memory kinds, options and kernel classes of the Python
    binding carry the values the header's enums give them."""
    src = open(os.path.join(ROOT, "include", "lflts.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    enum = {k: int(v) for k, v in re.findall(r"\b(LFLTS_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)}
    for name, value in enum.items():
        if name.startswith("LFLTS_KERNEL_"):
            cls = name[len("LFLTS_KERNEL_"):].lower()
            if cls != "classes":
                assert lib.KERNEL_CLASSES[cls] == value, name
        else:
            assert getattr(lib, name) == value, name
    assert len(lib.KERNEL_CLASSES) == enum["LFLTS_KERNEL_CLASSES"]
    assert enum["LFLTS_OPT_FUSED_INNER"] == 5 and enum["LFLTS_KERNEL_ADJ_EDGES"] == 6


@pytest.mark.parametrize("p,nu", [(1, 0.0), (2, 0.01), (4, 0.01), (8, 0.5), (16, 0.01)])
def test_library_constants_match_oracle(lib, p, nu):
    from oracle.lts import lts_constants
    dt = 3.7e-3
    L = lib.lflts_lts_constants(p, nu, dt)
    O = lts_constants(p, nu)
    assert L["delta"] == pytest.approx(O["delta"], rel=1e-15)
    assert L["omega"] == pytest.approx(O["omega"], rel=1e-14)
    # u-form coefficients of Alg. 2: c0 = 1/2 (dt/p)^2 2p^2/(omega delta), c_m = (dt/p)^2 2p^2/omega beta_{m+1/2}
    assert L["c0"] == pytest.approx(0.5 * (dt / p) ** 2 * 2 * p * p / (O["omega"] * O["delta"]), rel=1e-14)
    for m in range(1, p):
        assert L["beta"][m] == pytest.approx(O["beta"][m], rel=1e-14)
        assert L["c"][m] == pytest.approx((dt / p) ** 2 * 2 * p * p / O["omega"] * O["beta_half"][m], rel=1e-14)
    # away from P the scheme is leapfrog: the factor is dt^2 / 2 (Sec. 3.3)
    assert L["gamma"] == pytest.approx(0.5 * dt * dt, rel=1e-12)


def test_host_only_mesh_preparation(lib):
    from workload import psi_sine, square_mesh
    m = square_mesh(16, box=(0.4, 0.6, 0.4, 0.6), p=4)
    ctx = lib.lflts_create(-1)
    try:
        mid = lib.lflts_mesh_add(ctx, m.xy, m.tri, m.dirichlet, m.P, psi_sine(m, 5))
        info = lib.lflts_mesh_info(ctx, mid)
        order = lib.lflts_mesh_order(ctx, mid)
    finally:
        lib.lflts_destroy(ctx)
    free = ~m.dirichlet.astype(bool)
    P = m.P.astype(bool) & free
    touch = P[m.tri].any(axis=1)
    R = np.zeros(m.n_nodes, bool)
    R[m.tri[touch].ravel()] = True
    R &= free
    assert info["n_nodes"] == m.n_nodes and info["n_tri"] == m.n_tri
    assert info["n_free"] == free.sum() and info["n_P"] == P.sum() and info["n_R"] == R.sum()
    assert info["K"] == 5
    # edges with a nonzero stiffness entry: on the "/" grid the hypotenuses
    # carry none, every other edge with a free endpoint does
    from oracle.fem import stiffness
    Kfull = stiffness(m.xy, m.tri, np.ones(m.n_tri)).tocoo()
    off = (Kfull.row < Kfull.col) & (Kfull.data != 0) & (free[Kfull.row] | free[Kfull.col])
    assert info["n_edges"] == off.sum()
    nP_end = P[Kfull.row[off]] | P[Kfull.col[off]]
    assert info["n_edges_P"] == nP_end.sum()
    assert sorted(order.tolist()) == list(range(m.n_nodes))
    nP, nR, nF = info["n_P"], info["n_R"], info["n_free"]
    assert P[order[:nP]].all()
    assert R[order[nP:nR]].all() and not P[order[nP:nR]].any()
    assert free[order[nR:nF]].all() and not R[order[nR:nF]].any()
    assert not free[order[nF:]].any()
    # each group is in Morton (Z-curve) order of the coordinates
    lo, hi = m.xy.min(0), m.xy.max(0)
    q = ((m.xy - lo) * (65535.0 / (hi - lo))).astype(np.uint64)

    def spread(x):
        x = x & np.uint64(0xFFFF)
        for sh, mask in ((8, 0x00FF00FF), (4, 0x0F0F0F0F), (2, 0x33333333), (1, 0x55555555)):
            x = (x | (x << np.uint64(sh))) & np.uint64(mask)
        return x

    z = spread(q[:, 0]) | (spread(q[:, 1]) << np.uint64(1))
    for a, b in ((0, nP), (nP, nR), (nR, nF), (nF, m.n_nodes)):
        assert np.all(np.diff(z[order[a:b]].astype(np.int64)) >= 0)


def test_host_only_moving_mesh_keeps_every_edge(lib):
    """A mesh whose vertices move with the draw keeps the edges whose
    stiffness is zero on the reference mesh (the "/" diagonals, nonzero once
    the channel is squeezed) and refuses missing modes."""
    from workload.channel import channel_mesh, displacement_mode
    m = channel_mesh(20, 0)
    ctx = lib.lflts_create(-1)
    try:
        fixed = lib.lflts_mesh_info(ctx, lib.lflts_mesh_add(ctx, m.xy, m.tri, m.dirichlet, m.P,
                                                            np.zeros((m.n_tri, 1))))
        moving = lib.lflts_mesh_info(ctx, lib.lflts_mesh_add_moving(ctx, m.xy, m.tri, m.dirichlet, m.P,
                                                                    displacement_mode(m)[None]))
        with pytest.raises(ValueError):
            lib.lflts_mesh_add_moving(ctx, m.xy, m.tri, m.dirichlet, m.P, displacement_mode(m))
    finally:
        lib.lflts_destroy(ctx)
    e = np.sort(np.concatenate([m.tri[:, [0, 1]], m.tri[:, [1, 2]], m.tri[:, [2, 0]]]), axis=1)
    n_all = np.unique(e, axis=0).shape[0]
    assert moving["n_edges"] == n_all > fixed["n_edges"]
    assert moving["K"] == 1 and moving["n_R"] == fixed["n_R"] and moving["n_free"] == m.n_nodes


def test_invalid_mesh_rejected(lib):
    ctx = lib.lflts_create(-1)
    try:
        xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
        with pytest.raises(lib.LfltsError) as e:
            lib.lflts_mesh_add(ctx, xy, np.array([[0, 2, 1]]), np.zeros(3), None, np.zeros((1, 1)))
        assert e.value.code == lib.LFLTS_ERR_MESH
        with pytest.raises(lib.LfltsError) as e:
            lib.lflts_mesh_add(ctx, xy, np.array([[0, 1, 3]]), np.zeros(3), None, np.zeros((1, 1)))
        assert e.value.code == lib.LFLTS_ERR_MESH
        with pytest.raises(lib.LfltsError):
            lib.lflts_mesh_add(ctx, xy, np.array([[0, 1, 2]]), np.zeros(3), None, np.zeros((1, 17)))
    finally:
        lib.lflts_destroy(ctx)


def test_host_only_context_refuses_solves(lib):
    ctx = lib.lflts_create(-1)
    try:
        with pytest.raises(lib.LfltsError) as e:
            lib.lflts_field_add(ctx, 0, np.zeros(3))
        assert e.value.code == lib.LFLTS_ERR_ARG
    finally:
        lib.lflts_destroy(ctx)
