"""The hand-written adjoint (lflts_grad_xi) against the oracle's
tangent-linear derivative and central finite differences (needs a GB300).

Tolerances (relative to the largest |dQ/dxi| of the batch): FP64 adjoint vs
oracle tangent 1e-9, vs central differences 1e-4; FP32 adjoint vs oracle
tangent 2e-3 (FP32 states, FP64 accumulation)."""
import numpy as np
import pytest

from gpu_common import draws, rel_err, small_level

pytestmark = pytest.mark.gpu


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


def _oracle(lev, xi):
    from oracle.adjoint import tangent_gradient
    out = [tangent_gradient(lev, x) for x in xi]
    return np.array([o[0] for o in out]), np.array([o[1] for o in out])


@pytest.mark.parametrize("p", [2, 3, 5])
def test_fp64_adjoint_matches_tangent_and_fd(lf, ctx, p):
    from oracle.adjoint import fd_gradient
    lev = small_level(n=10, p=p, K=3, T=0.3)
    xi = draws(5, 3, seed=p)
    h = ctx.add_level(lev)
    Qo, Go = _oracle(lev, xi)
    Q, G = ctx.grad(h, xi, precision=64, ckpt_every=4)
    assert rel_err(Q, Qo) <= 1e-12
    assert rel_err(G, Go) <= 1e-9, rel_err(G, Go)
    fd = np.array([fd_gradient(lev, x) for x in xi[:2]])
    assert rel_err(G[:2], fd) <= 1e-4
    # checkpoint spacing changes nothing (same recomputed states)
    for k in (1, 7, 10**6):
        Qk, Gk = ctx.grad(h, xi, precision=64, ckpt_every=k)
        np.testing.assert_array_equal(Gk, G)
        np.testing.assert_array_equal(Qk, Q)


def test_fp32_adjoint(lf, ctx):
    lev = small_level(n=12, p=4, K=4, T=0.4)
    xi = draws(8, 4, seed=21)
    h = ctx.add_level(lev)
    Qo, Go = _oracle(lev, xi)
    Q, G = ctx.grad(h, xi, precision=32, ckpt_every=5)
    assert rel_err(Q, Qo) <= 1e-5
    assert rel_err(G, Go) <= 2e-3, rel_err(G, Go)


def test_adjoint_leapfrog_and_empty_mask(lf, ctx):
    """p = 1 and P = 0: the adjoint reduces to the leapfrog adjoint."""
    lev = small_level(n=10, p=3, K=3, T=0.3)
    lev = dict(lev, dt=lev["dt"] / 3, n_steps=lev["n_steps"] * 3)
    xi = draws(3, 3, seed=8)
    h = ctx.add_level(lev)
    G1 = ctx.grad(h, xi, precision=64)[1]
    h0 = ctx.add_level(lev, P=False)
    G0 = ctx.grad(h0, xi, precision=64)[1]
    from oracle.adjoint import tangent_gradient
    m = lev["mesh"]
    lev_lf = dict(lev, p=1)
    Go = np.array([tangent_gradient(lev_lf, x)[1] for x in xi])
    lev_p0 = dict(lev, mesh=m)
    assert rel_err(G0, Go) <= 1e-9
    # with the mask kept and p = 1 the scheme is leapfrog as well
    d = h.desc(64)
    d.p = 1
    Q, G = np.zeros(3), np.zeros((3, 3))
    lf.lflts_grad_xi(ctx.h, d, xi, 3, 8, Q, G)
    assert rel_err(G, Go) <= 1e-9


def test_autograd_function(lf, ctx):
    import torch
    from paper_2106_11117_gb300.autograd import lflts_qoi
    lev = small_level(n=10, p=3, K=3, T=0.3)
    h = ctx.add_level(lev)
    xi_np = draws(6, 3, seed=4)
    xi = torch.from_numpy(xi_np).cuda().requires_grad_(True)
    Q = lflts_qoi(ctx, h, xi, precision=64, ckpt_every=3)
    w = torch.linspace(0.5, 1.5, 6, dtype=torch.float64, device="cuda")
    (w * Q).sum().backward()
    _, G = ctx.grad(h, xi_np, precision=64)
    np.testing.assert_allclose(xi.grad.cpu().numpy(), w.cpu().numpy()[:, None] * G, rtol=1e-14, atol=1e-300)
    Qh = ctx.solve(h, xi_np, precision=64)
    np.testing.assert_array_equal(Q.detach().cpu().numpy(), Qh)


def test_adjoint_with_point_source(lf, ctx):
    from workload import point_source
    lev = small_level(n=10, p=3, K=3, T=0.3)
    nodes, w = point_source(lev["mesh"], (0.52, 0.49))
    lev = dict(lev, source={"nodes": nodes, "weights": w, "f0": 8.0, "t0": 0.12, "amp": 1.5})
    xi = draws(3, 3, seed=31)
    h = ctx.add_level(lev)
    Qo, Go = _oracle(lev, xi)
    Q, G = ctx.grad(h, xi, precision=64, ckpt_every=3)
    assert rel_err(Q, Qo) <= 1e-12
    assert rel_err(G, Go) <= 1e-9, rel_err(G, Go)


def test_fp32_adjoint_against_fd_on_the_adjoint_workload_mesh(lf, ctx):
    """The FP32 adjoint on the mesh of the adjoint workload (256^2 base cells,
    box refined 8x, p = 8, K = 16 field terms, 108 k free nodes) over a short
    horizon (120 outer steps, a QoI box next to the initial pulse, so that Q
    and its gradient are not small), against central differences of the FP64
    solve (delta = 1e-6, all 2K perturbed draws of every draw in one batch):
    within 1e-4 of each draw's largest |dQ/dxi_k|."""
    from workload import CONFIG_ADJOINT as cfg, box_qoi_weights, level_problem, xi_uniform
    lev = level_problem(cfg, 0)
    idx, g = box_qoi_weights(lev["mesh"], (0.25, 0.4, 0.25, 0.4))
    lev = dict(lev, n_steps=120, qoi_idx=idx, qoi_w=g)
    S, K, delta = 4, cfg.K, 1e-6
    xi = np.ascontiguousarray(xi_uniform(cfg.seed, 0, S, K))
    h = ctx.add_level(lev)
    Q32, G32 = ctx.grad(h, xi, precision=32, ckpt_every=16)
    pert = np.repeat(xi, 2 * K, axis=0).reshape(S, 2 * K, K)
    for k in range(K):
        pert[:, 2 * k, k] += delta
        pert[:, 2 * k + 1, k] -= delta
    Qp = ctx.solve(h, np.ascontiguousarray(pert.reshape(S * 2 * K, K)), precision=64).reshape(S, K, 2)
    fd = (Qp[:, :, 0] - Qp[:, :, 1]) / (2 * delta)
    Q64 = ctx.solve(h, xi, precision=64)
    assert np.abs(Q64).max() > 1e-2
    assert np.abs(Q32 - Q64).max() <= 1e-5 * np.abs(Q64).max()
    for s in range(S):
        scale = np.abs(fd[s]).max()
        assert scale > 0
        assert np.abs(G32[s] - fd[s]).max() <= 1e-4 * scale, (s, np.abs(G32[s] - fd[s]).max() / scale)
