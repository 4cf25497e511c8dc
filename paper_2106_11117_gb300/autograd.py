"""torch.autograd.Function around the CUDA solve and its adjoint.

``lflts_qoi(ctx, level, xi)`` returns Q(xi) [S] for draws xi [S, K] (CUDA,
float64); ``Q.backward(gQ)`` puts sum_s gQ[s] dQ[s]/dxi into xi.grad, with
dQ/dxi from ``lflts_grad_xi`` (discrete adjoint, forward recomputation from
checkpoints every ``ckpt_every`` steps).  The forward pass runs
``lflts_solve``; the backward pass reruns the forward inside the adjoint, so
nothing is kept between the two but the draws.
"""
from __future__ import annotations

import torch

from . import lflts


class _LFLTSQoI(torch.autograd.Function):
    @staticmethod
    def forward(fctx, xi, handle, desc_tuple, ckpt_every):
        desc = lflts.SolveDesc(*desc_tuple)
        xi = xi.detach().contiguous()
        S = xi.shape[0]
        Q = torch.empty(S, dtype=torch.float64, device=xi.device)
        st = torch.cuda.current_stream(xi.device).cuda_stream
        lflts.lflts_solve(handle, desc, xi, S, Q, None, lflts.LFLTS_MEM_DEVICE, st)
        fctx.save_for_backward(xi)
        fctx.handle, fctx.desc_tuple, fctx.ckpt_every = handle, desc_tuple, ckpt_every
        return Q

    @staticmethod
    def backward(fctx, gQ):
        (xi,) = fctx.saved_tensors
        S, K = xi.shape
        desc = lflts.SolveDesc(*fctx.desc_tuple)
        Q = torch.empty(S, dtype=torch.float64, device=xi.device)
        G = torch.empty(S, K, dtype=torch.float64, device=xi.device)
        st = torch.cuda.current_stream(xi.device).cuda_stream
        lflts.lflts_grad_xi(fctx.handle, desc, xi, S, fctx.ckpt_every, Q, G, lflts.LFLTS_MEM_DEVICE, st)
        return gQ.to(torch.float64)[:, None] * G, None, None, None


def lflts_qoi(ctx: "lflts.Context", level: "lflts.LevelHandle", xi: torch.Tensor, precision: int = 64,
              ckpt_every: int = 16) -> torch.Tensor:
    """Q(xi) with a hand-written adjoint for xi.grad (xi: CUDA float64 [S, K])."""
    if xi.dtype != torch.float64 or not xi.is_cuda or xi.dim() != 2:
        raise ValueError("xi must be a CUDA float64 tensor [S, K]")
    d = level.desc(precision)
    desc_tuple = (d.mesh_id, d.qoi_id, d.u0_field, d.v0_field, d.precision, d.p, d.nu, d.dt, d.n_steps,
                  d.source_id, d.src_f0, d.src_t0, d.src_amp)
    return _LFLTSQoI.apply(xi, ctx.h, desc_tuple, int(ckpt_every))
