"""Differentiable LP layer: x*(A, b, c) for  min c^T x  s.t.  A x = b, x >= 0.

x* = x / tau is the solution the ADMM inner loop returns at the final mu; its gradient
is that of the central point of the homogeneous self-dual embedding at that mu
(system HSD-log-kkt, Sec. 3.2), of which the ADMM iterate is the fixed point.
Forward: `abip_solve_batch` (dense instances, one persistent launch).  Backward:
`abip_backward_batch` (damped Newton polish onto the central point, then the adjoint
through the LU factors of the reduced KKT matrix K = Q + diag(0, S X^-1, kappa/tau, 0),
one CTA per instance).  Both run in the library's CUDA kernels;
this module only marshals tensors.
"""
from __future__ import annotations

import torch

from . import abip as _abip

_OK = (_abip.ABIP_OPTIMAL, _abip.ABIP_MAX_ITER)


class LPBatchFunction(torch.autograd.Function):
    """A [B, m, n], b [B, m], c [B, n] float64 (CUDA or CPU) -> x* [B, n]."""

    @staticmethod
    def forward(ctx, A, b, c, params: dict):
        prm = _abip.default_params(**(params or {}))
        B = A.shape[0]
        As = [A[k].detach().contiguous() for k in range(B)]
        bs = [b[k].detach().contiguous() for k in range(B)]
        cs = [c[k].detach().contiguous() for k in range(B)]
        infos, xs, ys, ss = _abip.abip_solve_batch(As, bs, cs, prm, device_out=A.is_cuda)
        bad = [k for k, f in enumerate(infos) if f["status"] not in _OK]
        if bad:
            raise _abip.AbipError(_abip.ABIP_E_NUMERICAL,
                                  f"instances {bad[:8]} ended {[infos[k]['status_name'] for k in bad[:8]]}: "
                                  "x* is not defined")
        out = torch.stack([torch.as_tensor(x, dtype=torch.float64) for x in xs]).to(A.device)
        ctx.prm = prm
        ctx.data = (As, bs, cs, xs, ys, ss, infos)
        ctx.infos = infos
        return out

    @staticmethod
    def backward(ctx, grad):
        As, bs, cs, xs, ys, ss, infos = ctx.data
        want = tuple(k for k, need in zip(("A", "b", "c"), ctx.needs_input_grad[:3]) if need)
        if not want:
            return None, None, None, None
        g = grad.detach().to(torch.float64).contiguous()
        gs = [g[k] if g.is_cuda else g[k].numpy() for k in range(g.shape[0])]
        dcs, dbs, dAs = _abip.abip_backward_batch(As, bs, cs, xs, ys, ss, infos, gs, ctx.prm, want=want,
                                                  device=grad.is_cuda)

        def stack(lst):
            if lst[0] is None:
                return None
            return torch.stack([torch.as_tensor(t, dtype=torch.float64) for t in lst]).to(grad.device)
        return stack(dAs), stack(dbs), stack(dcs), None


def lp_solve(A: torch.Tensor, b: torch.Tensor, c: torch.Tensor, **params) -> torch.Tensor:
    """x* of one LP ([m, n], [m], [n]) or a batch ([B, m, n], [B, m], [B, n]); differentiable
    in A, b and c.  `params` are abip_params fields (eps, max_admm_iters, ...)."""
    if A.dim() == 2:
        return LPBatchFunction.apply(A.unsqueeze(0), b.unsqueeze(0), c.unsqueeze(0), params)[0]
    return LPBatchFunction.apply(A, b, c, params)
