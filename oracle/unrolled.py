"""Checkpointed unrolled backward through the inner iteration of Algorithm 2, a
cross-check of the implicit-differentiation gradient of the barrier-smoothed solution.

TEST INFRASTRUCTURE, like the rest of this package: only the tests import it.  Plain
PyTorch on the CPU in float64, written from the paper's equations; it shares nothing
with the GPU library.

What it computes.  Hold mu fixed and run K inner iterations of Algorithm 2 with the
relaxation of Sec. 4.2 from a fixed start (u_0, v_0):

    u~  = (I + Q)^{-1} (u + v)                    (Eq. Simple-Update:Affine, r = 0, xi fixed)
    u^  = alpha u~ + (1 - alpha) u                 (Sec. 4.2)
    x, s    = prox(x^ - s, mu/beta)                (Eqs. Simple-Update:Barrier-X, Dual)
    tau, kappa = prox(tau^ - kappa, mu/beta)       (Eqs. Simple-Update:Barrier-tau, Dual)
    y, theta = y^, theta^

where prox(omega, c) is the positive root x of x^2 - omega x - c = 0 and s = x - omega.
Q is the skew-symmetric matrix of the embedding (Sec. 3.1), affine in (A, b, c) through
bbar = b - A e, cbar = c - e, zbar = c^T e + 1.  The gradient of L(x_K / tau_K) with
respect to (A, b, c) is taken by reverse-mode differentiation through all K iterations.
The iterate tends to the ADMM fixed point at mu, the central point of system HSD-log-kkt
with x o s = mu/beta e (Theorem 3.1), and, since the iteration map is a contraction near
it, the derivative of the K-th iterate tends to the derivative of the fixed point: the
implicit gradient, with an error that falls geometrically in K.

Checkpointing: the K iterations run in segments; the forward pass keeps only each
segment's starting state, and the backward pass recomputes one segment at a time
(torch.utils.checkpoint), so memory holds O(K / segment + segment) states.
"""
from __future__ import annotations

from typing import Callable

import numpy as np
import torch
from torch.utils.checkpoint import checkpoint


def embedding_matrix(A: torch.Tensor, b: torch.Tensor, c: torch.Tensor) -> torch.Tensor:
    """Q of Sec. 3.1 as a dense matrix, block order (y, x, tau, theta):
        [ 0       A      -b     bbar ]
        [-A^T     0       c    -cbar ]
        [ b^T    -c^T     0     zbar ]
        [-bbar^T  cbar^T -zbar  0    ]"""
    m, n = A.shape
    bbar = b - A.sum(dim=1)
    cbar = c - 1.0
    zbar = (c.sum() + 1.0).reshape(1)
    z1 = torch.zeros(1, dtype=A.dtype)
    rows = [
        torch.cat([torch.zeros(m, m, dtype=A.dtype), A, -b[:, None], bbar[:, None]], dim=1),
        torch.cat([-A.T, torch.zeros(n, n, dtype=A.dtype), c[:, None], -cbar[:, None]], dim=1),
        torch.cat([b, -c, z1, zbar])[None, :],
        torch.cat([-bbar, cbar, -zbar, z1])[None, :],
    ]
    return torch.cat(rows, dim=0)


def _prox(omega: torch.Tensor, cmu: float):
    """(x, s) with x the positive root of x^2 - omega x - cmu = 0 and s = x - omega, each
    root formed without cancellation (both forms are finite for cmu > 0, so the branch not
    taken contributes a zero gradient)."""
    D = torch.sqrt(omega * omega + 4.0 * cmu)
    pos = omega >= 0
    x = torch.where(pos, 0.5 * (omega + D), 2.0 * cmu / (D - omega))
    s = torch.where(pos, 2.0 * cmu / (omega + D), 0.5 * (D - omega))
    return x, s


def _iterate(P: torch.Tensor, m: int, n: int, xi: float, cmu: float, alpha: float, count: int,
             y, x, tau, theta, s, kappa):
    """`count` inner iterations from (y, x, tau, theta, s, kappa); P = (I + Q)^{-1}."""
    for _ in range(count):
        w = torch.cat([y, x + s, (tau + kappa).reshape(1), (theta + xi).reshape(1)])
        ut = P @ w
        yh = alpha * ut[:m] + (1.0 - alpha) * y
        xh = alpha * ut[m:m + n] + (1.0 - alpha) * x
        th = alpha * ut[m + n] + (1.0 - alpha) * tau
        thh = alpha * ut[m + n + 1] + (1.0 - alpha) * theta
        x, s = _prox(xh - s, cmu)
        tau, kappa = _prox(th - kappa, cmu)
        y, theta = yh, thh
    return y, x, tau, theta, s, kappa


def unrolled_grad(A, b, c, mu: float, dl_dxstar: Callable, start: dict, iters: int,
                  segment: int = 100, beta: float = 1.0, alpha: float = 1.8) -> dict:
    """Gradient of L(x*) with respect to (A, b, c), x* = x_K / tau_K after `iters` inner
    iterations at mu from `start` (keys y, x, tau, theta, s, kappa; held constant), by
    reverse mode through the iterations, `segment` iterations per checkpoint.

    dl_dxstar(xstar) returns dL/dx* (numpy in and out), evaluated at x_K / tau_K; the
    backward pass differentiates g^T x* with that g held fixed, as an adjoint does.
    Returns dA, db, dc, xstar and `change`: the max-norm of the last iteration's change of
    u = (y, x, tau, theta), a measure of how near the fixed point the iterate ended."""
    if iters < 1 or segment < 1:
        raise ValueError("iters and segment must be >= 1")
    At = torch.tensor(np.asarray(A, dtype=np.float64), requires_grad=True)
    bt = torch.tensor(np.asarray(b, dtype=np.float64), requires_grad=True)
    ct = torch.tensor(np.asarray(c, dtype=np.float64), requires_grad=True)
    m, n = At.shape
    xi = -float(n) - 1.0
    cmu = mu / beta
    P = torch.linalg.inv(torch.eye(m + n + 2, dtype=torch.float64) + embedding_matrix(At, bt, ct))
    state = tuple(torch.as_tensor(np.asarray(start[k], dtype=np.float64)).reshape(-1 if k in ("y", "x", "s") else ())
                  for k in ("y", "x", "tau", "theta", "s", "kappa"))

    def run(count, *st):
        return _iterate(P, m, n, xi, cmu, alpha, count, *st)

    done = 0
    prev_u = None
    while done < iters:
        count = min(segment, iters - done)
        if done + count == iters:               # keep the last step's input for `change`
            if count > 1:
                state = checkpoint(run, count - 1, *state, use_reentrant=False)
            prev_u = torch.cat([state[0], state[1], state[2].reshape(1), state[3].reshape(1)]).detach()
            state = run(1, *state)
        else:
            state = checkpoint(run, count, *state, use_reentrant=False)
        done += count
    y, x, tau, theta, s, kappa = state
    xstar = x / tau
    g = torch.as_tensor(np.asarray(dl_dxstar(xstar.detach().numpy()), dtype=np.float64))
    (g * xstar).sum().backward()
    u = torch.cat([y, x, tau.reshape(1), theta.reshape(1)]).detach()
    return dict(dA=At.grad.numpy(), db=bt.grad.numpy(), dc=ct.grad.numpy(),
                xstar=xstar.detach().numpy(), change=float((u - prev_u).abs().max()))
