"""Differentiable receiver misfit through the C ABI.

``ReceiverMisfit`` is a torch.autograd.Function:

    J(lambda, mu, rho) = sum_s 1/2 || Q x_s - d_s ||^2,   H(lambda, mu, rho) x_s = b_s,

whose forward builds a solver context for the medium and solves all sources in
one batch (bah_solve), evaluates J and the adjoint sources on the device
(bah_misfit), and keeps the forward wavefields x_s as the checkpoint for the
backward pass.  The backward pass solves the adjoint systems H^H y_s =
Q^H (Q x_s - d_s) in one batch (bah_solve_adjoint) and forms the pointwise
gradient (bah_gradient).  Every numerical step runs in libbah's kernels; this
module only orders the calls.
"""
from __future__ import annotations

import numpy as np
import torch

from . import Solver, bah_gradient, bah_misfit, bah_solve, bah_solve_adjoint, BAH_OK


def receiver_indices(n, row, component=None):
    """Indices (into one padded vector) of the u_d faces of receiver line
    ``row`` along x_d, one per cell along x_1 (2-D)."""
    n1, n2 = n[0], n[1]
    comp = 1 if component is None else component
    return np.array([comp * n1 * n2 + row * n1 + i for i in range(n1)], dtype=np.int32)


class ReceiverMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, lam, mu, rho, gamma, omega, n, h, b, d, rec, opts, rtol):
        solver = Solver(n, h, lam.detach().cpu().numpy(), mu.detach().cpu().numpy(), rho.detach().cpu().numpy(),
                        np.asarray(gamma), float(omega), **(opts or {}))
        nrhs = b.shape[0]
        x = torch.zeros_like(b)
        status, stats = bah_solve(solver.ctx, b, x, nrhs, rtol)
        if status != BAH_OK:
            raise RuntimeError(f"forward solve did not converge: {stats}")
        adj = torch.empty_like(b)
        mis = torch.empty(nrhs, dtype=torch.float64, device=b.device)
        bah_misfit(solver.ctx, x, d, rec, rec.numel(), nrhs, adj, mis)
        ctx.solver, ctx.rtol, ctx.nrhs = solver, rtol, nrhs
        ctx.shape, ctx.dev = lam.shape, lam.device
        ctx.save_for_backward(x, adj)
        return mis.sum()

    @staticmethod
    def backward(ctx, gJ):
        x, adj = ctx.saved_tensors
        solver = ctx.solver
        y = torch.zeros_like(adj)
        status, stats = bah_solve_adjoint(solver.ctx, adj, y, ctx.nrhs, ctx.rtol)
        if status != BAH_OK:
            raise RuntimeError(f"adjoint solve did not converge: {stats}")
        ncell = int(np.prod(ctx.shape))
        g = torch.zeros(3, ncell, dtype=torch.float64, device=x.device)
        bah_gradient(solver.ctx, x, y, ctx.nrhs, g[0], g[1], g[2])
        g = (g * gJ).reshape((3,) + tuple(ctx.shape)).to(ctx.dev)
        solver.close()
        return g[0], g[1], g[2], None, None, None, None, None, None, None, None, None


def misfit(lam, mu, rho, gamma, omega, n, h, b, d, rec, opts=None, rtol=1e-6):
    """J(lambda, mu, rho) with autograd support (see ReceiverMisfit)."""
    return ReceiverMisfit.apply(lam, mu, rho, gamma, omega, n, h, b, d, rec, opts, rtol)
