"""Differentiable SGML solve: u = solve(delta L(sigma) u = f) with an adjoint backward.

Forward: the batch of all-Dirichlet problems is solved by libsgml (the cycle of Algorithm 3 repeated
on the residual, Sec. 2) to a relative residual `rtol`.
Backward: with J(u) and g = dJ/du, the adjoint lambda solves delta L^T lambda = g with homogeneous
Dirichlet values -- delta L is symmetric for Dirichlet problems (the link coefficients of Eq. 5,
(sigma_i + sigma_j) / 2, are symmetric), so this is the same solve -- and
    dJ/df = lambda,
    dJ/dsigma_m = kappa/(2h^2) sum_{o: m+o inside} w_o (lambda_{m+o} - lambda_m)(u_{m+o} - u_m)
(the derivative of Eq. 5's link coefficients, evaluated by the library's gradient kernel).
When memory is tight (`save_solution=False`) the forward solution is not kept but recomputed by a
second forward solve in the backward pass.

Only argument marshalling happens here; every solve and the gradient run in libsgml's CUDA kernels.
"""
from __future__ import annotations

import torch

from . import sgml


def _as_batch(x, dim):
    return x if x.dim() == dim + 1 else x.unsqueeze(0)


class SGMLSolve(torch.autograd.Function):
    """u = SGMLSolve.apply(f, sigma, grid, rtol, save_solution).

    f, sigma: CUDA float64 tensors of shape (B, N, ..., N) (or one problem without the batch axis),
    the paper's sign L u = f with L = div(sigma grad).  `grid` is an ``sgml.Grid`` of B problems of
    the matching sizes whose faces are all Dirichlet (their values are the forward boundary data).
    """

    @staticmethod
    def _solve(grid, f, sigma, rtol):
        grid.set_coeffs(-1, sigma)
        grid.set_source(-1, f)
        st, cyc, rel = grid.solve_to_tol(rtol)
        if st != sgml.OK:
            raise RuntimeError(f"SGML solve did not converge (status {st}, cycles {cyc}, rel {rel})")
        u = torch.empty_like(f)
        for b in range(grid.batch):
            grid.get_solution(b, u[b])
        return u

    @staticmethod
    def forward(ctx, f, sigma, grid, rtol=1e-12, save_solution=True):
        if not (f.is_cuda and sigma.is_cuda) or f.dtype != torch.float64 or sigma.dtype != torch.float64:
            raise TypeError("f and sigma must be CUDA float64 tensors")
        dim = grid.dim
        fb = _as_batch(f, dim).contiguous()
        sb = _as_batch(sigma, dim).contiguous()
        if fb.shape[0] != grid.batch:
            raise ValueError("batch size does not match the grid")
        u = SGMLSolve._solve(grid, fb, sb, rtol)
        ctx.grid, ctx.rtol, ctx.squeeze = grid, rtol, f.dim() == dim
        ctx.bc = {b: grid.bc[b] for b in range(grid.batch)}
        for faces, _ in ctx.bc.values():
            if any(t != sgml.DIRICHLET for t in faces[: 2 * dim]):
                raise ValueError("the adjoint needs all faces Dirichlet")
        if save_solution:
            ctx.save_for_backward(fb, sb, u)
        else:
            ctx.save_for_backward(fb, sb)
        ctx.saved_u = save_solution
        return u[0] if ctx.squeeze else u

    @staticmethod
    def backward(ctx, gu):
        grid, rtol = ctx.grid, ctx.rtol
        if ctx.saved_u:
            fb, sb, u = ctx.saved_tensors
        else:
            fb, sb = ctx.saved_tensors
            u = SGMLSolve._solve(grid, fb, sb, rtol)  # recompute the forward solution
        g = _as_batch(gu, grid.dim).contiguous().to(torch.float64)
        # adjoint: homogeneous Dirichlet values, source dJ/du
        dim = grid.dim
        for b in range(grid.batch):
            grid.set_bc(b, [sgml.DIRICHLET] * (2 * dim), [0.0] * (2 * dim))
        lam = SGMLSolve._solve(grid, g, sb, rtol)
        dsig = torch.empty_like(sb)
        for b in range(grid.batch):
            grid.sigma_gradient(b, lam[b], u[b], dsig[b])
        # restore the forward boundary data for the next forward call
        for b, (faces, values) in ctx.bc.items():
            grid.set_bc(b, faces, values)
        if ctx.squeeze:
            lam, dsig = lam[0], dsig[0]
        return lam, dsig, None, None, None


def solve(f, sigma, grid, rtol=1e-12, save_solution=True):
    """Differentiable solve of the all-Dirichlet problems held by `grid` (boundary values taken from
    the grid's current faces, which must all be Dirichlet)."""
    return SGMLSolve.apply(f, sigma, grid, rtol, save_solution)
