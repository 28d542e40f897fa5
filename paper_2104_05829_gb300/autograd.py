"""Differentiable Helmholtz solve u = A(h1, h2)^{-1} b(f) through libsem.

Forward: solve of R Q^T A_L Q R^T u = R Q^T B_L f_L in FP64, by Jacobi-PCG (the paper's
viscous-substep solver) or by flexible PCG with the p-multigrid V-cycle carrying the nodal
h1 to its coarse levels (precond="pmg", V-cycle in `prec`).
Backward (hand-written adjoint, using A = A^T): with g = dL/du_L,
    A lam = R Q^T g                      (one more solve, same solver)
    dL/df_L  = B_L lam_L                 (sem_mass_local)
    dL/dh1_L = -sum_{m,m'} (D_m lam) G_mm' (D_m' u)   (sem_grad_h1, eq. Ae)
No Krylov iterates are stored: the adjoint is re-solved.
"""
from __future__ import annotations

import torch


class HelmholtzSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, h1_L, sem, h2, tol, maxit, precond, prec, outer_pairs):
        h1 = h1_L.detach().contiguous()
        u, _ = sem.solve(f.detach().contiguous(), h1_L=h1, h2=h2, tol=tol, maxit=maxit, precond=precond, prec=prec,
                         outer_pairs=outer_pairs)
        ctx.sem, ctx.h2, ctx.tol, ctx.maxit, ctx.precond, ctx.prec = sem, h2, tol, maxit, precond, prec
        ctx.outer_pairs = outer_pairs
        ctx.save_for_backward(u, h1)
        return u

    @staticmethod
    def backward(ctx, gu):
        u, h1_L = ctx.saved_tensors
        sem = ctx.sem
        g = gu.detach().contiguous().clone()
        sem.gs(g)                                   # Q Q^T g: the adjoint right-hand side, replicated
        lam, _ = sem.solve(g, h1_L=h1_L, h2=ctx.h2, tol=ctx.tol, maxit=ctx.maxit, precond=ctx.precond,
                           prec=ctx.prec, rhs="assembled", outer_pairs=ctx.outer_pairs)
        df = sem.mass_local(lam) if ctx.needs_input_grad[0] else None
        dh1 = sem.grad_h1(u, lam) if ctx.needs_input_grad[1] else None
        return df, dh1, None, None, None, None, None, None, None


def helmholtz_solve(sem, f, h1_L, h2: float = 1.0, tol: float = 1e-10, maxit: int = 10000, precond: str = "jacobi",
                    prec: str = "fp64", outer_pairs: bool = False):
    """u_L = A(h1_L, h2)^{-1} R Q^T B_L f_L, differentiable in f_L and h1_L. precond "jacobi"
    (Jacobi-PCG) or "pmg" (flexible PCG + p-multigrid with the nodal h1, V-cycle in prec);
    outer_pairs: the outer operator in FP32-pair arithmetic (about 48 bits)."""
    return HelmholtzSolve.apply(f, h1_L, sem, float(h2), float(tol), int(maxit), precond, prec, bool(outer_pairs))
