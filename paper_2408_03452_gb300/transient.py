"""Backward-Euler time stepping of the slightly compressible pressure problem.

Each step solves A p^{n+1} = q + d p^n (+ Dirichlet lifts): the linear
system of one Newton step (Section II.A, Eq. 5) of the implicit residual,
which is exact in one step because the problem is linear.  The accumulation
diagonal d = c V / dt is the one the coefficients were built with.  Every
step runs in the library's kernels: tpfa_build_rhs_transient, then cg_solve
started from p^n.
"""
from __future__ import annotations

import torch


def run(ctx, coef, coef64, K, p0, steps, d=None, d_uniform=0.0, dirichlet=None, q=None,
        pD=None, src_idx=None, src_val=None, tol=1e-8, maxit=200000):
    """Advance `steps` time steps from p0 (float64 [N] on the context's device).
    Returns (list of pressures p^1..p^steps, list of cg_solve infos)."""
    p = p0.clone()
    b = torch.empty_like(p0)
    out, infos = [], []
    for _ in range(steps):
        ctx.build_rhs_transient(K, p, dirichlet=dirichlet, q=q, pD=pD, src_idx=src_idx,
                                src_val=src_val, d=d, d_uniform=d_uniform, b=b)
        x = p.clone()  # warm start from the previous step
        x, info = ctx.cg_solve(coef, coef64, b, x=x, tol=tol, maxit=maxit)
        out.append(x)
        infos.append(info)
        p = x
    return out, infos
