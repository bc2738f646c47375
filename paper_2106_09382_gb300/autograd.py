"""torch.autograd wrappers of the CONCORD solve (argument marshalling only).

The forward pass is a solve of Eq. 1 on the library's state; the backward
pass is the library's implicit-differentiation adjoint (concord_adjoint and
concord_adjoint_data): no sweep is stored or replayed.  Gradients follow the
full-matrix convention (every entry of Omega, S and X an independent input).
"""
from __future__ import annotations

import torch

from . import concord as C


class SolveFromS(torch.autograd.Function):
    """Omega = argmin of Eq. 1 for the Gram S and lambda (0-dim tensor)."""

    @staticmethod
    def forward(ctx, S, lam, state, tol, max_sweeps, cg_tol):
        state.set_S(S.contiguous())
        r = state.run(float(lam), tol=tol, max_sweeps=max_sweeps)
        ctx.state, ctx.cg_tol, ctx.result = state, cg_tol, r
        return state.get_omega(torch.float64)

    @staticmethod
    def backward(ctx, g):
        st = ctx.state
        dS = None
        if ctx.needs_input_grad[0]:
            dS = torch.empty((st.p, st.p), dtype=torch.float64, device=g.device)
        info = st.adjoint(g.contiguous(), tol=ctx.cg_tol, dS_out=dS)
        dlam = torch.tensor(info.dlambda, dtype=torch.float64, device=g.device)
        return dS, dlam, None, None, None, None


class SolveFromX(torch.autograd.Function):
    """Omega = argmin of Eq. 1 for S = Z^T Z / n, Z = X after `prep`."""

    @staticmethod
    def forward(ctx, X, lam, state, prep, tol, max_sweeps, cg_tol):
        X = X.contiguous()
        r = state.solve_device(X, float(lam), tol=tol, max_sweeps=max_sweeps, prep=prep)
        ctx.state, ctx.prep, ctx.cg_tol, ctx.result = state, prep, cg_tol, r
        ctx.save_for_backward(X)
        return state.get_omega(torch.float64)

    @staticmethod
    def backward(ctx, g):
        (X,) = ctx.saved_tensors
        st = ctx.state
        info = st.adjoint(g.contiguous(), tol=ctx.cg_tol)
        dX = st.adjoint_data(X, ctx.prep) if ctx.needs_input_grad[0] else None
        dlam = torch.tensor(info.dlambda, dtype=torch.float64, device=g.device)
        return dX, dlam, None, None, None, None, None


def solve_S(S, lam, state, tol=1e-8, max_sweeps=10000, cg_tol=1e-10):
    lam = lam if torch.is_tensor(lam) else torch.tensor(float(lam), dtype=torch.float64)
    return SolveFromS.apply(S, lam, state, tol, max_sweeps, cg_tol)


def solve_X(X, lam, state, prep=C.PREP_STANDARDIZE, tol=1e-8, max_sweeps=10000, cg_tol=1e-10):
    lam = lam if torch.is_tensor(lam) else torch.tensor(float(lam), dtype=torch.float64)
    return SolveFromX.apply(X, lam, state, prep, tol, max_sweeps, cg_tol)
