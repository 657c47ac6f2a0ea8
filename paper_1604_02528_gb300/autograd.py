"""torch.autograd.Function over the GPU factorization and selected inversion.

    Z = SelInv.apply(ctx, A_vals)          # A_vals: FP64 CSC values on the device
    loss = (W * Z).sum(); loss.backward()  # A_vals.grad via the native adjoints

Forward: selinv_factor (LDL^T) then selinv_numeric; Z holds whole diagonal
blocks (the upper part mirrors the lower), and a loss may read any of its
entries: the adjoint folds a cotangent on an upper slot into its mirror.
Either direction raises SelinvError when the plan's status word reports a
zero pivot, a non-finite input or a wait that ran out.  Backward:
selinv_adjoint (leaves -> root, gathers of A^{-1}_{C,C} recomputed) then
selinv_factor_adjoint (root -> leaves), giving the derivative with respect to
each stored lower entry of A.  Both directions run entirely in the native
library; this module only forwards buffers.
"""
from __future__ import annotations

import torch

from . import _native as N
from .api import SelInvContext


class SelInv(torch.autograd.Function):
    @staticmethod
    def forward(fctx, sctx: SelInvContext, A_vals: torch.Tensor) -> torch.Tensor:
        if A_vals.dtype != torch.float64:
            raise TypeError("the adjoint path is FP64")
        A_vals = A_vals.contiguous()
        L, D = sctx.factor(A_vals)
        Z = sctx.selinv(L, D)
        _raise_on_status(sctx, "forward (selinv_factor, selinv_numeric)")
        fctx.sctx = sctx
        fctx.save_for_backward(L, D, Z)
        return Z

    @staticmethod
    def backward(fctx, Zbar: torch.Tensor):
        sctx: SelInvContext = fctx.sctx
        L, D, Z = fctx.saved_tensors
        Zbar = Zbar.contiguous()
        Lbar = torch.empty_like(L)
        Dbar = torch.empty_like(D)
        N.selinv_adjoint(sctx.plan, N.SELINV_F64, L, D, Z, Zbar, Lbar, Dbar)
        Abar = torch.empty(sctx.colptr[-1], dtype=torch.float64, device=L.device)
        N.selinv_factor_adjoint(sctx.plan, N.SELINV_F64, L, D, Lbar, Dbar, Abar)
        _raise_on_status(sctx, "backward (selinv_adjoint, selinv_factor_adjoint)")
        return None, Abar


def _raise_on_status(sctx: SelInvContext, what: str) -> None:
    """A zero pivot, a non-finite input or a wait that ran out is latched in
    the plan's device status word; surface it instead of returning values
    computed from it (reading the word waits for the plan's stream)."""
    st = sctx.status()
    if st != 0:
        raise N.SelinvError(st, what)


def selinv(sctx: SelInvContext, A_vals: torch.Tensor) -> torch.Tensor:
    return SelInv.apply(sctx, A_vals)
