"""Convenience layer over the C ABI: one object per sparsity pattern.

    ctx = SelInvContext(n, colptr, rowind, kind="relaxed", cap=128, fill=0.1)
    L, D = ctx.factor(A_vals)          # GPU LDL^T (prerequisite)
    Z = ctx.selinv(L, D)               # selected inverse, panel layout

All arithmetic runs in the native library; this module only allocates torch
buffers and forwards pointers.
"""
from __future__ import annotations

from typing import Optional, Tuple

import numpy as np

from . import _native as N

KIND = {"fundamental": 0, "relaxed": 1}


def torch_dtype(dtype: int):
    import torch
    return torch.float64 if dtype == N.SELINV_F64 else torch.complex128


def selinv_dtype_of(t, hermitian: bool = False) -> int:
    import torch
    if t.dtype == torch.complex128:
        return N.SELINV_C128H if hermitian else N.SELINV_C128
    if t.dtype == torch.float64:
        return N.SELINV_F64
    raise TypeError(f"unsupported dtype {t.dtype}: float64 or complex128")


class SelInvContext:
    """Symbolic analysis + device plan of one lower-CSC pattern."""

    def __init__(self, n: int, colptr, rowind, kind: str = "fundamental", cap: int = 64,
                 fill: float = 0.0, opts: Optional[N.selinv_opts] = None, hermitian: bool = False):
        self.n = int(n)
        self.hermitian = bool(hermitian)   # complex values are Hermitian (A = A^H), not symmetric
        self.colptr = np.ascontiguousarray(colptr, dtype=np.int64)
        self.rowind = np.ascontiguousarray(rowind, dtype=np.int32)
        self.analysis = N.selinv_analyse(self.n, self.colptr, self.rowind, KIND[kind], cap, fill)
        a = self.analysis
        self.nsuper = a["nsuper"]
        self.plan = N.selinv_symbolic(self.n, self.nsuper, a["super_ptr"], a["sparent"],
                                      a["rowptr"], a["rows"], opts)
        self._matrix_attached = False

    @classmethod
    def from_problem(cls, p, opts: Optional[N.selinv_opts] = None) -> "SelInvContext":
        sn = p.supernodes
        return cls(p.n, p.colptr, p.rowind, str(sn["kind"]), int(sn["cap"]), float(sn["fill"]), opts,
                   hermitian=bool(getattr(p, "hermitian", False)))

    @property
    def nnz(self) -> int:
        return self.plan.nnz

    def stats(self, dtype: int) -> Tuple[float, float]:
        return N.selinv_plan_stats(self.plan, dtype)

    def empty_panels(self, dtype: int, device="cuda"):
        import torch
        return torch.empty(self.nnz, dtype=torch_dtype(dtype), device=device)

    def set_options(self, **kw):
        o = N.selinv_default_opts()
        for k, v in kw.items():
            setattr(o, k, v)
        N.selinv_plan_set_opts(self.plan, o)

    def attach_matrix(self):
        if not self._matrix_attached:
            N.selinv_plan_set_matrix(self.plan, self.n, self.colptr, self.rowind)
            self._matrix_attached = True

    def factor(self, A_vals, L=None, D=None, stream=None):
        """L (panels) and D of A = L D L^T from A's CSC values on the device."""
        import torch
        dt = selinv_dtype_of(A_vals, self.hermitian)
        self.attach_matrix()
        if L is None:
            L = self.empty_panels(dt, A_vals.device)
        if D is None:
            D = torch.empty(self.n, dtype=A_vals.dtype, device=A_vals.device)
        N.selinv_factor(self.plan, dt, A_vals, L, D, stream)
        return L, D

    def selinv(self, L, D, out=None, stream=None):
        """Selected inverse on the pattern of L (panel layout)."""
        dt = selinv_dtype_of(L, self.hermitian)
        if out is None:
            out = self.empty_panels(dt, L.device)
        N.selinv_numeric(self.plan, dt, L, D, out, stream)
        return out

    def selinv_host(self, L_host, D_host, out=None, stream=None):
        """Selected inverse of host panels (CPU tensors; pinned for the copies
        to overlap the traversal), returned in a host tensor (pinned when it
        is allocated here).  The device staging buffers are kept on the
        context and reused; synchronizes the stream before returning."""
        import torch
        dt = selinv_dtype_of(L_host, self.hermitian)
        if out is None:
            out = torch.empty(self.nnz, dtype=torch_dtype(dt)).pin_memory()
        st = getattr(self, "_host_staging", None)
        if st is None or st[0].dtype != L_host.dtype:
            st = (torch.empty(self.nnz, dtype=L_host.dtype, device="cuda"),
                  torch.empty(self.n, dtype=D_host.dtype, device="cuda"),
                  torch.empty(self.nnz, dtype=L_host.dtype, device="cuda"))
            self._host_staging = st
        if stream is None:
            stream = torch.cuda.current_stream()
        N.selinv_numeric_host(self.plan, dt, L_host, D_host, out, st[0], st[1], st[2], stream)
        stream.synchronize()
        return out

    def select(self, rows, cols) -> np.ndarray:
        """Restrict later selected inversions to the entries (rows[e], cols[e])
        (and the supernodes they need); returns their panel positions.  Empty
        arrays restore the full inversion."""
        return N.selinv_plan_select(self.plan, rows, cols)

    def gather(self, Ainv, out=None, stream=None):
        """The selected entries of a panel array, in selection order."""
        import torch
        n = int(N.selinv_plan_selected(self.plan).size)
        if out is None:
            out = torch.empty(n, dtype=Ainv.dtype, device=Ainv.device)
        N.selinv_gather(self.plan, selinv_dtype_of(Ainv), Ainv, out, stream)
        return out

    def status(self) -> int:
        return N.selinv_status(self.plan)


def pole_sum(Ainvs, weights, pos, stream=None):
    """sum_l weights[l] * Ainvs[l][pos] on the device (complex128), e.g. a
    pole expansion of a matrix function's diagonal; pos: device int64 panel
    positions (from SelInvContext.select)."""
    import torch
    out = torch.empty(pos.numel(), dtype=torch.complex128, device=pos.device)
    N.selinv_pole_sum([selinv_dtype_of(z) for z in Ainvs], list(Ainvs), weights, pos, out, stream)
    return out
