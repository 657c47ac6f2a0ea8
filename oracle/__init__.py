"""CPU oracle for supernodal selected inversion -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  It wraps a plain C library
(``liboracle.so``, built from this directory by ``build.py``) that restates
the paper's definitions and algorithms with plain loops:

* ``symbolic``  -- elimination tree, column structures, supernodes (Sec. II-A)
* ``plan``      -- level of each supernode, the sets C of Alg. 1 split by
                   owning ancestor, and relative row indices
* ``ldlt``      -- LDL^T without pivoting on the supernodal pattern (Sec. IV)
* ``selinv``    -- Alg. 1 (pull), diagonal blocks symmetrized (Sec. II-C);
                   ``hermitian=True``: conjugate transposes, A = A^H
* ``selinv_levels`` -- the same per-supernode steps, one tree level at a time
                   on several host threads (bit for bit ``selinv``)
* ``selinv_push`` -- Alg. 2 (left-looking push), a different summation order
* ``lu``, ``selinv_lu`` -- nonsymmetric values: LU without pivoting (U kept
                   transposed in the panel layout) and Alg. 1 in its LU form
* ``selinv_adjoint``, ``ldlt_adjoint`` -- reverse mode of the two numeric steps
* ``panel_position``, ``needed_supernodes`` -- subset selection (Sec. I: all
  or a subset of the entries on the factors' pattern): where an entry of
  A^{-1} is stored, and which supernodes Alg. 1 must run to produce it
* ``pole_sum``  -- sum_l w_l A_l^{-1}[pos] over selected inverses of shifted
  matrices (the density-functional-theory use Sec. I names)

It shares no code with the GPU library.
"""
from __future__ import annotations

import ctypes as ct
import os
from dataclasses import dataclass
from typing import Dict, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def _load():
    global _lib
    if _lib is None:
        from . import build as _b
        path = _b.build()
        lib = ct.CDLL(path)
        P = ct.c_void_p
        lib.orc_symbolic.restype = P
        lib.orc_symbolic.argtypes = [ct.c_int32, P, P, ct.c_int, ct.c_int, ct.c_double,
                                     ct.POINTER(ct.c_int)]
        lib.orc_sym_get.restype = ct.c_int64
        lib.orc_sym_get.argtypes = [P, ct.c_int, P]
        lib.orc_sym_free.argtypes = [P]
        lib.orc_plan.restype = ct.c_int
        lib.orc_plan.argtypes = [ct.c_int32, P, P, P, P, P, P, P, P, P, P, P,
                                 ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int64)]
        for sfx in ("_d", "_z"):
            f = getattr(lib, "orc_ldlt" + sfx)
            f.restype = ct.c_int
            f.argtypes = [ct.c_int32, P, P, P, ct.c_int32, P, P, P, P, P, P]
            for name in ("orc_selinv", "orc_selinv_push"):
                f = getattr(lib, name + sfx)
                f.restype = ct.c_int
                f.argtypes = [ct.c_int32, P, P, P, P, P, P, P, ct.c_int]
            f = getattr(lib, "orc_selinv_top" + sfx)
            f.restype = ct.c_int
            f.argtypes = [ct.c_int32, P, P, P, P, P, P, P, ct.c_int, ct.c_int32]
            f = getattr(lib, "orc_selinv_adjoint" + sfx)
            f.restype = ct.c_int
            f.argtypes = [ct.c_int32, P, P, P, P, P, P, P, P, P, P]
            f = getattr(lib, "orc_solve" + sfx)
            f.restype = ct.c_int
            f.argtypes = [ct.c_int32, P, P, P, P, P, P, P]
            f = getattr(lib, "orc_ldlt_adjoint" + sfx)
            f.restype = ct.c_int
            f.argtypes = [ct.c_int32, P, P, P, P, P, P, P, P, P]
        for sfx in ("_d", "_z", "_h"):
            f = getattr(lib, "orc_selinv_levels" + sfx)
            f.restype = ct.c_int
            f.argtypes = [ct.c_int32, P, P, P, P, P, P, P, ct.c_int, ct.c_int32, ct.c_int]
        # complex Hermitian: the factorization and Alg. 1 only
        lib.orc_ldlt_h.restype = ct.c_int
        lib.orc_ldlt_h.argtypes = [ct.c_int32, P, P, P, ct.c_int32, P, P, P, P, P, P]
        lib.orc_selinv_h.restype = ct.c_int
        lib.orc_selinv_h.argtypes = [ct.c_int32, P, P, P, P, P, P, P, ct.c_int]
        lib.orc_selinv_top_h.restype = ct.c_int
        lib.orc_selinv_top_h.argtypes = [ct.c_int32, P, P, P, P, P, P, P, ct.c_int, ct.c_int32]
        # nonsymmetric values: LU and its Alg. 1
        for sfx in ("_d", "_z"):
            f = getattr(lib, "orc_lu" + sfx)
            f.restype = ct.c_int
            f.argtypes = [ct.c_int32, P, P, P, P, ct.c_int32, P, P, P, P, P, P]
            f = getattr(lib, "orc_selinv_lu" + sfx)
            f.restype = ct.c_int
            f.argtypes = [ct.c_int32, P, P, P, P, P, P, P, P]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ct.c_void_p)


@dataclass
class Sym:
    """Symbolic structure: column etree + supernodal partition and rows."""
    n: int
    parent: np.ndarray      # column elimination tree, -1 = root
    cstruct_ptr: np.ndarray
    cstruct: np.ndarray     # struct(j) of L, ascending, diagonal first
    super_ptr: np.ndarray   # int32 [nsuper+1]
    sparent: np.ndarray     # int32 [nsuper]
    rowptr: np.ndarray      # int64 [nsuper+1]
    rows: np.ndarray        # int32, per supernode: own columns then C
    nnz_true: int

    @property
    def nsuper(self) -> int:
        return int(self.super_ptr.size - 1)

    def sizes(self) -> Tuple[np.ndarray, np.ndarray]:
        """(s, c) per supernode."""
        s = np.diff(self.super_ptr).astype(np.int64)
        m = np.diff(self.rowptr).astype(np.int64)
        return s, m - s

    def panel_offsets(self) -> np.ndarray:
        s, c = self.sizes()
        off = np.zeros(self.nsuper + 1, dtype=np.int64)
        off[1:] = np.cumsum((s + c) * s)
        return off

    @property
    def nnz_panels(self) -> int:
        return int(self.panel_offsets()[-1])


ERRORS = {0: "ok", -1: "invalid argument", -2: "bad pattern", -4: "zero pivot", -5: "out of memory"}


def symbolic(n: int, colptr: np.ndarray, rowind: np.ndarray, kind: str = "fundamental",
             cap: int = 64, fill: float = 0.0) -> Sym:
    lib = _load()
    colptr = np.ascontiguousarray(colptr, dtype=np.int64)
    rowind = np.ascontiguousarray(rowind, dtype=np.int32)
    err = ct.c_int(0)
    h = lib.orc_symbolic(int(n), _p(colptr), _p(rowind), 1 if kind == "relaxed" else 0,
                         int(cap), float(fill), ct.byref(err))
    if not h:
        raise ValueError(f"oracle symbolic failed: {ERRORS.get(err.value, err.value)}")
    try:
        def get(field, dtype):
            cnt = lib.orc_sym_get(h, field, None)
            out = np.zeros(max(cnt, 0), dtype=dtype)
            if cnt > 0:
                lib.orc_sym_get(h, field, _p(out))
            return out
        sym = Sym(int(n), get(0, np.int32), get(1, np.int64), get(2, np.int32), get(3, np.int32),
                  get(4, np.int32), get(5, np.int64), get(6, np.int32), int(lib.orc_sym_get(h, 8, None)))
    finally:
        lib.orc_sym_free(h)
    return sym


def symbolic_for(problem) -> Sym:
    sn = problem.supernodes
    return symbolic(problem.n, problem.colptr, problem.rowind, str(sn["kind"]), int(sn["cap"]),
                    float(sn["fill"]))


def plan(sym: Sym) -> Dict[str, np.ndarray]:
    """Levels, owner segments of C and relative indices, from the definitions."""
    lib = _load()
    ns = sym.nsuper
    nseg, nrel = ct.c_int64(0), ct.c_int64(0)
    rc = lib.orc_plan(ns, _p(sym.super_ptr), _p(sym.sparent), _p(sym.rowptr), _p(sym.rows),
                      None, None, None, None, None, None, None, ct.byref(nseg), ct.byref(nrel))
    if rc != 0:
        raise ValueError("oracle plan failed")
    out = {
        "level": np.zeros(ns, np.int32),
        "seg_ptr": np.zeros(ns + 1, np.int64),
        "seg_owner": np.zeros(max(nseg.value, 1), np.int32),
        "seg_start": np.zeros(max(nseg.value, 1), np.int32),
        "seg_coloff": np.zeros(max(nseg.value, 1), np.int32),
        "rel_ptr": np.zeros(nseg.value + 1, np.int64),
        "relidx": np.zeros(max(nrel.value, 1), np.int32),
    }
    rc = lib.orc_plan(ns, _p(sym.super_ptr), _p(sym.sparent), _p(sym.rowptr), _p(sym.rows),
                      _p(out["level"]), _p(out["seg_ptr"]), _p(out["seg_owner"]),
                      _p(out["seg_start"]), _p(out["seg_coloff"]), _p(out["rel_ptr"]),
                      _p(out["relidx"]), ct.byref(nseg), ct.byref(nrel))
    if rc != 0:
        raise ValueError("oracle plan failed")
    for k in ("seg_owner", "seg_start", "seg_coloff"):
        out[k] = out[k][: nseg.value]
    out["relidx"] = out["relidx"][: nrel.value]
    return out


def _sfx(dtype) -> str:
    return "_z" if np.dtype(dtype).kind == "c" else "_d"


def _sym_args(sym: Sym):
    return (sym.nsuper, _p(sym.super_ptr), _p(sym.sparent), _p(sym.rowptr), _p(sym.rows))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed: {ERRORS.get(rc, rc)}")


def ldlt(problem, sym: Sym) -> Tuple[np.ndarray, np.ndarray]:
    """L (panel layout, unit diagonal block) and D of P A P^T = L D L^T
    (L D L^H for a Hermitian problem)."""
    lib = _load()
    dt = np.complex128 if problem.values.dtype.kind == "c" else np.float64
    herm = bool(getattr(problem, "hermitian", False))
    vals = np.ascontiguousarray(problem.values, dtype=dt)
    colptr = np.ascontiguousarray(problem.colptr, dtype=np.int64)
    rowind = np.ascontiguousarray(problem.rowind, dtype=np.int32)
    L = np.zeros(sym.nnz_panels, dtype=dt)
    D = np.zeros(sym.n, dtype=dt)
    rc = getattr(lib, "orc_ldlt" + ("_h" if herm else _sfx(dt)))(int(problem.n), _p(colptr), _p(rowind), _p(vals),
                                            *_sym_args(sym), _p(L), _p(D))
    _check(rc, "ldlt")
    return L, D


def selinv(sym: Sym, L: np.ndarray, D: np.ndarray, symmetrize: bool = True,
           hermitian: bool = False) -> np.ndarray:
    """Selected inverse on the pattern of L (Alg. 1), panel layout; with
    hermitian=True the conjugate-transpose form for A = A^H."""
    lib = _load()
    L = np.ascontiguousarray(L); D = np.ascontiguousarray(D, dtype=L.dtype)
    Z = np.zeros_like(L)
    if hermitian and L.dtype.kind != "c":
        raise ValueError("the Hermitian form takes complex values")
    rc = getattr(lib, "orc_selinv" + ("_h" if hermitian else _sfx(L.dtype)))(*_sym_args(sym), _p(L), _p(D), _p(Z),
                                                                            int(symmetrize))
    _check(rc, "selinv")
    return Z


def selinv_top(sym: Sym, L: np.ndarray, D: np.ndarray, kmin: int, Z: np.ndarray = None,
               symmetrize: bool = True) -> np.ndarray:
    """Alg. 1 for the supernodes K >= kmin only (root side of the tree)."""
    lib = _load()
    L = np.ascontiguousarray(L); D = np.ascontiguousarray(D, dtype=L.dtype)
    if Z is None:
        Z = np.zeros_like(L)
    rc = getattr(lib, "orc_selinv_top" + _sfx(L.dtype))(*_sym_args(sym), _p(L), _p(D), _p(Z),
                                                       int(symmetrize), int(kmin))
    _check(rc, "selinv_top")
    return Z


def selinv_levels(sym: Sym, L: np.ndarray, D: np.ndarray, nthreads: int, kmin: int = 0,
                  Z: np.ndarray = None, symmetrize: bool = True, hermitian: bool = False) -> np.ndarray:
    """Alg. 1 with the supernodes of one tree level on ``nthreads`` host
    threads at a time (root level first); supernodes K >= kmin.  Bit for bit
    the result of ``selinv`` / ``selinv_top``."""
    lib = _load()
    L = np.ascontiguousarray(L); D = np.ascontiguousarray(D, dtype=L.dtype)
    if Z is None:
        Z = np.zeros_like(L)
    if hermitian and L.dtype.kind != "c":
        raise ValueError("the Hermitian form takes complex values")
    fn = getattr(lib, "orc_selinv_levels" + ("_h" if hermitian else _sfx(L.dtype)))
    rc = fn(*_sym_args(sym), _p(L), _p(D), _p(Z), int(symmetrize), int(kmin), int(nthreads))
    _check(rc, "selinv_levels")
    return Z


def selinv_push(sym: Sym, L: np.ndarray, D: np.ndarray, symmetrize: bool = True) -> np.ndarray:
    """Selected inverse by the left-looking push form (Alg. 2), panel layout."""
    lib = _load()
    L = np.ascontiguousarray(L); D = np.ascontiguousarray(D, dtype=L.dtype)
    Z = np.zeros_like(L)
    rc = getattr(lib, "orc_selinv_push" + _sfx(L.dtype))(*_sym_args(sym), _p(L), _p(D), _p(Z),
                                                        int(symmetrize))
    _check(rc, "selinv_push")
    return Z


def solve(sym: Sym, L: np.ndarray, D: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x with L D L^T x = b (forward / back substitution with the panels)."""
    lib = _load()
    L = np.ascontiguousarray(L); D = np.ascontiguousarray(D, dtype=L.dtype)
    x = np.array(b, dtype=L.dtype, copy=True)
    rc = getattr(lib, "orc_solve" + _sfx(L.dtype))(*_sym_args(sym), _p(L), _p(D), _p(x))
    _check(rc, "solve")
    return x


def selected_column(sym: Sym, L: np.ndarray, D: np.ndarray, j: int) -> np.ndarray:
    """Column j of A^{-1} (all n entries) by one solve."""
    e = np.zeros(sym.n, dtype=L.dtype)
    e[j] = 1
    return solve(sym, L, D, e)


def selinv_adjoint(sym: Sym, L, D, Z, Zbar) -> Tuple[np.ndarray, np.ndarray]:
    """(Lbar, Dbar) from the cotangent Zbar of the stored lower entries of Z."""
    lib = _load()
    L = np.ascontiguousarray(L); D = np.ascontiguousarray(D, dtype=L.dtype)
    Z = np.ascontiguousarray(Z, dtype=L.dtype)
    Zb = np.array(Zbar, dtype=L.dtype, copy=True)
    Lb = np.zeros_like(L); Db = np.zeros_like(D)
    rc = getattr(lib, "orc_selinv_adjoint" + _sfx(L.dtype))(*_sym_args(sym), _p(L), _p(D), _p(Z),
                                                           _p(Zb), _p(Lb), _p(Db))
    _check(rc, "selinv_adjoint")
    return Lb, Db


def ldlt_adjoint(sym: Sym, L, D, Lbar, Dbar) -> np.ndarray:
    """Abar on the pattern of L (panel layout) from (Lbar, Dbar)."""
    lib = _load()
    L = np.ascontiguousarray(L); D = np.ascontiguousarray(D, dtype=L.dtype)
    Lb = np.ascontiguousarray(Lbar, dtype=L.dtype); Db = np.ascontiguousarray(Dbar, dtype=L.dtype)
    Ab = np.zeros_like(L)
    rc = getattr(lib, "orc_ldlt_adjoint" + _sfx(L.dtype))(*_sym_args(sym), _p(L), _p(D), _p(Lb),
                                                         _p(Db), _p(Ab))
    _check(rc, "ldlt_adjoint")
    return Ab


# ---------------------------------------------------------------------------
# layout helpers (format conversions only)
# ---------------------------------------------------------------------------

def panel_entries(sym: Sym) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(row, col, is_lower_stored) of every panel slot, in storage order.

    is_lower_stored marks the slots that carry a stored lower entry (row >=
    col); the strictly upper part of the diagonal blocks is False."""
    s, c = sym.sizes()
    rows_out, cols_out = [], []
    for K in range(sym.nsuper):
        R = sym.rows[sym.rowptr[K]:sym.rowptr[K + 1]]
        cols = np.arange(sym.super_ptr[K], sym.super_ptr[K + 1])
        rows_out.append(np.tile(R, cols.size))
        cols_out.append(np.repeat(cols, R.size))
    r = np.concatenate(rows_out) if rows_out else np.zeros(0, np.int64)
    cc = np.concatenate(cols_out) if cols_out else np.zeros(0, np.int64)
    return r.astype(np.int64), cc.astype(np.int64), r >= cc


def panels_to_dense(sym: Sym, Z: np.ndarray, hermitian: bool = False) -> np.ndarray:
    """Symmetric (Hermitian) dense matrix from the stored lower entries (small n)."""
    r, c, low = panel_entries(sym)
    out = np.zeros((sym.n, sym.n), dtype=Z.dtype)
    out[c[low], r[low]] = np.conj(Z[low]) if hermitian else Z[low]
    out[r[low], c[low]] = Z[low]
    return out


def dense_to_panels(sym: Sym, M: np.ndarray) -> np.ndarray:
    r, c, low = panel_entries(sym)
    out = np.zeros(r.size, dtype=M.dtype)
    out[low] = M[r[low], c[low]]
    return out


def lower_mask(sym: Sym) -> np.ndarray:
    return panel_entries(sym)[2]


def block_errors(sym: Sym, G: np.ndarray, O: np.ndarray) -> np.ndarray:
    """Relative Frobenius error per supernode panel (lower-stored slots)."""
    off = sym.panel_offsets()
    low = lower_mask(sym)
    d = np.where(low, G - O, 0)
    o = np.where(low, O, 0)
    num = np.sqrt(np.add.reduceat(np.abs(d) ** 2, off[:-1])) if sym.nsuper else np.zeros(0)
    den = np.sqrt(np.add.reduceat(np.abs(o) ** 2, off[:-1])) if sym.nsuper else np.zeros(0)
    return num / np.where(den == 0, 1, den)


# ---------------------------------------------------------------------------
# subset selection and the pole-expansion sum
# ---------------------------------------------------------------------------

def panel_position(sym: Sym, i: int, j: int) -> int:
    """Panel slot of entry (i, j) of A^{-1}: the stored lower entry
    (max(i, j), min(i, j)) in the panel of the supernode owning the column,
    at the row's place in that supernode's row list.  KeyError if the entry
    is not on the pattern of L + L^T."""
    i, j = max(int(i), int(j)), min(int(i), int(j))
    K = int(np.searchsorted(sym.super_ptr, j, side="right")) - 1
    R = sym.rows[sym.rowptr[K]:sym.rowptr[K + 1]]
    k = int(np.searchsorted(R, i))
    if k >= R.size or R[k] != i:
        raise KeyError((i, j))
    return int(sym.panel_offsets()[K] + (j - sym.super_ptr[K]) * R.size + k)


def needed_supernodes(sym: Sym, cols) -> np.ndarray:
    """Boolean mask of the supernodes Alg. 1 runs to produce entries in the
    given columns: a supernode reads only blocks of its ancestors, so the
    owners of the columns and every ancestor of an owner (walked up sparent)."""
    need = np.zeros(sym.nsuper, dtype=bool)
    for c in np.asarray(cols).ravel():
        K = int(np.searchsorted(sym.super_ptr, int(c), side="right")) - 1
        while K >= 0:
            need[K] = True
            K = int(sym.sparent[K])
    return need


def pole_sum(Zs, weights, pos) -> np.ndarray:
    """sum_l w_l Z_l[pos] (complex), terms added in the order given."""
    out = np.zeros(len(pos), dtype=np.complex128)
    for Z, w in zip(Zs, weights):
        out = out + complex(w) * np.asarray(Z)[np.asarray(pos)]
    return out


# ---------------------------------------------------------------------------
# nonsymmetric values (LU form)
# ---------------------------------------------------------------------------

def lu(problem, sym: Sym) -> Tuple[np.ndarray, np.ndarray]:
    """L (panels, unit diagonal block) and Ut (U transposed, same layout: the
    diagonal block holds U_KK^T, rows s.. hold U(K,C)^T) of P A P^T = L U for a
    problem with nonsymmetric values (``meta["upper"]``: the values a_ji on
    the positions of the lower CSC)."""
    lib = _load()
    dt = np.complex128 if problem.values.dtype.kind == "c" else np.float64
    lo = np.ascontiguousarray(problem.values, dtype=dt)
    up = np.ascontiguousarray(problem.meta["upper"], dtype=dt)
    colptr = np.ascontiguousarray(problem.colptr, dtype=np.int64)
    rowind = np.ascontiguousarray(problem.rowind, dtype=np.int32)
    L = np.zeros(sym.nnz_panels, dtype=dt)
    Ut = np.zeros(sym.nnz_panels, dtype=dt)
    rc = getattr(lib, "orc_lu" + _sfx(dt))(int(problem.n), _p(colptr), _p(rowind), _p(lo), _p(up),
                                          *_sym_args(sym), _p(L), _p(Ut))
    _check(rc, "lu")
    return L, Ut


def selinv_lu(sym: Sym, L: np.ndarray, Ut: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Alg. 1 in its LU form: (Zl, Zu) -- Zl holds the full diagonal blocks of
    A^{-1} and A^{-1}_{C,K}, Zu their transposes and A^{-1}(K,C)^T."""
    lib = _load()
    L = np.ascontiguousarray(L)
    Ut = np.ascontiguousarray(Ut, dtype=L.dtype)
    Zl, Zu = np.zeros_like(L), np.zeros_like(L)
    rc = getattr(lib, "orc_selinv_lu" + _sfx(L.dtype))(*_sym_args(sym), _p(L), _p(Ut), _p(Zl), _p(Zu))
    _check(rc, "selinv_lu")
    return Zl, Zu


def panels_to_dense_lu(sym: Sym, Zl: np.ndarray, Zu: np.ndarray) -> np.ndarray:
    """Dense matrix from the LU-form panels: (i, j), i >= j, from Zl; (j, i) from Zu."""
    r, c, low = panel_entries(sym)
    out = np.zeros((sym.n, sym.n), dtype=Zl.dtype)
    out[c[low], r[low]] = Zu[low]
    out[r[low], c[low]] = Zl[low]
    return out
