"""ctypes binding of libselinv.so (argument marshalling only).

Every function here has the name of the C entry point it calls
(include/selinv.h).  Device buffers are torch tensors on a CUDA device;
their data pointers are passed through unchanged.  There is no fallback: if
the native library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Dict, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libselinv.so")

SELINV_F64 = 0
SELINV_C128 = 1
SELINV_C128H = 2   # complex Hermitian (conjugate transposes)
SELINV_SCHED_PLAIN = 0
SELINV_SCHED_LEVEL = 1
SELINV_SCHED_PERSISTENT = 2
SELINV_SCHED_PUSH = 3

SELINV_OK = 0
SELINV_ERR_INVALID_ARG = -1
SELINV_ERR_BAD_ETREE = -2
SELINV_ERR_BAD_PATTERN = -3
SELINV_ERR_ZERO_PIVOT = -4
SELINV_ERR_NONFINITE = -5
SELINV_ERR_OOM = -6
SELINV_ERR_CUDA = -7
SELINV_ERR_TIMEOUT = -8
SELINV_ERR_UNSUPPORTED = -9
SELINV_ERR_BAD_INDEX = -10
DEBUG_CHECK_FINITE, DEBUG_TIMEOUT_TEST, DEBUG_CHECK_GATHER = 1, 2, 4   # selinv_opts.debug_checks bits

# kernel kinds reported by selinv_numeric_profile
PROFILE_KINDS = ("k_linv", "k_lhat", "k_selinv", "k_lhat_digits", "k_selinv_oz", "k_diag",
                 "k_linv_digits", "k_lhat_oz", "k_selinv_persist", "k_selinv_tc",
                 "k_tc_reduce", "k_diag_fin", "k_push_diag", "k_push", "k_dinv", "k_diag_tc",
                 "k_selinv_tiny")


class SelinvError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: selinv error {code} ({error_string(code)})")


class selinv_opts(ct.Structure):
    _fields_ = [("symmetrize", ct.c_int), ("schedule", ct.c_int), ("autotune", ct.c_int),
                ("debug_checks", ct.c_int), ("spin_limit", ct.c_longlong), ("use_graph", ct.c_int),
                ("fast_contraction", ct.c_int), ("split_target", ct.c_int), ("split_min_steps", ct.c_int),
                ("oz_min_s", ct.c_int)]


def _load() -> ct.CDLL:
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"native library {_LIB_PATH} is missing: build it with "
                          "paper_1604_02528_gb300/build.py (no fallback path exists)")
    lib = ct.CDLL(_LIB_PATH)
    P, I32, I64, I = ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_int
    sig = {
        "selinv_default_opts": (None, [P]),
        "selinv_analyse": (I, [I32, P, P, I, I32, ct.c_double, P]),
        "selinv_analysis_get": (I64, [P, I, P]),
        "selinv_analysis_destroy": (None, [P]),
        "selinv_symbolic": (I, [I32, I32, P, P, P, P, P, P]),
        "selinv_plan_destroy": (None, [P]),
        "selinv_plan_nnz": (I64, [P]),
        "selinv_plan_panel_offset": (I64, [P, I32]),
        "selinv_plan_stats": (I, [P, I, P, P]),
        "selinv_plan_get": (I64, [P, I, P]),
        "selinv_plan_set_opts": (I, [P, P]),
        "selinv_plan_get_opts": (I, [P, P]),
        "selinv_numeric": (I, [P, I, P, P, P, P]),
        "selinv_numeric_host": (I, [P, I, P, P, P, P, P, P, P]),
        "selinv_numeric_batched": (I, [I, P, P, P, P, P, P]),
        "selinv_numeric_profile": (I, [P, I, P, P, P, P, P, P]),
        "selinv_plan_set_matrix": (I, [P, I32, P, P]),
        "selinv_factor": (I, [P, I, P, P, P, P]),
        "selinv_adjoint": (I, [P, I, P, P, P, P, P, P, P]),
        "selinv_factor_adjoint": (I, [P, I, P, P, P, P, P, P]),
        "selinv_status": (I, [P]),
        "selinv_error_string": (ct.c_char_p, [I]),
        "selinv_launch_count": (I64, []),
        "selinv_release_cached_memory": (I, []),
        "selinv_dinv_noalloc": (I, [I32, P, I64, P, P, I64, P]),
        "selinv_plan_select": (I, [P, I64, P, P, P]),
        "selinv_numeric_lu": (I, [P, I, P, P, P, P, P]),
        "selinv_plan_selected": (I64, [P, P]),
        "selinv_gather": (I, [P, I, P, P, P]),
        "selinv_pole_sum": (I, [I, P, P, P, I64, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


LIB = _load()

# the C-ABI symbols this binding requires (all declared in include/selinv.h)
REQUIRED_SYMBOLS = ("selinv_default_opts", "selinv_analyse", "selinv_analysis_get",
                    "selinv_analysis_destroy", "selinv_symbolic", "selinv_plan_destroy",
                    "selinv_plan_nnz", "selinv_plan_panel_offset", "selinv_plan_stats",
                    "selinv_plan_get", "selinv_plan_set_opts", "selinv_plan_get_opts", "selinv_numeric",
                    "selinv_numeric_host",
                    "selinv_numeric_batched", "selinv_numeric_profile", "selinv_plan_set_matrix", "selinv_factor",
                    "selinv_adjoint", "selinv_factor_adjoint", "selinv_status",
                    "selinv_error_string", "selinv_launch_count", "selinv_dinv_noalloc",
                    "selinv_plan_select", "selinv_plan_selected", "selinv_gather", "selinv_pole_sum",
                    "selinv_numeric_lu", "selinv_release_cached_memory")


def error_string(code: int) -> str:
    return LIB.selinv_error_string(int(code)).decode()


selinv_error_string = error_string


def _check(rc: int, what: str):
    if rc != 0:
        raise SelinvError(rc, what)


def _np(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ct.c_void_p)


def _dptr(t) -> ct.c_void_p:
    """Device pointer of a torch CUDA tensor (contiguous)."""
    if t is None:
        return ct.c_void_p(0)
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ct.c_void_p(t.data_ptr())


def _stream(stream) -> ct.c_void_p:
    if stream is None:
        import torch
        return ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ct.c_void_p(stream)
    return ct.c_void_p(stream.cuda_stream)


def selinv_default_opts() -> selinv_opts:
    o = selinv_opts()
    LIB.selinv_default_opts(ct.byref(o))
    return o


def selinv_analyse(n: int, colptr, rowind, kind: int = 0, cap: int = 64,
                   fill: float = 0.0) -> Dict[str, np.ndarray]:
    """Symbolic analysis of a lower CSC pattern -> etree and supernodes."""
    colptr = _np(colptr, np.int64)
    rowind = _np(rowind, np.int32)
    h = ct.c_void_p()
    _check(LIB.selinv_analyse(int(n), _ptr(colptr), _ptr(rowind), int(kind), int(cap),
                              float(fill), ct.byref(h)), "selinv_analyse")
    try:
        out = {}
        for name, field, dt in (("parent", 0, np.int32), ("super_ptr", 3, np.int32),
                                ("sparent", 4, np.int32), ("rowptr", 5, np.int64),
                                ("rows", 6, np.int32)):
            cnt = LIB.selinv_analysis_get(h, field, None)
            arr = np.zeros(max(cnt, 0), dtype=dt)
            if cnt > 0:
                LIB.selinv_analysis_get(h, field, _ptr(arr))
            out[name] = arr
        out["nsuper"] = int(LIB.selinv_analysis_get(h, 7, None))
        out["nnz_true"] = int(LIB.selinv_analysis_get(h, 8, None))
    finally:
        LIB.selinv_analysis_destroy(h)
    return out


class Plan:
    """Owner of a selinv_plan handle (destroyed with the object)."""

    def __init__(self, handle: ct.c_void_p, n: int, nsuper: int):
        self.handle = handle
        self.n = n
        self.nsuper = nsuper

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            LIB.selinv_plan_destroy(h)
            self.handle = None

    @property
    def nnz(self) -> int:
        return int(LIB.selinv_plan_nnz(self.handle))


def selinv_symbolic(n: int, nsuper: int, super_ptr, sparent, rowptr, rowind,
                    opts: Optional[selinv_opts] = None) -> Plan:
    sp = _np(super_ptr, np.int32)
    par = _np(sparent, np.int32)
    rp = _np(rowptr, np.int64)
    ri = _np(rowind, np.int32)
    h = ct.c_void_p()
    _check(LIB.selinv_symbolic(int(n), int(nsuper), _ptr(sp), _ptr(par), _ptr(rp), _ptr(ri),
                               ct.byref(opts) if opts is not None else None, ct.byref(h)),
           "selinv_symbolic")
    return Plan(h, int(n), int(nsuper))


def selinv_plan_destroy(plan: Plan):
    plan.__del__()


def selinv_plan_nnz(plan: Plan) -> int:
    return int(LIB.selinv_plan_nnz(plan.handle))


def selinv_plan_panel_offset(plan: Plan, K: int) -> int:
    return int(LIB.selinv_plan_panel_offset(plan.handle, int(K)))


def selinv_plan_stats(plan: Plan, dtype: int) -> Tuple[float, float]:
    f, b = ct.c_double(), ct.c_double()
    _check(LIB.selinv_plan_stats(plan.handle, int(dtype), ct.byref(f), ct.byref(b)), "selinv_plan_stats")
    return f.value, b.value


_PLAN_FIELDS = {"level": (0, np.int32), "seg_ptr": (1, np.int64), "seg_owner": (2, np.int32),
                "seg_start": (3, np.int32), "seg_coloff": (4, np.int32), "rel_ptr": (5, np.int64),
                "relidx": (6, np.int32), "level_ptr": (7, np.int64), "level_list": (8, np.int32),
                "panel_off": (9, np.int64), "active": (10, np.int32), "colbase": (11, np.int64),
                "relbase": (12, np.int64)}


def selinv_plan_get(plan: Plan, name: str) -> np.ndarray:
    field, dt = _PLAN_FIELDS[name]
    cnt = LIB.selinv_plan_get(plan.handle, field, None)
    if cnt < 0:
        raise SelinvError(int(cnt), "selinv_plan_get")
    arr = np.zeros(cnt, dtype=dt)
    if cnt > 0:
        LIB.selinv_plan_get(plan.handle, field, _ptr(arr))
    return arr


def selinv_plan_set_opts(plan: Plan, opts: selinv_opts):
    _check(LIB.selinv_plan_set_opts(plan.handle, ct.byref(opts)), "selinv_plan_set_opts")


def selinv_plan_get_opts(plan: Plan) -> selinv_opts:
    o = selinv_opts()
    _check(LIB.selinv_plan_get_opts(plan.handle, ct.byref(o)), "selinv_plan_get_opts")
    return o


def _need(t, elems: int, dtype: int, what: str):
    """The library writes and reads whole panel / diagonal arrays: a smaller
    buffer would be accessed out of bounds, so refuse it here."""
    if t is None:
        return
    es = 8 if int(dtype) == SELINV_F64 else 16
    if t.numel() * t.element_size() < elems * es:
        raise ValueError(f"{what}: {t.numel() * t.element_size()} bytes, need {elems * es} "
                         f"({elems} elements of {es} bytes)")


def _need_panels(plan: Plan, dtype: int, panels=(), diags=()):
    nnz = plan.nnz
    for name, t in panels:
        _need(t, nnz, dtype, name)
    for name, t in diags:
        _need(t, plan.n, dtype, name)


def selinv_numeric(plan: Plan, dtype: int, L, D, Ainv, stream=None):
    _need_panels(plan, dtype, [("L", L), ("Ainv", Ainv)], [("D", D)])
    _check(LIB.selinv_numeric(plan.handle, int(dtype), _dptr(L), _dptr(D), _dptr(Ainv),
                              _stream(stream)), "selinv_numeric")


def _hptr(t, n_bytes: int, what: str) -> ct.c_void_p:
    """Host pointer of a contiguous CPU tensor of at least n_bytes."""
    if t.is_cuda:
        raise ValueError(f"{what}: expected a CPU tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what}: expected a contiguous tensor")
    if t.numel() * t.element_size() < n_bytes:
        raise ValueError(f"{what}: {t.numel() * t.element_size()} bytes, need {n_bytes}")
    return ct.c_void_p(t.data_ptr())


def selinv_numeric_host(plan: Plan, dtype: int, L_host, D_host, Ainv_host, L_dev, D_dev, Ainv_dev,
                        stream=None):
    """Host L, D in and A^{-1} out (CPU tensors, pinned for the copies to
    overlap), through the caller's device staging buffers."""
    es = 8 if int(dtype) == SELINV_F64 else 16
    _need_panels(plan, dtype, [("L_dev", L_dev), ("Ainv_dev", Ainv_dev)], [("D_dev", D_dev)])
    _check(LIB.selinv_numeric_host(plan.handle, int(dtype), _hptr(L_host, plan.nnz * es, "L_host"),
                                   _hptr(D_host, plan.n * es, "D_host"),
                                   _hptr(Ainv_host, plan.nnz * es, "Ainv_host"), _dptr(L_dev), _dptr(D_dev),
                                   _dptr(Ainv_dev), _stream(stream)), "selinv_numeric_host")


def selinv_numeric_lu(plan: Plan, dtype: int, L, Ut, Zl, Zu, stream=None):
    """The LU form: L and U^T panels in, the lower and the transposed upper
    panels of A^{-1} out."""
    _need_panels(plan, dtype, [("L", L), ("Ut", Ut), ("Zl", Zl), ("Zu", Zu)])
    _check(LIB.selinv_numeric_lu(plan.handle, int(dtype), _dptr(L), _dptr(Ut), _dptr(Zl), _dptr(Zu),
                                 _stream(stream)), "selinv_numeric_lu")


def selinv_numeric_profile(plan: Plan, dtype: int, L, D, Ainv, stream=None):
    """Per-kernel-kind device time (ms) and launch counts of one call, indexed
    by PROFILE_KINDS."""
    _need_panels(plan, dtype, [("L", L), ("Ainv", Ainv)], [("D", D)])
    ms = (ct.c_double * len(PROFILE_KINDS))()
    cnt = (ct.c_int64 * len(PROFILE_KINDS))()
    _check(LIB.selinv_numeric_profile(plan.handle, int(dtype), _dptr(L), _dptr(D), _dptr(Ainv),
                                      _stream(stream), ms, cnt), "selinv_numeric_profile")
    return list(ms), list(cnt)


def selinv_numeric_batched(plans: Sequence[Plan], dtypes: Sequence[int], Ls, Ds, Zs, stream=None):
    n = len(plans)
    for p, d, L, D, Z in zip(plans, dtypes, Ls, Ds, Zs):
        _need_panels(p, d, [("L", L), ("Ainv", Z)], [("D", D)])
    arr = lambda xs, T: (T * n)(*xs)
    _check(LIB.selinv_numeric_batched(
        n, arr([p.handle for p in plans], ct.c_void_p), arr([int(d) for d in dtypes], ct.c_int),
        arr([_dptr(t) for t in Ls], ct.c_void_p), arr([_dptr(t) for t in Ds], ct.c_void_p),
        arr([_dptr(t) for t in Zs], ct.c_void_p), _stream(stream)), "selinv_numeric_batched")


def selinv_plan_select(plan: Plan, rows, cols) -> np.ndarray:
    """Restricts the plan to the entries (rows[e], cols[e]); returns their
    panel positions.  Empty arrays restore the full inversion."""
    r = _np(rows, np.int32)
    c = _np(cols, np.int32)
    if r.size != c.size:
        raise ValueError("rows and cols differ in length")
    pos = np.zeros(max(r.size, 1), dtype=np.int64)
    _check(LIB.selinv_plan_select(plan.handle, int(r.size), _ptr(r), _ptr(c), _ptr(pos)), "selinv_plan_select")
    return pos[:r.size]


def selinv_plan_selected(plan: Plan) -> np.ndarray:
    n = LIB.selinv_plan_selected(plan.handle, None)
    pos = np.zeros(max(n, 1), dtype=np.int64)
    LIB.selinv_plan_selected(plan.handle, _ptr(pos))
    return pos[:n]


def selinv_gather(plan: Plan, dtype: int, Ainv, out, stream=None):
    _need_panels(plan, dtype, [("Ainv", Ainv)])
    _need(out, int(LIB.selinv_plan_selected(plan.handle, None)), dtype, "out")
    _check(LIB.selinv_gather(plan.handle, int(dtype), _dptr(Ainv), _dptr(out), _stream(stream)), "selinv_gather")


def selinv_pole_sum(dtypes: Sequence[int], Ainvs, weights, pos, out, stream=None):
    """out[e] = sum_l weights[l] * Ainvs[l][pos[e]] (complex128 out, device pos)."""
    n = len(Ainvs)
    if len(dtypes) != n or len(weights) != n:
        raise ValueError("one dtype and one weight per term")
    _need(out, int(pos.numel()), SELINV_C128, "out")
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.complex128)).view(np.float64)
    arr = lambda xs, T: (T * n)(*xs)
    _check(LIB.selinv_pole_sum(n, arr([int(d) for d in dtypes], ct.c_int), arr([_dptr(t) for t in Ainvs], ct.c_void_p),
                               _ptr(w), int(pos.numel()), _dptr(pos), _dptr(out), _stream(stream)), "selinv_pole_sum")


def selinv_plan_set_matrix(plan: Plan, n: int, colptr, rowind):
    cp = _np(colptr, np.int64)
    ri = _np(rowind, np.int32)
    _check(LIB.selinv_plan_set_matrix(plan.handle, int(n), _ptr(cp), _ptr(ri)), "selinv_plan_set_matrix")


def selinv_factor(plan: Plan, dtype: int, A_vals, L, D, stream=None):
    _need_panels(plan, dtype, [("L", L)], [("D", D)])
    _check(LIB.selinv_factor(plan.handle, int(dtype), _dptr(A_vals), _dptr(L), _dptr(D),
                             _stream(stream)), "selinv_factor")


def selinv_adjoint(plan: Plan, dtype: int, L, D, Ainv, Ainv_bar, L_bar, D_bar, stream=None):
    _need_panels(plan, dtype, [("L", L), ("Ainv", Ainv), ("Ainv_bar", Ainv_bar), ("L_bar", L_bar)],
                 [("D", D), ("D_bar", D_bar)])
    _check(LIB.selinv_adjoint(plan.handle, int(dtype), _dptr(L), _dptr(D), _dptr(Ainv),
                              _dptr(Ainv_bar), _dptr(L_bar), _dptr(D_bar), _stream(stream)),
           "selinv_adjoint")


def selinv_factor_adjoint(plan: Plan, dtype: int, L, D, L_bar, D_bar, A_bar_vals, stream=None):
    _need_panels(plan, dtype, [("L", L), ("L_bar", L_bar)], [("D", D), ("D_bar", D_bar)])
    _check(LIB.selinv_factor_adjoint(plan.handle, int(dtype), _dptr(L), _dptr(D), _dptr(L_bar),
                                     _dptr(D_bar), _dptr(A_bar_vals), _stream(stream)),
           "selinv_factor_adjoint")


def selinv_dinv_noalloc(s: int, Lkk, ld: int, D, Dinv, ldo: int, stream=None):
    """Dinv = L^{-T} D^{-1} L^{-1} of one block with no allocation (scratch in a
    static device array; s <= 128)."""
    _check(LIB.selinv_dinv_noalloc(int(s), _dptr(Lkk), int(ld), _dptr(D), _dptr(Dinv), int(ldo),
                                   _stream(stream)), "selinv_dinv_noalloc")


def selinv_status(plan: Plan) -> int:
    return int(LIB.selinv_status(plan.handle))


def selinv_launch_count() -> int:
    return int(LIB.selinv_launch_count())


def selinv_release_cached_memory():
    """Frees the device buffers that destroyed plans left in the library's
    reuse cache."""
    _check(LIB.selinv_release_cached_memory(), "selinv_release_cached_memory")
