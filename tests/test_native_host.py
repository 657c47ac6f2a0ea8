"""Host-side checks of the native library (no GPU needed).

* the library loads and exports every entry point declared in include/selinv.h;
* its symbolic analysis equals the oracle's, bit for bit;
* its plan (levels, owner segments, relative indices) equals the oracle's
  index sets, bit for bit;
* malformed inputs are rejected with the documented error codes.
"""
import ctypes as ct
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROBLEMS = [
    lambda: synth.random_sparse_spd(60, 0.08, 1),
    lambda: synth.random_sparse_spd(200, 0.02, 2, supernodes=synth.problems.RELAXED_128),
    lambda: synth.random_sparse_spd(80, 0.1, 3, complex_values=True),
    lambda: synth.tridiagonal(100),
    lambda: synth.tridiagonal(127, nd=True),
    lambda: synth.laplacian_3d(10, seed=4),
    lambda: synth.dft_sheet(side=6, nbasis=4),
    lambda: synth.diffusion_3d(8),
    lambda: synth.make_config(1),
    lambda: synth.make_config(5),
]


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "selinv.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(selinv_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(native):
    names = declared_symbols()
    assert len(names) >= 20
    lib = ct.CDLL(native._LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name
    assert set(native.REQUIRED_SYMBOLS) <= set(names)


@pytest.mark.parametrize("make", PROBLEMS)
def test_analysis_matches_oracle_bit_exact(native, make):
    p = make()
    sn = p.supernodes
    kind = 1 if sn["kind"] == "relaxed" else 0
    a = native.selinv_analyse(p.n, p.colptr, p.rowind, kind, sn["cap"], sn["fill"])
    o = oracle.symbolic_for(p)
    assert np.array_equal(a["parent"], o.parent)
    assert np.array_equal(a["super_ptr"], o.super_ptr)
    assert np.array_equal(a["sparent"], o.sparent)
    assert np.array_equal(a["rowptr"], o.rowptr)
    assert np.array_equal(a["rows"], o.rows)
    assert a["nnz_true"] == o.nnz_true


@pytest.mark.parametrize("cfg", [2, 3])
def test_analysis_matches_oracle_on_full_workloads(native, cfg):
    p = synth.make_config(cfg)
    sn = p.supernodes
    a = native.selinv_analyse(p.n, p.colptr, p.rowind, 1 if sn["kind"] == "relaxed" else 0,
                              sn["cap"], sn["fill"])
    o = oracle.symbolic_for(p)
    for k in ("super_ptr", "sparent", "rowptr", "rows"):
        assert np.array_equal(a[k], getattr(o, k)), k


def test_release_cached_memory_without_device_buffers(native):
    """An empty reuse cache is emptied without touching the device."""
    native.selinv_release_cached_memory()
    native.selinv_release_cached_memory()


def test_rejects_unclosed_structure_on_the_threaded_path(native):
    """A row list that is not closed under the tree is rejected also when the
    relative indices are filled by several host threads (large plans)."""
    p = synth.laplacian_3d(26, seed=2)
    sym, (sp, par, rp, rows) = _sym_arrays(p)
    ns = sym.nsuper
    # relative indices + row-list positions above the library's single-thread threshold (2^18)
    assert oracle.plan(sym)["relidx"].size + rp[-1] > (1 << 18)
    col2s = np.repeat(np.arange(ns), np.diff(sp))
    for K in range(ns - 1, -1, -1):                # a supernode near the root: late in the fill
        s = sp[K + 1] - sp[K]
        C = rows[rp[K] + s:rp[K + 1]]
        if C.size < 2:
            continue
        J = col2s[C[0]]
        below = [x for x in C[1:] if x >= sp[J + 1]]
        if below:
            break
    RJ = rows[rp[J]:rp[J + 1]]
    drop = rp[J] + int(np.searchsorted(RJ, below[0]))
    rows2 = np.delete(rows, drop)
    rp2 = rp.copy()
    rp2[J + 1:] -= 1
    with pytest.raises(native.SelinvError) as e:
        native.selinv_symbolic(sym.n, ns, sp, par, rp2, rows2)
    assert e.value.code in (-3, -2)
    native.selinv_symbolic(sym.n, ns, sp, par, rp, rows)   # the intact structure still plans


def make_plan(native, sym):
    return native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows)


@pytest.mark.parametrize("make", PROBLEMS + [lambda: synth.make_config(2)])
def test_plan_matches_oracle_bit_exact(native, make):
    p = make()
    sym = oracle.symbolic_for(p)
    plan = make_plan(native, sym)
    ref = oracle.plan(sym)
    for k in ("level", "seg_ptr", "seg_owner", "seg_start", "seg_coloff", "rel_ptr", "relidx"):
        got = native.selinv_plan_get(plan, k)
        assert np.array_equal(got, ref[k]), k
    lp = native.selinv_plan_get(plan, "level_ptr")
    ll = native.selinv_plan_get(plan, "level_list")
    for l in range(lp.size - 1):
        ks = ll[lp[l]:lp[l + 1]]
        assert np.all(np.diff(ks) > 0) and np.all(ref["level"][ks] == l)
    assert np.array_equal(native.selinv_plan_get(plan, "panel_off"), sym.panel_offsets())
    assert plan.nnz == sym.nnz_panels
    for K in (0, sym.nsuper // 2, sym.nsuper - 1):
        assert native.selinv_plan_panel_offset(plan, K) == sym.panel_offsets()[K]


@pytest.mark.parametrize("make", PROBLEMS[:3] + [lambda: synth.laplacian_3d(26, seed=2)])
def test_gather_addresses_follow_the_definition(native, make):
    """The per-position gather bases: entry (C[p], C[q]), p >= q, of A^{-1}
    sits in the panel of the owner J of column C[q] (Sec. II-B), column
    C[q] - first column of J, at the row of C[p] in rows(J).  Checked from the
    row lists alone for every q and a spread of p (26^3 fills on several
    host threads)."""
    p = make()
    sym = oracle.symbolic_for(p)
    plan = make_plan(native, sym)
    cb = native.selinv_plan_get(plan, "colbase")
    rb = native.selinv_plan_get(plan, "relbase")
    rel = native.selinv_plan_get(plan, "relidx")
    sp, rp, rows = sym.super_ptr, sym.rowptr, sym.rows
    off = sym.panel_offsets()
    col2s = np.repeat(np.arange(sym.nsuper), np.diff(sp))
    assert cb.size == rp[-1] and rb.size == rp[-1]
    for K in range(sym.nsuper):
        s = sp[K + 1] - sp[K]
        C = rows[rp[K] + s:rp[K + 1]]
        assert not cb[rp[K]:rp[K] + s].any() and not rb[rp[K]:rp[K] + s].any()
        for q in range(C.size):
            J = col2s[C[q]]
            RJ = rows[rp[J]:rp[J + 1]]
            pos = rp[K] + s + q
            assert cb[pos] == off[J] + (C[q] - sp[J]) * RJ.size
            ps = np.unique(np.r_[q, C.size - 1, np.linspace(q, C.size - 1, 5).astype(int)])
            assert np.array_equal(RJ[rel[rb[pos] + ps]], C[ps])


def test_plan_stats_formula(native):
    p = synth.make_config(1)
    sym = oracle.symbolic_for(p)
    plan = make_plan(native, sym)
    s, c = sym.sizes()
    F = float((2 * c * c * s + 2 * c * s * s + c * s * s + s ** 3).sum())
    B = float((8 * (c * (c + 1) // 2 + 2 * (c + s) * s + s)).sum())
    f, b = native.selinv_plan_stats(plan, native.SELINV_F64)
    assert f == F and b == B
    f2, b2 = native.selinv_plan_stats(plan, native.SELINV_C128)
    assert f2 == 4 * F and b2 == 2 * B


def _sym_arrays(p):
    sym = oracle.symbolic_for(p)
    return sym, [sym.super_ptr.copy(), sym.sparent.copy(), sym.rowptr.copy(), sym.rows.copy()]


def test_rejects_malformed_plans(native):
    p = synth.laplacian_3d(5, seed=1)
    sym, (sp, par, rp, rows) = _sym_arrays(p)
    n, ns = sym.n, sym.nsuper

    def code(sp_, par_, rp_, rows_, n_=n, ns_=ns):
        try:
            native.selinv_symbolic(n_, ns_, sp_, par_, rp_, rows_)
            return 0
        except native.SelinvError as e:
            return e.code

    assert code(sp, par, rp, rows) == 0
    # parent not the owner of the first row below (breaks the tree)
    K = int(np.nonzero(par >= 0)[0][0])
    bad = par.copy(); bad[K] = K
    assert code(sp, bad, rp, rows) == -2
    bad = par.copy(); bad[ns - 1] = 0
    assert code(sp, bad, rp, rows) == -2
    # unsorted rows
    K = int(np.argmax(np.diff(rp) - np.diff(sp) >= 2))
    bad = rows.copy()
    s = sp[K + 1] - sp[K]
    a, b = rp[K] + s, rp[K] + s + 1
    bad[a], bad[b] = bad[b], bad[a]
    assert code(sp, par, rp, bad) == -3
    # structure not closed under the tree: remove from the row list of the
    # owner J of C_K[0] a row C_K[p] that lies below J's own columns
    col2s = np.repeat(np.arange(ns), np.diff(sp))
    found = False
    for K in range(ns):
        s = sp[K + 1] - sp[K]
        C = rows[rp[K] + s:rp[K + 1]]
        if C.size < 2:
            continue
        J = col2s[C[0]]
        below = [x for x in C[1:] if x >= sp[J + 1]]
        if not below:
            continue
        RJ = rows[rp[J]:rp[J + 1]]
        drop = rp[J] + int(np.searchsorted(RJ, below[0]))
        rows2 = np.delete(rows, drop)
        rp2 = rp.copy(); rp2[J + 1:] -= 1
        assert code(sp, par, rp2, rows2) in (-3, -2)
        found = True
        break
    assert found
    # super_ptr not increasing / not ending at n
    bad = sp.copy(); bad[-1] = n + 1
    assert code(bad, par, rp, rows) == -1
    # bad sizes
    assert code(sp, par, rp, rows, ns_=-1) == -1
    # one dense supernode of 129 columns: wider than the kernels' column tile
    m = 129
    rows_d = np.arange(m, dtype=np.int32)
    assert code(np.array([0, m], np.int32), np.array([-1], np.int32), np.array([0, m], np.int64), rows_d,
                n_=m, ns_=1) == native.SELINV_ERR_UNSUPPORTED
    assert code(np.array([0, 128], np.int32), np.array([-1], np.int32), np.array([0, 128], np.int64),
                rows_d[:128], n_=128, ns_=1) == 0


def test_analysis_rejects_bad_csc(native):
    p = synth.random_sparse_spd(30, 0.2, 9)
    ri = p.rowind.copy()
    c0 = int(np.argmax(np.diff(p.colptr) >= 2))
    ri[p.colptr[c0]] = -1 if c0 == 0 else c0 - 1         # row above the diagonal
    with pytest.raises(native.SelinvError) as e:
        native.selinv_analyse(p.n, p.colptr, ri, 0, 64, 0.0)
    assert e.value.code == -3
    with pytest.raises(native.SelinvError) as e:
        native.selinv_analyse(p.n, p.colptr, p.rowind, 0, 0, 0.0)
    assert e.value.code == -1


def test_status_without_device_work_is_ok(native):
    p = synth.tridiagonal(10)
    sym = oracle.symbolic_for(p)
    plan = make_plan(native, sym)
    assert native.selinv_status(plan) == 0


def test_binding_constants_match_header(native):
    import re
    from pathlib import Path
    hdr = (Path(__file__).resolve().parents[1] / "include" / "selinv.h").read_text()
    codes = dict(re.findall(r"#define (SELINV_(?:OK|ERR_\w+))\s+\(?(-?\d+)\)?", hdr))
    assert len(codes) == 11
    for name, val in codes.items():
        assert getattr(native, name) == int(val), name
    kinds = int(re.search(r"#define SELINV_PROFILE_KINDS (\d+)", hdr).group(1))
    assert len(native.PROFILE_KINDS) == kinds


def test_options_round_trip_and_validation(native):
    p = synth.laplacian_3d(5, seed=1)
    sym, (sp, par, rp, rows) = _sym_arrays(p)
    plan = native.selinv_symbolic(sym.n, sym.nsuper, sp, par, rp, rows)
    o = native.selinv_default_opts()
    assert (o.fast_contraction, o.split_target, o.split_min_steps, o.oz_min_s) == (1, 2, 16, 16)
    o.split_target, o.split_min_steps, o.oz_min_s, o.fast_contraction = 4, 32, 64, 2
    native.selinv_plan_set_opts(plan, o)
    g = native.selinv_plan_get_opts(plan)
    assert (g.fast_contraction, g.split_target, g.split_min_steps, g.oz_min_s) == (2, 4, 32, 64)
    # the debug bits (non-finite scan, timeout test, bounds-checked gathers) round trip
    for bits in (native.DEBUG_CHECK_FINITE, native.DEBUG_TIMEOUT_TEST, native.DEBUG_CHECK_GATHER, 7):
        b = native.selinv_default_opts()
        b.debug_checks = bits
        native.selinv_plan_set_opts(plan, b)
        assert native.selinv_plan_get_opts(plan).debug_checks == bits
    assert "outside the panel" in native.error_string(native.SELINV_ERR_BAD_INDEX)
    for field, bad in (("split_target", 0), ("split_target", 9), ("split_min_steps", 12),
                       ("split_min_steps", 0), ("oz_min_s", 0), ("fast_contraction", 3), ("schedule", 4),
                       ("spin_limit", 0), ("debug_checks", 8), ("debug_checks", -1)):
        b = native.selinv_default_opts()
        setattr(b, field, bad)
        with pytest.raises(native.SelinvError) as e:
            native.selinv_plan_set_opts(plan, b)
        assert e.value.code == native.SELINV_ERR_INVALID_ARG, field


def test_binding_refuses_undersized_buffers(native):
    """A panel or diagonal buffer smaller than the plan needs is refused
    before anything reaches the library (a complex type needs 16 bytes per
    element: a float64 buffer of nnz elements is half the size)."""
    import torch
    p = synth.laplacian_3d(6, seed=1)
    sym = oracle.symbolic_for(p)
    plan = native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows)
    real = torch.zeros(plan.nnz, dtype=torch.float64)
    d = torch.zeros(sym.n, dtype=torch.complex128)
    for dt in (native.SELINV_C128, native.SELINV_C128H):
        with pytest.raises(ValueError, match="need"):
            native.selinv_numeric(plan, dt, real, d, real)
    with pytest.raises(ValueError, match="need"):
        native.selinv_numeric(plan, native.SELINV_F64, real, real[:3], real)
    # the host-buffer call checks its host buffers too (no device needed to refuse)
    with pytest.raises(ValueError, match="need"):
        native.selinv_numeric_host(plan, native.SELINV_F64, real[:5], real, real, real, real, real)
