"""Nonsymmetric values on the symmetric pattern: the LU form of Alg. 1.

CPU: the oracle's LU (no pivoting) and its LU-form selected inversion
against numpy's dense matrix and inverse, and the reduction to the LDL^T
form for symmetric values.  GPU (marked): selinv_numeric_lu against the
oracle, real and complex, level and plain schedules.
"""
import numpy as np
import pytest

import oracle
import synth

TOL = 1e-10

CASES = [
    ("nonsym80", lambda: synth.random_sparse_nonsym(80, 0.08, 3)),
    ("nonsym200-relaxed", lambda: synth.random_sparse_nonsym(200, 0.03, 4, supernodes=synth.problems.RELAXED_128)),
    ("nonsym120-dense-relaxed", lambda: synth.random_sparse_nonsym(120, 1.0, 6, supernodes=synth.problems.RELAXED_128)),
    ("nonsym150-c128", lambda: synth.random_sparse_nonsym(150, 0.05, 5, complex_values=True,
                                                          supernodes=synth.problems.RELAXED_128)),
]


def pattern_mask(sym):
    r, c, low = oracle.panel_entries(sym)
    m = np.zeros((sym.n, sym.n), bool)
    m[r[low], c[low]] = True
    return m | m.T


@pytest.mark.parametrize("name,make", CASES)
def test_lu_oracle_matches_dense(name, make):
    p = make()
    A = p.dense()
    assert np.abs(A - A.T).max() > 0.1            # really nonsymmetric
    sym = oracle.symbolic_for(p)
    L, Ut = oracle.lu(p, sym)
    low = oracle.lower_mask(sym)
    Ld = np.tril(oracle.panels_to_dense_lu(sym, np.where(low, L, 0), np.zeros_like(L)), -1) + np.eye(p.n)
    Ud = np.triu(oracle.panels_to_dense_lu(sym, np.where(low, Ut, 0), np.zeros_like(Ut)).T)
    assert np.abs(Ld @ Ud - A).max() <= 1e-12 * np.abs(A).max()
    Zl, Zu = oracle.selinv_lu(sym, L, Ut)
    Ainv = np.linalg.inv(A)
    G = oracle.panels_to_dense_lu(sym, Zl, Zu)
    m = pattern_mask(sym)
    assert np.abs((G - Ainv)[m]).max() <= TOL * np.abs(Ainv).max()
    # Zu's diagonal blocks are the transposes of Zl's
    off = sym.panel_offsets()
    s, c = sym.sizes()
    for K in range(sym.nsuper):
        ld = s[K] + c[K]
        bl = Zl[off[K]:off[K + 1]].reshape(s[K], ld).T[:s[K]]
        bu = Zu[off[K]:off[K + 1]].reshape(s[K], ld).T[:s[K]]
        assert np.array_equal(bl, bu.T)


def test_lu_form_on_symmetric_values_is_the_ldlt_one():
    """For a symmetric matrix U = D L^T: the LU form returns the LDL^T form's
    selected inverse in both panel sets."""
    p = synth.random_sparse_spd(100, 0.06, 9, supernodes=synth.problems.RELAXED_128)
    q = p.with_values(p.values)
    q.meta["upper"] = p.values.copy()
    sym = oracle.symbolic_for(p)
    L, D = oracle.ldlt(p, sym)
    Z = oracle.selinv(sym, L, D)
    L2, Ut = oracle.lu(q, sym)
    Zl, Zu = oracle.selinv_lu(sym, L2, Ut)
    low = oracle.lower_mask(sym)
    assert np.abs(np.where(low, L2 - L, 0)).max() <= 1e-13
    assert oracle.block_errors(sym, Zl, Z).max() <= 1e-12
    assert oracle.block_errors(sym, Zu, Z).max() <= 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("schedule", [1, 0])
@pytest.mark.parametrize("name,make", CASES)
def test_gpu_lu_matches_oracle(native, cuda_device, name, make, schedule):
    import torch
    p = make()
    sym = oracle.symbolic_for(p)
    L, Ut = oracle.lu(p, sym)
    Zl0, Zu0 = oracle.selinv_lu(sym, L, Ut)
    plan = native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows)
    o = native.selinv_default_opts()
    o.schedule = schedule
    native.selinv_plan_set_opts(plan, o)
    dt = native.SELINV_C128 if L.dtype.kind == "c" else native.SELINV_F64
    Lt, Ut_t = torch.from_numpy(L).cuda(), torch.from_numpy(Ut).cuda()
    Zl = torch.full_like(Lt, float("nan"))
    Zu = torch.full_like(Lt, float("nan"))
    for _ in range(2):
        native.selinv_numeric_lu(plan, dt, Lt, Ut_t, Zl, Zu)
    torch.cuda.synchronize()
    assert native.selinv_status(plan) == 0
    low = oracle.lower_mask(sym)
    Zl_g, Zu_g = Zl.cpu().numpy(), Zu.cpu().numpy()
    assert oracle.block_errors(sym, Zl_g, Zl0).max() <= TOL
    assert oracle.block_errors(sym, np.where(low, Zu_g, 0), np.where(low, Zu0, 0)).max() <= TOL
