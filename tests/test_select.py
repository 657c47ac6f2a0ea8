"""Subset selection and the pole-expansion sum.

CPU: the oracle's helpers against what fixes them independently (the dense
matrix, closed forms, the elimination tree), and the library's host-side
selection (panel positions, the set of supernodes that run) against the
oracle.  GPU (marked): a restricted selected inversion returns the oracle's
values at the selected entries, skips exactly the supernodes outside the
selection's ancestor chains, and the pole sum matches the oracle's.
"""
import numpy as np
import pytest

import oracle
import synth

TOL = 1e-10


def plan_for(native, sym):
    return native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows)


def pattern_entries(sym, rng, k):
    """k random stored lower entries (i, j) of the pattern of L, plus their mirror images."""
    r, c, low = oracle.panel_entries(sym)
    idx = rng.choice(np.flatnonzero(low), size=k, replace=False)
    return r[idx], c[idx]


# ---------------------------------------------------------------------------
# oracle pins
# ---------------------------------------------------------------------------

def test_panel_position_agrees_with_the_dense_inverse():
    p = synth.random_sparse_spd(70, 0.06, 11, supernodes=synth.problems.RELAXED_128)
    sym = oracle.symbolic_for(p)
    L, D = oracle.ldlt(p, sym)
    Z = oracle.selinv(sym, L, D)
    Ainv = np.linalg.inv(p.dense())
    r, c, low = oracle.panel_entries(sym)
    for i, j in zip(r[low][::7], c[low][::7]):
        for a, b in ((i, j), (j, i)):
            assert abs(Z[oracle.panel_position(sym, a, b)] - Ainv[a, b]) <= 1e-10 * np.abs(Ainv).max()
    # an entry off the pattern of L + L^T
    full = np.zeros((sym.n, sym.n), bool)
    full[r[low], c[low]] = True
    off = np.argwhere(~(full | full.T))
    if off.size:
        with pytest.raises(KeyError):
            oracle.panel_position(sym, *off[0])


def test_needed_supernodes_is_the_ancestor_closure():
    p = synth.laplacian_3d(9, seed=12)
    sym = oracle.symbolic_for(p)
    rng = np.random.default_rng(0)
    cols = rng.choice(sym.n, size=5, replace=False)
    need = oracle.needed_supernodes(sym, cols)
    owner = np.searchsorted(sym.super_ptr, cols, side="right") - 1
    assert need[owner].all()
    # closed under parents, and every needed supernode lies above an owner
    par = sym.sparent
    for K in np.flatnonzero(need):
        if par[K] >= 0:
            assert need[par[K]]
    above = np.zeros(sym.nsuper, bool)
    for K in owner:
        while K >= 0:
            above[K] = True
            K = par[K]
    assert np.array_equal(above, need)
    # a root column needs only the root chain, every column needs everything above it
    assert oracle.needed_supernodes(sym, [sym.n - 1]).sum() == 1


def test_pole_sum_two_pole_identity():
    """1/((x-a)(x-b)) = (1/(x-a) - 1/(x-b)) / (a-b): the two-term pole sum of
    selected inverses equals the diagonal of (A - aI)^{-1} (A - bI)^{-1}."""
    p = synth.random_sparse_spd(60, 0.08, 13)
    sym = oracle.symbolic_for(p)
    a, b = complex(0.3, 0.05), complex(-0.7, 0.2)
    Zs = []
    for z in (a, b):
        q = p.with_values(synth.problems.shifted_values(p, z))
        L, D = oracle.ldlt(q, sym)
        Zs.append(oracle.selinv(sym, L, D))
    pos = [oracle.panel_position(sym, i, i) for i in range(sym.n)]
    got = oracle.pole_sum(Zs, [1 / (a - b), -1 / (a - b)], pos)
    A = p.dense().astype(complex)
    I = np.eye(p.n)
    want = np.diag(np.linalg.inv(A - a * I) @ np.linalg.inv(A - b * I))
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


def test_pole_sum_diagonal_matrix_closed_form():
    d = np.linspace(1.0, 3.0, 5)
    z = np.array([0.5 + 0.1j, 2.2 - 0.3j, -1.0 + 0.0j])
    w = np.array([1.0 + 0.5j, -0.25j, 2.0])
    Zs = [1.0 / (d - zl) for zl in z]
    got = oracle.pole_sum(Zs, w, np.arange(5))
    want = np.array([sum(wl / (di - zl) for wl, zl in zip(w, z)) for di in d])
    assert np.abs(got - want).max() <= 1e-14


# ---------------------------------------------------------------------------
# host-side selection of the library (no GPU)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("make", [lambda: synth.laplacian_3d(10, seed=4),
                                  lambda: synth.random_sparse_spd(200, 0.02, 2, supernodes=synth.problems.RELAXED_128),
                                  lambda: synth.dft_sheet(side=6, nbasis=4)])
def test_selection_positions_and_active_set(native, make):
    p = make()
    sym = oracle.symbolic_for(p)
    plan = plan_for(native, sym)
    assert native.selinv_plan_get(plan, "active").all()
    rng = np.random.default_rng(1)
    r, c = pattern_entries(sym, rng, 12)
    rows = np.concatenate([r, c[:4], np.arange(3)])        # some upper entries and diagonals
    cols = np.concatenate([c, r[:4], np.arange(3)])
    pos = native.selinv_plan_select(plan, rows, cols)
    want = [oracle.panel_position(sym, i, j) for i, j in zip(rows, cols)]
    assert np.array_equal(pos, want)
    assert np.array_equal(native.selinv_plan_selected(plan), want)
    need = oracle.needed_supernodes(sym, np.minimum(rows, cols))
    assert np.array_equal(native.selinv_plan_get(plan, "active").astype(bool), need)
    # reset
    native.selinv_plan_select(plan, [], [])
    assert native.selinv_plan_get(plan, "active").all()
    assert native.selinv_plan_selected(plan).size == 0


def test_selection_rejects_entries_off_the_pattern(native):
    p = synth.laplacian_3d(8, seed=3)
    sym = oracle.symbolic_for(p)
    plan = plan_for(native, sym)
    r, c, low = oracle.panel_entries(sym)
    full = np.zeros((sym.n, sym.n), bool)
    full[r[low], c[low]] = True
    off = np.argwhere(~(full | full.T))
    assert off.size
    before = native.selinv_plan_select(plan, [5], [5])
    with pytest.raises(native.SelinvError) as e:
        native.selinv_plan_select(plan, [off[0][0]], [off[0][1]])
    assert e.value.code == native.SELINV_ERR_BAD_PATTERN
    assert np.array_equal(native.selinv_plan_selected(plan), before)   # unchanged
    with pytest.raises(native.SelinvError) as e:
        native.selinv_plan_select(plan, [sym.n], [0])
    assert e.value.code == native.SELINV_ERR_INVALID_ARG


# ---------------------------------------------------------------------------
# GPU
# ---------------------------------------------------------------------------

GPU_CASES = [
    ("lap3d-12", lambda: synth.laplacian_3d(12, seed=44)),
    ("rand300-relaxed", lambda: synth.random_sparse_spd(300, 0.02, 2, supernodes=synth.problems.RELAXED_128)),
    ("dft-c128", lambda: synth.dft_sheet(side=8, nbasis=4)),
]


def run_numeric(native, plan, L, D, **opts):
    import torch
    o = native.selinv_default_opts()
    for k, v in opts.items():
        setattr(o, k, v)
    native.selinv_plan_set_opts(plan, o)
    dt = native.SELINV_C128 if L.dtype.kind == "c" else native.SELINV_F64
    Lt, Dt = torch.from_numpy(L).cuda(), torch.from_numpy(np.ascontiguousarray(D)).cuda()
    Zt = torch.full_like(Lt, float("nan"))
    native.selinv_numeric(plan, dt, Lt, Dt, Zt)
    torch.cuda.synchronize()
    return Zt, dt


@pytest.mark.gpu
@pytest.mark.parametrize("sched", [(1, 1), (1, 0), (2, 1), (0, 1)])
@pytest.mark.parametrize("name,make", GPU_CASES)
def test_selected_entries_match_oracle(native, cuda_device, name, make, sched):
    """The diagonal of the columns of one subtree plus a few off-diagonal
    entries: values equal the oracle's; supernodes outside the ancestor
    chains are not written; the gather returns the entries in order."""
    import torch
    p = make()
    sym = oracle.symbolic_for(p)
    L, D = oracle.ldlt(p, sym)
    Z = oracle.selinv(sym, L, D)
    plan = plan_for(native, sym)
    cols = np.arange(0, sym.super_ptr[min(3, sym.nsuper)])     # the first supernodes' columns
    rng = np.random.default_rng(5)
    r, c = pattern_entries(sym, rng, 6)
    rows = np.concatenate([cols, r])
    cols = np.concatenate([cols, c])
    pos = native.selinv_plan_select(plan, rows, cols)
    need = oracle.needed_supernodes(sym, np.minimum(rows, cols))
    assert not need.all()                     # something is skipped
    Zt, dt = run_numeric(native, plan, L, D, schedule=sched[0], fast_contraction=sched[1])
    assert native.selinv_status(plan) == 0
    out = torch.empty(len(pos), dtype=Zt.dtype, device="cuda")
    native.selinv_gather(plan, dt, Zt, out)
    got = out.cpu().numpy()
    scale = np.abs(Z).max()
    assert np.abs(got - Z[pos]).max() <= TOL * scale
    G = Zt.cpu().numpy()
    off = sym.panel_offsets()
    low = oracle.lower_mask(sym)
    for K in range(sym.nsuper):
        blk = slice(off[K], off[K + 1])
        if need[K]:
            assert np.isfinite(G[blk][low[blk]]).all()
        else:
            assert np.isnan(G[blk]).all()
    # the full inversion again on the same plan
    native.selinv_plan_select(plan, [], [])
    Zt2, _ = run_numeric(native, plan, L, D, schedule=sched[0], fast_contraction=sched[1])
    assert oracle.block_errors(sym, Zt2.cpu().numpy(), Z).max() <= TOL


@pytest.mark.gpu
def test_pole_sum_matches_oracle(native, cuda_device):
    """A batch of complex pole shifts of one pattern plus the real matrix,
    diagonal only: the device pole sum equals the oracle's."""
    import torch
    base = synth.laplacian_3d(10, seed=7)
    sym = oracle.symbolic_for(base)
    e, eta = synth.pole_shifts(npoles=5)
    probs = [base.with_values(synth.problems.shifted_values(base, complex(e[l], eta[l]))) for l in range(5)]
    probs.append(base)
    weights = np.array([0.3 - 0.2j, -1.1 + 0.05j, 0.7j, 2.0, -0.4 - 0.4j, 0.25])
    plan = plan_for(native, sym)
    diag = np.arange(sym.n)
    pos = native.selinv_plan_select(plan, diag, diag)
    Zs, Ls, Ds, Gs, dts = [], [], [], [], []
    for q in probs:
        L, D = oracle.ldlt(q, sym)
        Zs.append(oracle.selinv(sym, L, D))
        Ls.append(torch.from_numpy(L).cuda())
        Ds.append(torch.from_numpy(np.ascontiguousarray(D)).cuda())
        Gs.append(torch.full_like(Ls[-1], float("nan")))
        dts.append(native.SELINV_C128 if L.dtype.kind == "c" else native.SELINV_F64)
    native.selinv_numeric_batched([plan] * len(probs), dts, Ls, Ds, Gs)
    pos_t = torch.from_numpy(pos).cuda()
    out = torch.empty(len(pos), dtype=torch.complex128, device="cuda")
    native.selinv_pole_sum(dts, Gs, weights, pos_t, out)
    torch.cuda.synchronize()
    assert native.selinv_status(plan) == 0
    want = oracle.pole_sum(Zs, weights, pos)
    assert np.abs(out.cpu().numpy() - want).max() <= TOL * np.abs(want).max()


@pytest.mark.gpu
def test_adjoint_refuses_an_active_selection(native, cuda_device):
    import torch
    p = synth.laplacian_3d(6, seed=2)
    sym = oracle.symbolic_for(p)
    plan = plan_for(native, sym)
    native.selinv_plan_select(plan, [0], [0])
    x = torch.zeros(plan.nnz, dtype=torch.float64, device="cuda")
    d = torch.ones(sym.n, dtype=torch.float64, device="cuda")
    with pytest.raises(native.SelinvError) as e:
        native.selinv_adjoint(plan, native.SELINV_F64, x, d, x, x, x.clone(), d.clone())
    assert e.value.code == native.SELINV_ERR_UNSUPPORTED
