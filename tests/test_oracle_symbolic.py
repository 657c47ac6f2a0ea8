"""Pins for the oracle's symbolic part (CPU only).

Column structures and the elimination tree are checked against brute-force
boolean graph elimination (eliminate vertices in order; each elimination
makes a clique of the remaining neighbours), which is exact.  The supernode
partition is checked against the paper's definition (Sec. II-A: contiguous
columns, dense diagonal block, identical structure below) and against the
closure property that the recursion relies on.
"""
import numpy as np
import pytest

import oracle
import synth


def brute_force_structs(problem):
    n = problem.n
    adj = [set() for _ in range(n)]
    cols = np.repeat(np.arange(n), np.diff(problem.colptr))
    for i, j in zip(problem.rowind, cols):
        if i != j:
            adj[i].add(int(j)); adj[j].add(int(i))
    structs, parent = [], []
    for j in range(n):
        nb = sorted(i for i in adj[j] if i > j)
        structs.append([j] + nb)
        parent.append(nb[0] if nb else -1)
        for a in nb:
            for b in nb:
                if a != b:
                    adj[a].add(b)
    return structs, parent


SMALL = [
    lambda: synth.random_sparse_spd(40, 0.08, 1),
    lambda: synth.random_sparse_spd(70, 0.04, 2),
    lambda: synth.random_sparse_spd(50, 0.3, 3),
    lambda: synth.laplacian_2d(7),
    lambda: synth.laplacian_3d(4, seed=1),
    lambda: synth.tridiagonal(30),
    lambda: synth.tridiagonal(31, nd=True),
]


@pytest.mark.parametrize("make", SMALL)
def test_etree_and_structs_match_brute_force(make):
    p = make()
    structs, parent = brute_force_structs(p)
    sym = oracle.symbolic(p.n, p.colptr, p.rowind, "fundamental", 1000, 0.0)
    assert sym.parent.tolist() == parent
    for j in range(p.n):
        got = sym.cstruct[sym.cstruct_ptr[j]:sym.cstruct_ptr[j + 1]].tolist()
        assert got == structs[j], j
    assert sym.nnz_true == sum(len(s) for s in structs)


@pytest.mark.parametrize("make", SMALL)
@pytest.mark.parametrize("cap", [1, 3, 64])
def test_fundamental_supernodes_follow_definition(make, cap):
    p = make()
    structs, parent = brute_force_structs(p)
    sym = oracle.symbolic(p.n, p.colptr, p.rowind, "fundamental", cap, 0.0)
    sp = sym.super_ptr
    assert sp[0] == 0 and sp[-1] == p.n and np.all(np.diff(sp) >= 1)
    assert np.all(np.diff(sp) <= cap)
    nchild = np.bincount([x for x in parent if x >= 0], minlength=p.n)
    for K in range(sym.nsuper):
        f, l = sp[K], sp[K + 1] - 1
        rows = sym.rows[sym.rowptr[K]:sym.rowptr[K + 1]].tolist()
        # dense diagonal block + identical structure below: every member's
        # structure is its own tail of the row list
        for j in range(f, l + 1):
            assert structs[j] == rows[j - f:], (K, j)
        if K + 1 < sym.nsuper:
            g = sp[K + 1]
            # the boundary is forced by the cap, the tree, or the structure
            same = structs[l][1:] == structs[g]
            assert (l - f + 1 == cap) or parent[l] != g or nchild[g] != 1 or not same
        # supernodal parent = owner of the first row below
        C = rows[l - f + 1:]
        if C:
            owner = np.searchsorted(sp, C[0], side="right") - 1
            assert sym.sparent[K] == owner
        else:
            assert sym.sparent[K] == -1


@pytest.mark.parametrize("make", [lambda: synth.laplacian_3d(8, seed=3),
                                  lambda: synth.diffusion_3d(6),
                                  lambda: synth.random_sparse_spd(120, 0.03, 7)])
@pytest.mark.parametrize("cap,fill", [(128, 0.10), (16, 0.10), (128, 0.3)])
def test_relaxed_supernodes_bound_fill_and_stay_closed(make, cap, fill):
    p = make()
    structs, _ = brute_force_structs(p)
    sym = oracle.symbolic(p.n, p.colptr, p.rowind, "relaxed", cap, fill)
    fund = oracle.symbolic(p.n, p.colptr, p.rowind, "fundamental", cap, 0.0)
    sp = sym.super_ptr
    # every relaxed supernode is a union of consecutive fundamental ones
    assert set(sp.tolist()) <= set(fund.super_ptr.tolist())
    assert sym.nsuper <= fund.nsuper
    col2s = np.repeat(np.arange(sym.nsuper), np.diff(sp))
    for K in range(sym.nsuper):
        f, l = sp[K], sp[K + 1] - 1
        s = l - f + 1
        rows = sym.rows[sym.rowptr[K]:sym.rowptr[K + 1]]
        assert rows[:s].tolist() == list(range(f, l + 1))
        assert np.all(np.diff(rows) > 0)
        c = rows.size - s
        stored = s * (s + 1) // 2 + s * c
        true = sum(len(structs[j]) for j in range(f, l + 1))
        for j in range(f, l + 1):  # stored pattern covers the true structure
            assert set(structs[j]) <= set(rows.tolist())
        merged = not np.isin(f, fund.super_ptr) or np.sum((fund.super_ptr >= f) & (fund.super_ptr <= l)) > 1
        if merged:
            assert stored - true <= fill * stored + 1e-9
            assert s <= cap
        # closure: rows below C[q] in C lie in the row list of C[q]'s owner
        C = rows[s:]
        for q in range(C.size):
            J = col2s[C[q]]
            RJ = set(sym.rows[sym.rowptr[J]:sym.rowptr[J + 1]].tolist())
            assert set(C[q:].tolist()) <= RJ


@pytest.mark.parametrize("make", SMALL[:5] + [lambda: synth.make_config(1)])
def test_plan_indices_are_positions(make):
    p = make()
    sym = oracle.symbolic_for(p)
    pl = oracle.plan(sym)
    sp = sym.super_ptr
    col2s = np.repeat(np.arange(sym.nsuper), np.diff(sp))
    # level = number of proper ancestors, found by walking the parent chain
    for K in range(sym.nsuper):
        d, J = 0, sym.sparent[K]
        while J >= 0:
            d += 1; J = sym.sparent[J]
        assert pl["level"][K] == d
    for K in range(sym.nsuper):
        s = sp[K + 1] - sp[K]
        C = sym.rows[sym.rowptr[K] + s:sym.rowptr[K + 1]]
        segs = range(pl["seg_ptr"][K], pl["seg_ptr"][K + 1])
        covered = []
        for t in segs:
            J, st = pl["seg_owner"][t], pl["seg_start"][t]
            assert C[st] - sp[J] == pl["seg_coloff"][t]
            RJ = sym.rows[sym.rowptr[J]:sym.rowptr[J + 1]]
            rel = pl["relidx"][pl["rel_ptr"][t]:pl["rel_ptr"][t + 1]]
            assert rel.size == C.size - st
            assert np.array_equal(RJ[rel], C[st:])
            covered.append(st)
        # segments are the maximal runs of one owner
        owners = col2s[C] if C.size else np.zeros(0, int)
        starts = [0] + [q for q in range(1, C.size) if owners[q] != owners[q - 1]] if C.size else []
        assert covered == starts
