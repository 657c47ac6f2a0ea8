"""The Hermitian variant (Sec. II-C: conjugate transposes for A = A^H).

CPU: the oracle's Hermitian factorization and Alg. 1 against the dense
matrix and its inverse (numpy), and the reduction to the symmetric form on
real values.  GPU (marked): SELINV_C128H selected inversion and factorization
against the oracle, alone, batched with other element types, in every
schedule.
"""
import numpy as np
import pytest

import oracle
import synth

TOL = 1e-10

HERM_CASES = [
    ("hpd80", lambda: synth.random_sparse_hpd(80, 0.08, 3)),
    ("hpd200-relaxed", lambda: synth.random_sparse_hpd(200, 0.03, 4, supernodes=synth.problems.RELAXED_128)),
    ("hpd120-dense-relaxed", lambda: synth.random_sparse_hpd(120, 1.0, 5, supernodes=synth.problems.RELAXED_128)),
    ("maglap3d-8", lambda: synth.magnetic_laplacian_3d(8, seed=2)),
]


def pattern_mask(sym):
    r, c, low = oracle.panel_entries(sym)
    m = np.zeros((sym.n, sym.n), bool)
    m[r[low], c[low]] = True
    return m | m.T


# ---------------------------------------------------------------------------
# oracle pins
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,make", HERM_CASES)
def test_hermitian_oracle_matches_dense_inverse(name, make):
    p = make()
    A = p.dense()
    assert np.array_equal(A, A.conj().T)
    sym = oracle.symbolic_for(p)
    L, D = oracle.ldlt(p, sym)
    # A = L D L^H on the dense matrix
    Ld = oracle.panels_to_dense(sym, np.where(oracle.lower_mask(sym), L, 0))
    Ld = np.tril(Ld, -1) + np.eye(p.n)
    assert np.abs(Ld @ np.diag(D) @ Ld.conj().T - A).max() <= 1e-12 * np.abs(A).max()
    assert np.abs(D.imag).max() <= 1e-12 * np.abs(D).max()
    Z = oracle.selinv(sym, L, D, hermitian=True)
    Ainv = np.linalg.inv(A)
    G = oracle.panels_to_dense(sym, Z, hermitian=True)
    m = pattern_mask(sym)
    assert np.abs((G - Ainv)[m]).max() <= TOL * np.abs(Ainv).max()
    # the diagonal of A^{-1} of a Hermitian matrix is real after the symmetrization
    assert np.abs(np.diag(G).imag).max() == 0.0
    # the complex-symmetric form (plain transposes) is not the inverse here
    Zs = oracle.selinv(sym, L, D)
    assert np.abs((oracle.panels_to_dense(sym, Zs) - Ainv)[m]).max() > 1e-3 * np.abs(Ainv).max()


def test_hermitian_form_on_real_values_is_the_symmetric_one():
    p = synth.random_sparse_spd(90, 0.06, 8, supernodes=synth.problems.RELAXED_128)
    sym = oracle.symbolic_for(p)
    L, D = oracle.ldlt(p, sym)
    Zd = oracle.selinv(sym, L, D)
    Lc, Dc = L.astype(np.complex128), D.astype(np.complex128)
    Zh = oracle.selinv(sym, Lc, Dc, hermitian=True)
    Zz = oracle.selinv(sym, Lc, Dc)
    assert np.array_equal(Zh, Zz)
    assert np.array_equal(Zh.real, Zd) and not Zh.imag.any()


# ---------------------------------------------------------------------------
# GPU
# ---------------------------------------------------------------------------

def run(native, plan, L, D, dtype, **opts):
    import torch
    o = native.selinv_default_opts()
    for k, v in opts.items():
        setattr(o, k, v)
    native.selinv_plan_set_opts(plan, o)
    Lt, Dt = torch.from_numpy(L).cuda(), torch.from_numpy(np.ascontiguousarray(D)).cuda()
    Zt = torch.full_like(Lt, float("nan"))
    native.selinv_numeric(plan, dtype, Lt, Dt, Zt)
    torch.cuda.synchronize()
    return Zt.cpu().numpy(), native.selinv_status(plan)


@pytest.mark.gpu
@pytest.mark.parametrize("schedule", [1, 2, 0])
@pytest.mark.parametrize("name,make", HERM_CASES)
def test_gpu_hermitian_selinv_matches_oracle(native, cuda_device, name, make, schedule):
    p = make()
    sym = oracle.symbolic_for(p)
    L, D = oracle.ldlt(p, sym)
    Z = oracle.selinv(sym, L, D, hermitian=True)
    plan = native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows)
    G, st = run(native, plan, L, D, native.SELINV_C128H, schedule=schedule)
    assert st == 0
    assert oracle.block_errors(sym, G, Z).max() <= TOL
    # the same plan and buffers as a complex symmetric problem: the plain-transpose result
    Gs, st = run(native, plan, L, D, native.SELINV_C128, schedule=schedule)
    assert st == 0
    assert oracle.block_errors(sym, Gs, oracle.selinv(sym, L, D)).max() <= TOL


@pytest.mark.gpu
def test_gpu_hermitian_in_a_mixed_batch(native, cuda_device):
    import torch
    probs = [(synth.magnetic_laplacian_3d(9, seed=3), True),
             (synth.random_sparse_spd(150, 0.05, 8, complex_values=True), False),
             (synth.random_sparse_hpd(150, 0.05, 9, supernodes=synth.problems.RELAXED_128), True),
             (synth.laplacian_3d(8, seed=1), False)]
    plans, dts, Ls, Ds, Zs, want, syms = [], [], [], [], [], [], []
    for q, herm in probs:
        sym = oracle.symbolic_for(q)
        L, D = oracle.ldlt(q, sym)
        want.append(oracle.selinv(sym, L, D, hermitian=herm))
        syms.append(sym)
        plans.append(native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows))
        dts.append(native.SELINV_C128H if herm else (native.SELINV_C128 if L.dtype.kind == "c" else native.SELINV_F64))
        Ls.append(torch.from_numpy(L).cuda())
        Ds.append(torch.from_numpy(np.ascontiguousarray(D)).cuda())
        Zs.append(torch.full_like(Ls[-1], float("nan")))
    for sched in (1, 2):
        o = native.selinv_default_opts()
        o.schedule = sched
        native.selinv_plan_set_opts(plans[0], o)
        native.selinv_numeric_batched(plans, dts, Ls, Ds, Zs)
        torch.cuda.synchronize()
        assert native.selinv_status(plans[0]) == 0
        for i in range(len(probs)):
            assert oracle.block_errors(syms[i], Zs[i].cpu().numpy(), want[i]).max() <= TOL, (sched, i)


@pytest.mark.gpu
@pytest.mark.parametrize("name,make", HERM_CASES)
def test_gpu_hermitian_factor_and_end_to_end(native, cuda_device, name, make):
    """GPU L D L^H against the oracle's, then GPU factor -> GPU selected
    inversion against the dense inverse on the pattern."""
    import torch
    from paper_1604_02528_gb300.api import SelInvContext
    p = make()
    sym = oracle.symbolic_for(p)
    L0, D0 = oracle.ldlt(p, sym)
    ctx = SelInvContext.from_problem(p)
    assert ctx.hermitian
    L, D = ctx.factor(torch.from_numpy(p.values).cuda())
    Z = ctx.selinv(L, D)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    r, c, _ = oracle.panel_entries(sym)
    strict = r > c
    assert np.abs(D.cpu().numpy() - D0).max() <= 1e-12 * np.abs(D0).max()
    assert oracle.block_errors(sym, np.where(strict, L.cpu().numpy(), 0), np.where(strict, L0, 0)).max() <= TOL
    G = oracle.panels_to_dense(sym, Z.cpu().numpy(), hermitian=True)
    Ainv = np.linalg.inv(p.dense())
    m = pattern_mask(sym)
    assert np.abs((G - Ainv)[m]).max() <= TOL * np.abs(Ainv).max()


@pytest.mark.gpu
@pytest.mark.parametrize("name,make", HERM_CASES)
def test_gpu_hermitian_tensor_core_path(native, cuda_device, name, make):
    """Hermitian supernodes on tcgen05 (entries above the diagonal of
    A^{-1}_{C,C} conjugated in the gather, Lhat^H in the diagonal block),
    every supernode (oz_min_s 1), with and without k-splits: within 1e-10 of
    the oracle, the k-split bitwise irrelevant, and the diagonal blocks
    exactly Hermitian with a real diagonal."""
    p = make()
    sym = oracle.symbolic_for(p)
    L, D = oracle.ldlt(p, sym)
    Z = oracle.selinv(sym, L, D, hermitian=True)
    plan = native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows)
    outs = []
    for target, mins in ((1, 64), (8, 8)):
        G, st = run(native, plan, L, D, native.SELINV_C128H, fast_contraction=1, oz_min_s=1,
                    split_target=target, split_min_steps=mins)
        assert st == 0
        assert oracle.block_errors(sym, G, Z).max() <= TOL, (name, target)
        outs.append(G)
    assert np.array_equal(outs[0], outs[1])
    G = outs[0]
    off = sym.panel_offsets()
    s, c = sym.sizes()
    for K in range(0, sym.nsuper, max(1, sym.nsuper // 40)):
        blk = G[off[K]:off[K + 1]].reshape(s[K], s[K] + c[K]).T[: s[K], :]
        assert np.array_equal(blk, blk.conj().T)
        assert np.all(blk.diagonal().imag == 0)
