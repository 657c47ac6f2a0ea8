"""The push schedule (the left-looking form of Alg. 2 on the GPU): every
finished supernode pushes its outer- and inner-product updates into its
descendants.  Same result as the pull form (Alg. 1), held to the oracle's
tolerance for real, complex symmetric and Hermitian problems, alone,
batched and under a subset selection."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10

CASES = [
    ("rand300-relaxed", lambda: synth.random_sparse_spd(300, 0.02, 2, supernodes=synth.problems.RELAXED_128), False),
    ("lap3d-14", lambda: synth.laplacian_3d(14, seed=6), False),
    ("lap2d-63", lambda: synth.make_config(1), False),
    ("dft-8x8-c128", lambda: synth.dft_sheet(side=8, nbasis=16), False),
    ("maglap3d-9-herm", lambda: synth.magnetic_laplacian_3d(9, seed=4), True),
    ("tridiag", lambda: synth.tridiagonal(400), False),
]


def dtype_of(native, L, herm):
    if L.dtype.kind != "c":
        return native.SELINV_F64
    return native.SELINV_C128H if herm else native.SELINV_C128


@pytest.mark.parametrize("name,make,herm", CASES)
def test_push_matches_oracle(native, cuda_device, name, make, herm):
    import torch
    p = make()
    sym = oracle.symbolic_for(p)
    L, D = oracle.ldlt(p, sym)
    Z = oracle.selinv(sym, L, D, hermitian=herm)
    plan = native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows)
    o = native.selinv_default_opts()
    o.schedule = native.SELINV_SCHED_PUSH
    native.selinv_plan_set_opts(plan, o)
    dt = dtype_of(native, L, herm)
    Lt, Dt = torch.from_numpy(L).cuda(), torch.from_numpy(np.ascontiguousarray(D)).cuda()
    Zt = torch.full_like(Lt, float("nan"))
    for _ in range(2):   # the accumulation buffer is cleared by every call
        native.selinv_numeric(plan, dt, Lt, Dt, Zt)
    torch.cuda.synchronize()
    assert native.selinv_status(plan) == 0
    assert oracle.block_errors(sym, Zt.cpu().numpy(), Z).max() <= TOL
    if not herm and L.dtype.kind != "c":
        # the oracle's own left-looking form: the same values in another order
        assert oracle.block_errors(sym, Zt.cpu().numpy(), oracle.selinv_push(sym, L, D)).max() <= TOL


def test_push_batched_and_selected(native, cuda_device):
    import torch
    probs = [(synth.laplacian_3d(10, seed=7), False), (synth.magnetic_laplacian_3d(8, seed=1), True),
             (synth.random_sparse_spd(150, 0.05, 8, complex_values=True), False)]
    plans, dts, Ls, Ds, Zs, want, syms = [], [], [], [], [], [], []
    for q, herm in probs:
        sym = oracle.symbolic_for(q)
        L, D = oracle.ldlt(q, sym)
        want.append(oracle.selinv(sym, L, D, hermitian=herm))
        syms.append(sym)
        plans.append(native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows))
        dts.append(dtype_of(native, L, herm))
        Ls.append(torch.from_numpy(L).cuda())
        Ds.append(torch.from_numpy(np.ascontiguousarray(D)).cuda())
        Zs.append(torch.full_like(Ls[-1], float("nan")))
    o = native.selinv_default_opts()
    o.schedule = native.SELINV_SCHED_PUSH
    native.selinv_plan_set_opts(plans[0], o)
    native.selinv_numeric_batched(plans, dts, Ls, Ds, Zs)
    torch.cuda.synchronize()
    assert native.selinv_status(plans[0]) == 0
    for i in range(len(probs)):
        assert oracle.block_errors(syms[i], Zs[i].cpu().numpy(), want[i]).max() <= TOL, i
    # a selection on the first problem: only its ancestor chains push
    sym = syms[0]
    cols = np.arange(sym.super_ptr[2])
    pos = native.selinv_plan_select(plans[0], cols, cols)
    native.selinv_numeric(plans[0], dts[0], Ls[0], Ds[0], Zs[0])
    torch.cuda.synchronize()
    assert native.selinv_status(plans[0]) == 0
    got = Zs[0].cpu().numpy()[pos]
    assert np.abs(got - want[0][pos]).max() <= TOL * np.abs(want[0]).max()
