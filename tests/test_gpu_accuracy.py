"""Stress of the FP64-exact tensor-core contraction's error bound.

The tensor-core kernels cut each operand into 7 base-256 digits on a grid
shared by a row of the gathered A^{-1}(C,C) (bounded by the largest whole
column of the ancestors it reads) or a column of Lhat, and drop the digit
pairs below the 2^-53 level of that grid.  The error of an entry is
therefore bounded relative to (row bound) x (column bound), like a DGEMM
under a max-norm bound: it is weakest where A^{-1} decays fast away from
the diagonal or spans many orders of magnitude within a row.  These inputs
do exactly that; every supernode block must still meet the 1e-10 relative
Frobenius gate against the oracle, with every supernode on the tensor cores
(oz_min_s 1) and both tensor engines (tcgen05 and mma.sync), and so must
the largest elementwise error of a block relative to its largest entry.
Entries far below their block's largest carry less relative accuracy than
a DFMA sum would give them: that is the price of the shared grid.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10

CASES = [
    ("lap3d-16-shift20", lambda: synth.laplacian_3d(16, seed=81, shift=20.0)),
    ("lap3d-16-shift200", lambda: synth.laplacian_3d(16, seed=82, shift=200.0)),
    ("diffusion-14-sigma2", lambda: synth.diffusion_3d(14, seed=83, sigma=2.0)),
    ("rand400-scaled6", lambda: synth.symmetric_scaling(
        synth.random_sparse_spd(400, 0.03, 84, supernodes=synth.problems.RELAXED_128), 6.0, 85)),
    ("lap3d-14-scaled6", lambda: synth.symmetric_scaling(synth.laplacian_3d(14, seed=86), 6.0, 87)),
]


def _run(native, sym, L, D, fast, ozm):
    import torch
    plan = native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows)
    o = native.selinv_default_opts()
    o.fast_contraction = fast
    o.oz_min_s = ozm
    o.split_min_steps = 8
    native.selinv_plan_set_opts(plan, o)
    Lt = torch.from_numpy(L).cuda()
    Dt = torch.from_numpy(np.ascontiguousarray(D)).cuda()
    Zt = torch.full_like(Lt, float("nan"))
    native.selinv_numeric(plan, native.SELINV_F64, Lt, Dt, Zt, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert native.selinv_status(plan) == 0
    return Zt.cpu().numpy()


@pytest.mark.parametrize("fast", [1, 2])
@pytest.mark.parametrize("name,make", CASES)
def test_tensor_core_error_bound_on_fast_decay_and_wide_range(native, cuda_device, name, make, fast):
    p = make()
    sym = oracle.symbolic_for(p)
    L, D = oracle.ldlt(p, sym)
    Z = oracle.selinv(sym, L, D)
    G = _run(native, sym, L, D, fast, 1)
    low = oracle.lower_mask(sym)
    assert np.all(np.isfinite(G[low]))
    err = oracle.block_errors(sym, G, Z)
    assert err.max() <= TOL, (name, fast, float(err.max()))
    # the scheme's error is bounded relative to the largest entries (a
    # max-norm bound): max |G - O| over a block against its largest entry
    off = sym.panel_offsets()
    worst = 0.0
    for K in range(sym.nsuper):
        o = Z[off[K]:off[K + 1]]
        g = G[off[K]:off[K + 1]]
        m = np.abs(o).max()
        if m > 0:
            worst = max(worst, float(np.abs(g - o).max() / m))
    assert worst <= TOL, (name, fast, worst)
