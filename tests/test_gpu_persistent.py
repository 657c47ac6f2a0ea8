"""The persistent schedule (one launch; CTAs claim supernodes from a ticket in
root-level-first order and wait on their parent's completion flag), its
bounded waits, and the input checks.

The persistent traversal runs the DFMA kernel of the level schedule item by
item (the level schedule gives supernodes of at most 8 columns and 64 rows a
warp each instead, another summation order), so with the DFMA path forced on
both sides the two schedules agree to rounding; every output is also held to
the oracle's tolerance, and the persistent schedule with and without a CUDA
graph agree bit for bit.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10

CASES = [
    ("rand300-relaxed", lambda: synth.random_sparse_spd(300, 0.02, 2, supernodes=synth.problems.RELAXED_128)),
    ("dense200-c128-relaxed", lambda: synth.random_sparse_spd(200, 1.0, 5, complex_values=True,
                                                              supernodes=synth.problems.RELAXED_128)),
    ("lap3d-14-relaxed", lambda: synth.laplacian_3d(14, seed=6)),
    ("tridiag", lambda: synth.tridiagonal(500)),
]


def run(native, plan, L, D, **opts):
    import torch
    o = native.selinv_default_opts()
    for k, v in opts.items():
        setattr(o, k, v)
    native.selinv_plan_set_opts(plan, o)
    dt = native.SELINV_C128 if L.dtype.kind == "c" else native.SELINV_F64
    Lt = torch.from_numpy(L).cuda()
    Dt = torch.from_numpy(np.ascontiguousarray(D)).cuda()
    Zt = torch.full_like(Lt, float("nan"))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        native.selinv_numeric(plan, dt, Lt, Dt, Zt, s)
    s.synchronize()
    return Zt.cpu().numpy(), native.selinv_status(plan)


def setup(native, p):
    sym = oracle.symbolic_for(p)
    L, D = oracle.ldlt(p, sym)
    Z = oracle.selinv(sym, L, D)
    plan = native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows)
    return sym, L, D, Z, plan


@pytest.mark.parametrize("name,make", CASES)
def test_persistent_matches_level_and_oracle(native, cuda_device, name, make):
    sym, L, D, Z, plan = setup(native, make())
    G_lvl, st0 = run(native, plan, L, D, schedule=native.SELINV_SCHED_LEVEL, fast_contraction=0)
    G_per, st1 = run(native, plan, L, D, schedule=native.SELINV_SCHED_PERSISTENT, fast_contraction=0)
    G_gr, st2 = run(native, plan, L, D, schedule=native.SELINV_SCHED_PERSISTENT, fast_contraction=0, use_graph=0)
    assert st0 == st1 == st2 == 0
    assert oracle.block_errors(sym, G_per, G_lvl).max() <= 1e-13
    assert np.array_equal(G_gr, G_per)
    assert oracle.block_errors(sym, G_per, Z).max() <= TOL
    # default options (tensor-core normalization where eligible), run twice on
    # the same buffers: flags and ticket are reset by every call
    G_a, st3 = run(native, plan, L, D, schedule=native.SELINV_SCHED_PERSISTENT)
    assert st3 == 0
    assert oracle.block_errors(sym, G_a, Z).max() <= TOL


def test_persistent_batched_mixed_types(native, cuda_device):
    import torch
    probs = [synth.laplacian_3d(10, seed=7), synth.random_sparse_spd(150, 0.05, 8, complex_values=True),
             synth.make_config(1)]
    runs = [setup(native, p) for p in probs]
    plans = [r[4] for r in runs]
    o = native.selinv_default_opts()
    o.schedule = native.SELINV_SCHED_PERSISTENT
    native.selinv_plan_set_opts(plans[0], o)
    dts, Ls, Ds, Zs = [], [], [], []
    for (sym, L, D, Z, plan) in runs:
        dts.append(native.SELINV_C128 if L.dtype.kind == "c" else native.SELINV_F64)
        Ls.append(torch.from_numpy(L).cuda())
        Ds.append(torch.from_numpy(np.ascontiguousarray(D)).cuda())
        Zs.append(torch.full_like(Ls[-1], float("nan")))
    s = torch.cuda.Stream()
    for _ in range(2):
        native.selinv_numeric_batched(plans, dts, Ls, Ds, Zs, s)
    s.synchronize()
    assert native.selinv_status(plans[0]) == 0
    for i, (sym, L, D, Z, plan) in enumerate(runs):
        assert oracle.block_errors(sym, Zs[i].cpu().numpy(), Z).max() <= TOL, i


def test_wait_that_runs_out_reports_timeout_and_context_survives(native, cuda_device):
    """Every wait targets a flag that nothing sets; each gives up after
    spin_limit polls, the status reads SELINV_ERR_TIMEOUT, and the next call on
    the same plan and context is correct."""
    sym, L, D, Z, plan = setup(native, synth.laplacian_3d(8, seed=9))
    _, st = run(native, plan, L, D, schedule=native.SELINV_SCHED_PERSISTENT, debug_checks=2, spin_limit=2000)
    assert st == native.SELINV_ERR_TIMEOUT
    assert native.selinv_status(plan) == 0          # reading the status cleared it
    G, st = run(native, plan, L, D, schedule=native.SELINV_SCHED_PERSISTENT)
    assert st == 0
    assert oracle.block_errors(sym, G, Z).max() <= TOL


def test_nonfinite_input_is_reported(native, cuda_device):
    sym, L, D, Z, plan = setup(native, synth.random_sparse_spd(60, 0.08, 1))
    L2 = L.copy()
    L2[len(L2) // 2] = np.nan
    _, st = run(native, plan, L2, D, debug_checks=1)
    assert st == native.SELINV_ERR_NONFINITE
    D2 = np.ascontiguousarray(D).copy()
    D2[-1] = np.inf
    _, st = run(native, plan, L, D2, debug_checks=1)
    assert st == native.SELINV_ERR_NONFINITE
    G, st = run(native, plan, L, D, debug_checks=1)
    assert st == 0
    assert oracle.block_errors(sym, G, Z).max() <= TOL
