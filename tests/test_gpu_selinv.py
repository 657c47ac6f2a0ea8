"""GPU parity of the selected inversion against the CPU oracle.

The GPU path receives the oracle's own factors L, D (so the comparison
isolates the selected inversion) and its output is compared block by block:
relative Frobenius error of every supernode panel <= 1e-10.  Sizes span
several 64-row tiles, every width class (s up to 128) and ragged tails.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10

CASES = [
    ("rand60", lambda: synth.random_sparse_spd(60, 0.08, 1)),
    ("rand300-relaxed", lambda: synth.random_sparse_spd(300, 0.02, 2, supernodes=synth.problems.RELAXED_128)),
    ("rand80-c128", lambda: synth.random_sparse_spd(80, 0.1, 3, complex_values=True)),
    ("dense150", lambda: synth.random_sparse_spd(150, 1.0, 4)),                       # s = 64 chain
    ("dense200-c128-relaxed", lambda: synth.random_sparse_spd(200, 1.0, 5, complex_values=True,
                                                              supernodes=synth.problems.RELAXED_128)),
    ("tridiag", lambda: synth.tridiagonal(500)),
    ("lap2d-63", lambda: synth.make_config(1)),
    ("lap3d-14-relaxed", lambda: synth.laplacian_3d(14, seed=6)),
    ("dft-8x8", lambda: synth.dft_sheet(side=8, nbasis=16)),
    ("diffusion-10", lambda: synth.diffusion_3d(10)),
    ("single-column", lambda: synth.tridiagonal(1)),
]


def oracle_run(p):
    sym = oracle.symbolic_for(p)
    L, D = oracle.ldlt(p, sym)
    Z = oracle.selinv(sym, L, D)
    return sym, L, D, Z


def gpu_selinv(native, sym, L, D, schedule=1, use_graph=1, plan=None, repeat=1):
    import torch
    if plan is None:
        plan = native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows)
    o = native.selinv_default_opts()
    o.schedule = schedule
    o.use_graph = use_graph
    native.selinv_plan_set_opts(plan, o)
    dt = native.SELINV_C128 if L.dtype.kind == "c" else native.SELINV_F64
    Lt = torch.from_numpy(L).cuda()
    Dt = torch.from_numpy(np.ascontiguousarray(D)).cuda()
    Zt = torch.full_like(Lt, float("nan"))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(repeat):
            native.selinv_numeric(plan, dt, Lt, Dt, Zt, s)
    s.synchronize()
    assert native.selinv_status(plan) == 0
    return Zt.cpu().numpy(), plan


@pytest.mark.parametrize("name,make", CASES)
def test_selinv_matches_oracle(native, cuda_device, name, make):
    p = make()
    sym, L, D, Z = oracle_run(p)
    G, _ = gpu_selinv(native, sym, L, D)
    low = oracle.lower_mask(sym)
    assert np.all(np.isfinite(G[low]))
    err = oracle.block_errors(sym, G, Z)
    assert err.max() <= TOL, (name, err.max())
    # the full diagonal block is written, symmetric
    off = sym.panel_offsets()
    s, c = sym.sizes()
    for K in range(0, sym.nsuper, max(1, sym.nsuper // 50)):
        blk = G[off[K]:off[K + 1]].reshape(s[K], s[K] + c[K]).T[: s[K], :]
        assert np.array_equal(blk, blk.T)


@pytest.mark.parametrize("name,make", [CASES[1], CASES[4], CASES[7]])
def test_schedules_and_graphs_agree_bitwise(native, cuda_device, name, make):
    p = make()
    sym, L, D, Z = oracle_run(p)
    G_level, plan = gpu_selinv(native, sym, L, D, schedule=1, use_graph=1)
    G_plain, _ = gpu_selinv(native, sym, L, D, schedule=0, use_graph=0, plan=plan)
    G_nograph, _ = gpu_selinv(native, sym, L, D, schedule=1, use_graph=0, plan=plan)
    G_rep, _ = gpu_selinv(native, sym, L, D, schedule=1, use_graph=1, plan=plan, repeat=3)
    # plain runs every DFMA supernode as CTA tiles, level the tiniest as a warp each
    assert oracle.block_errors(sym, G_level, G_plain).max() <= 1e-13
    assert np.array_equal(G_level, G_nograph)
    assert np.array_equal(G_level, G_rep)
    assert oracle.block_errors(sym, G_level, Z).max() <= TOL


def test_batched_mixed_problems_match_oracle(native, cuda_device):
    import torch
    probs = [synth.laplacian_3d(12, seed=7), synth.random_sparse_spd(150, 0.05, 8, complex_values=True),
             synth.make_config(1)]
    runs = [oracle_run(p) for p in probs]
    plans, dts, Ls, Ds, Zs = [], [], [], [], []
    for (sym, L, D, Z) in runs:
        plans.append(native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows))
        dts.append(native.SELINV_C128 if L.dtype.kind == "c" else native.SELINV_F64)
        Ls.append(torch.from_numpy(L).cuda())
        Ds.append(torch.from_numpy(np.ascontiguousarray(D)).cuda())
        Zs.append(torch.full_like(Ls[-1], float("nan")))
    # the same plan twice in one batch (two pole shifts of one pattern)
    sym0, L0, D0, Z0 = runs[0]
    plans.append(plans[0]); dts.append(dts[0])
    Ls.append(Ls[0].clone()); Ds.append(Ds[0].clone()); Zs.append(torch.full_like(Ls[0], float("nan")))
    s = torch.cuda.Stream()
    native.selinv_numeric_batched(plans, dts, Ls, Ds, Zs, s)
    s.synchronize()
    assert native.selinv_status(plans[0]) == 0
    for i, (sym, L, D, Z) in enumerate(runs + [runs[0]]):
        G = Zs[i].cpu().numpy()
        assert oracle.block_errors(sym, G, Z).max() <= TOL, i


@pytest.mark.parametrize("name,make", [CASES[1], CASES[3], CASES[7], CASES[9]])
def test_tensor_core_and_dfma_paths_match_oracle(native, cuda_device, name, make):
    """The FP64-exact bf16 tensor-core contraction (tcgen05 and mma.sync) and
    the DFMA contraction all meet the tolerance; they differ only by rounding."""
    import torch
    p = make()
    sym, L, D, Z = oracle_run(p)
    plan = native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows)
    outs = []
    for fast, ozm in ((1, 16), (2, 16), (0, 16), (1, 1), (2, 1)):   # oz_min_s 1: every supernode on the tensor cores
        o = native.selinv_default_opts()
        o.fast_contraction = fast
        o.oz_min_s = ozm
        native.selinv_plan_set_opts(plan, o)
        Lt = torch.from_numpy(L).cuda(); Dt = torch.from_numpy(D).cuda()
        Zt = torch.full_like(Lt, float("nan"))
        native.selinv_numeric(plan, native.SELINV_F64, Lt, Dt, Zt, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert native.selinv_status(plan) == 0
        outs.append(Zt.cpu().numpy())
    for G in outs:
        assert oracle.block_errors(sym, G, Z).max() <= TOL
    for G in outs[:2] + outs[3:]:
        assert oracle.block_errors(sym, G, outs[2]).max() <= TOL


def test_tensor_core_result_is_independent_of_the_k_split(native, cuda_device):
    """The tcgen05 contraction's split-k partial sums are exact int64 words,
    added exactly by k_tc_reduce, and every k-range works on the same row and
    column exponent grids: the result is bitwise the same for any k-split
    (one CTA per output tile, or up to several k-ranges of >= 8 steps)."""
    import torch
    p = synth.laplacian_3d(26, seed=4)          # c up to 880 rows: up to 6 k-ranges of >= 8 steps
    sym = oracle.symbolic_for(p)
    L, D = oracle.ldlt(p, sym)
    plan = native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows)
    Lt, Dt = torch.from_numpy(L).cuda(), torch.from_numpy(D).cuda()
    outs = []
    for target, min_steps in ((1, 64), (2, 8), (8, 8), (4, 16)):
        o = native.selinv_default_opts()
        o.fast_contraction = 1
        o.split_target = target
        o.split_min_steps = min_steps
        native.selinv_plan_set_opts(plan, o)
        Zt = torch.full_like(Lt, float("nan"))
        native.selinv_numeric(plan, native.SELINV_F64, Lt, Dt, Zt, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert native.selinv_status(plan) == 0
        outs.append(Zt.cpu().numpy())
    for G in outs[1:]:
        assert np.array_equal(G, outs[0])
    assert oracle.block_errors(sym, outs[0], oracle.selinv(sym, L, D)).max() <= TOL


def test_replanning_reuses_cached_workspaces(native, cuda_device):
    """Plans destroyed and re-created (one pattern, then another) run on
    workspace buffers from the reuse cache, whose old contents must not leak
    into the result; the cache is then emptied."""
    import gc
    cases = [CASES[7], CASES[3], CASES[7]]
    for name, make in cases:
        p = make()
        sym, L, D, Z = oracle_run(p)
        for _ in range(2):
            G, plan = gpu_selinv(native, sym, L, D)
            assert oracle.block_errors(sym, G, Z).max() <= TOL, name
            del plan
            gc.collect()
    native.selinv_release_cached_memory()


def test_other_buffers_on_one_plan_are_read(native, cuda_device):
    """Calls on one plan with other device buffers (another matrix of the same
    pattern) keep its schedule and graph; the kernels must read the new
    buffers (the descriptors are rewritten in stream order)."""
    import torch
    p = CASES[7][1]()
    sym, L, D, Z = oracle_run(p)
    v = p.values.copy()
    v[p.diag_positions()] += 1.5
    L2, D2 = oracle.ldlt(p.with_values(v), sym)
    Z2 = oracle.selinv(sym, L2, D2)
    plan = native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows)
    bufs = []
    for (Lh, Dh) in ((L, D), (L2, D2), (L, D)):
        Lt = torch.from_numpy(Lh).cuda()
        Dt = torch.from_numpy(np.ascontiguousarray(Dh)).cuda()
        bufs.append((Lt, Dt, torch.full_like(Lt, float("nan"))))   # all alive: distinct addresses
    s = torch.cuda.Stream()
    for Lt, Dt, Zt in bufs:
        native.selinv_numeric(plan, native.SELINV_F64, Lt, Dt, Zt, s)
    s.synchronize()
    assert native.selinv_status(plan) == 0
    G = [b[2].cpu().numpy() for b in bufs]
    assert oracle.block_errors(sym, G[0], Z).max() <= TOL
    assert oracle.block_errors(sym, G[1], Z2).max() <= TOL
    assert np.array_equal(G[0], G[2])


@pytest.mark.parametrize("name,make", [CASES[7], CASES[8], CASES[9]])
def test_host_buffer_call_matches_device_call(native, cuda_device, name, make):
    """selinv_numeric_host (host L, D in, A^{-1} out, the copies overlapped
    with the traversal) gives the device call's result bit for bit, also on
    a second call with other values of the pattern."""
    import torch
    p = make()
    sym, L, D, Z = oracle_run(p)
    G_dev, plan = gpu_selinv(native, sym, L, D)
    dt = native.SELINV_C128 if L.dtype.kind == "c" else native.SELINV_F64
    Lh = torch.from_numpy(L).pin_memory()
    Dh = torch.from_numpy(np.ascontiguousarray(D)).pin_memory()
    Zh = torch.full(Lh.shape, float("nan"), dtype=Lh.dtype).pin_memory()
    Ld, Dd = torch.empty_like(Lh, device="cuda"), torch.empty_like(Dh, device="cuda")
    Zd = torch.empty_like(Lh, device="cuda")
    s = torch.cuda.Stream()
    for _ in range(2):
        Zh.fill_(float("nan"))
        native.selinv_numeric_host(plan, dt, Lh, Dh, Zh, Ld, Dd, Zd, s)
        s.synchronize()
        assert native.selinv_status(plan) == 0
        assert np.array_equal(Zh.numpy(), G_dev), name
    # pageable host buffers: the same result (the copies then serialize)
    Zp = torch.full(Lh.shape, float("nan"), dtype=Lh.dtype)
    native.selinv_numeric_host(plan, dt, torch.from_numpy(L), torch.from_numpy(np.ascontiguousarray(D)), Zp,
                               Ld, Dd, Zd, s)
    s.synchronize()
    assert np.array_equal(Zp.numpy(), G_dev), name
    if dt == native.SELINV_F64:
        v = p.values.copy()
        v[p.diag_positions()] += 1.5
        L2, D2 = oracle.ldlt(p.with_values(v), sym)
        Lh.copy_(torch.from_numpy(L2))
        Dh.copy_(torch.from_numpy(np.ascontiguousarray(D2)))
        native.selinv_numeric_host(plan, dt, Lh, Dh, Zh, Ld, Dd, Zd, s)
        s.synchronize()
        assert oracle.block_errors(sym, Zh.numpy(), oracle.selinv(sym, L2, D2)).max() <= TOL


def test_context_host_call_matches_oracle(native, cuda_device):
    """SelInvContext.selinv_host: host panels in, host A^{-1} out."""
    import torch
    from paper_1604_02528_gb300.api import SelInvContext
    p = synth.laplacian_3d(12, seed=8)
    sym, L, D, Z = oracle_run(p)
    ctx = SelInvContext.from_problem(p)
    G = ctx.selinv_host(torch.from_numpy(L).pin_memory(), torch.from_numpy(np.ascontiguousarray(D)).pin_memory())
    assert ctx.status() == 0
    assert oracle.block_errors(sym, G.numpy(), Z).max() <= TOL


def test_autotuned_plan_matches_oracle(native, cuda_device):
    """The first call tunes (engine, k-split, narrowest tensor-core supernode)
    on the caller's data; the tuned options stay valid and every result meets
    the tolerance."""
    import torch
    p = synth.laplacian_3d(16, seed=11)
    sym, L, D, Z = oracle_run(p)
    plan = native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows)
    o = native.selinv_default_opts()
    o.autotune = 1
    native.selinv_plan_set_opts(plan, o)
    Lt = torch.from_numpy(L).cuda(); Dt = torch.from_numpy(D).cuda()
    for _ in range(2):
        Zt = torch.full_like(Lt, float("nan"))
        native.selinv_numeric(plan, native.SELINV_F64, Lt, Dt, Zt, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert native.selinv_status(plan) == 0
        assert oracle.block_errors(sym, Zt.cpu().numpy(), Z).max() <= TOL
    t = native.selinv_plan_get_opts(plan)
    assert t.fast_contraction in (0, 1, 2)
    assert t.split_target in (1, 2, 4) and t.split_min_steps in (8, 16, 32) and t.oz_min_s in (1, 8, 16, 32, 64)


@pytest.mark.parametrize("name,make", [CASES[2], CASES[4], CASES[8],
                                       ("dft-6x6-nb32", lambda: synth.dft_sheet(side=6, nbasis=32, seed=13)),
                                       ("rand300-c128-relaxed", lambda: synth.random_sparse_spd(
                                           300, 0.02, 14, complex_values=True, supernodes=synth.problems.RELAXED_128))])
def test_complex_tensor_core_path_matches_oracle(native, cuda_device, name, make):
    """Complex symmetric supernodes on tcgen05 (the real contraction over
    k' = 2q + part with the 2s-row complex Lhat operand), every supernode
    (oz_min_s 1) and the default threshold, with and without k-splits: each
    block within 1e-10 of the oracle, the k-split bitwise irrelevant, and the
    FP64-pipe result within the same tolerance."""
    import torch
    p = make()
    sym, L, D, Z = oracle_run(p)
    plan = native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows)
    Lt = torch.from_numpy(L).cuda(); Dt = torch.from_numpy(D).cuda()
    outs = {}
    for fast, ozm, target, mins in ((1, 1, 1, 64), (1, 1, 8, 8), (1, 16, 2, 8), (0, 16, 2, 16)):
        o = native.selinv_default_opts()
        o.fast_contraction = fast
        o.oz_min_s = ozm
        o.split_target = target
        o.split_min_steps = mins
        native.selinv_plan_set_opts(plan, o)
        Zt = torch.full_like(Lt, float("nan"))
        native.selinv_numeric(plan, native.SELINV_C128, Lt, Dt, Zt, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert native.selinv_status(plan) == 0
        G = Zt.cpu().numpy()
        assert np.all(np.isfinite(G[oracle.lower_mask(sym)]))
        err = oracle.block_errors(sym, G, Z)
        assert err.max() <= TOL, (name, fast, ozm, target, float(err.max()))
        outs[(fast, ozm, target)] = G
    assert np.array_equal(outs[(1, 1, 1)], outs[(1, 1, 8)])
    # the full diagonal block is written, symmetric (plain transpose)
    G = outs[(1, 1, 1)]
    off = sym.panel_offsets()
    s, c = sym.sizes()
    for K in range(0, sym.nsuper, max(1, sym.nsuper // 40)):
        blk = G[off[K]:off[K + 1]].reshape(s[K], s[K] + c[K]).T[: s[K], :]
        assert np.array_equal(blk, blk.T)


@pytest.mark.parametrize("name,make", [CASES[1], CASES[4], CASES[7], CASES[8]])
def test_bounds_checked_gathers_change_nothing(native, cuda_device, name, make):
    """debug_checks bit 2 checks every gather address against the panel
    array before the load; on a valid plan no address fails, the status
    stays clear and every engine and schedule gives bit for bit the result
    it gives without the check."""
    import torch
    p = make()
    sym, L, D, Z = oracle_run(p)
    plan = native.selinv_symbolic(sym.n, sym.nsuper, sym.super_ptr, sym.sparent, sym.rowptr, sym.rows)
    dt = native.SELINV_C128 if L.dtype.kind == "c" else native.SELINV_F64
    Lt = torch.from_numpy(L).cuda(); Dt = torch.from_numpy(D).cuda()
    for fast, ozm, sched in ((1, 1, 1), (1, 16, 1), (2, 16, 1), (0, 16, 1), (0, 16, 3), (1, 16, 0)):
        if fast == 2 and dt != native.SELINV_F64:
            continue
        outs = []
        for checks in (0, native.DEBUG_CHECK_GATHER):
            o = native.selinv_default_opts()
            o.fast_contraction, o.oz_min_s, o.schedule, o.debug_checks = fast, ozm, sched, checks
            native.selinv_plan_set_opts(plan, o)
            Zt = torch.full_like(Lt, float("nan"))
            native.selinv_numeric(plan, dt, Lt, Dt, Zt, torch.cuda.current_stream())
            torch.cuda.synchronize()
            assert native.selinv_status(plan) == 0, (name, fast, sched, checks)
            outs.append(Zt.cpu().numpy())
        assert np.array_equal(outs[0], outs[1]), (name, fast, sched)
        assert oracle.block_errors(sym, outs[1], Z).max() <= TOL
