"""GPU reverse mode against the oracle's reverse mode, the dense gradient and
central differences (FP64)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

CASES = [
    ("rand60", lambda: synth.random_sparse_spd(60, 0.08, 41)),
    ("rand200-relaxed", lambda: synth.random_sparse_spd(200, 0.03, 42, supernodes=synth.problems.RELAXED_128)),
    ("dense150", lambda: synth.random_sparse_spd(150, 1.0, 43, supernodes=synth.problems.RELAXED_128)),
    ("diffusion-8", lambda: synth.diffusion_3d(8)),
    ("lap3d-12", lambda: synth.laplacian_3d(12, seed=44)),
    ("diffusion-16", lambda: synth.diffusion_3d(16)),
    # narrow supernodes with 256 or more rows below: the split path whatever their width
    ("rand400-long-c", lambda: synth.random_sparse_spd(400, 0.03, 46)),
]


def a_positions(sym, p):
    off = sym.panel_offsets()
    sp = sym.super_ptr
    col2s = np.repeat(np.arange(sym.nsuper), np.diff(sp))
    cols = np.repeat(np.arange(p.n), np.diff(p.colptr))
    pos = np.empty(p.rowind.size, dtype=np.int64)
    for k, (i, j) in enumerate(zip(p.rowind, cols)):
        K = col2s[j]
        R = sym.rows[sym.rowptr[K]:sym.rowptr[K + 1]]
        pos[k] = off[K] + (j - sp[K]) * R.size + np.searchsorted(R, i)
    return pos


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("engine,ozm", [(1, 16), (1, 8), (2, 16), (0, 16)])
@pytest.mark.parametrize("name,make", CASES)
def test_adjoints_match_oracle(native, cuda_device, name, make, engine, ozm):
    """engines 1 and 2 (the forward's tcgen05 or mma.sync choice): supernodes
    of ozm columns or more take the split path (tcgen05 gather-GEMM, 32 x 32
    blocks for the s-inner products); 0: every supernode on the fused FP64
    kernels."""
    import torch
    from paper_1604_02528_gb300.api import SelInvContext
    p = make()
    sym = oracle.symbolic_for(p)
    L, D = oracle.ldlt(p, sym)
    Z = oracle.selinv(sym, L, D)
    low = oracle.lower_mask(sym)
    W = np.where(low, np.random.default_rng(7).standard_normal(low.size), 0.0)
    Lb0, Db0 = oracle.selinv_adjoint(sym, L, D, Z, W)
    Ab0 = oracle.ldlt_adjoint(sym, L, D, Lb0, Db0)
    ctx = SelInvContext.from_problem(p)
    ctx.attach_matrix()
    o = native.selinv_default_opts()
    o.fast_contraction = engine
    o.oz_min_s = ozm
    o.split_min_steps = 8       # k-split tcgen05 items from c >= 256 on
    native.selinv_plan_set_opts(ctx.plan, o)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    Lt, Dt, Zt, Wt = t(L), t(D), t(Z), t(W)
    Lb = torch.full_like(Lt, float("nan")); Db = torch.full_like(Dt, float("nan"))
    native.selinv_adjoint(ctx.plan, native.SELINV_F64, Lt, Dt, Zt, Wt, Lb, Db)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    r, c, _ = oracle.panel_entries(sym)
    strict = r > c
    Lbg = Lb.cpu().numpy()
    assert rel(np.where(strict, Lbg, 0), np.where(strict, Lb0, 0)) <= 1e-10
    assert rel(Db.cpu().numpy(), Db0) <= 1e-10
    # factorization adjoint from the oracle's (Lbar, Dbar): isolates that kernel chain
    Ab = torch.full((p.nnz_lower,), float("nan"), dtype=torch.float64, device="cuda")
    native.selinv_factor_adjoint(ctx.plan, native.SELINV_F64, Lt, Dt, t(Lb0), t(Db0), Ab)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    pos = a_positions(sym, p)
    assert rel(Ab.cpu().numpy(), Ab0[pos]) <= 1e-10


def test_autograd_diffusion_gradient(native, cuda_device):
    """Loss on the selected entries -> d loss / d theta on a 10^3 diffusion
    grid: GPU autograd vs the oracle chain, and vs central differences."""
    import torch
    from paper_1604_02528_gb300.api import SelInvContext
    from paper_1604_02528_gb300.autograd import SelInv
    p = synth.diffusion_3d(10)
    meta = p.meta
    sym = oracle.symbolic_for(p)
    low = oracle.lower_mask(sym)
    W = np.where(low, synth.lower_pattern_weights(low.size), 0.0)
    ctx = SelInvContext.from_problem(p)
    # theta -> A values through the assembly map (sign * theta[edge] summed per entry)
    ent = torch.from_numpy(meta["asm_entry"]).cuda()
    edg = torch.from_numpy(meta["asm_edge"]).cuda()
    sgn = torch.from_numpy(meta["asm_sign"]).cuda()
    theta = torch.from_numpy(meta["theta"]).cuda().requires_grad_(True)
    A = torch.zeros(p.nnz_lower, dtype=torch.float64, device="cuda").index_add(0, ent, sgn * theta[edg])
    Z = SelInv.apply(ctx, A)
    loss = (torch.from_numpy(W).cuda() * Z).sum()
    loss.backward()
    g = theta.grad.cpu().numpy()
    # oracle chain
    L0, D0 = oracle.ldlt(p, sym)
    Z0 = oracle.selinv(sym, L0, D0)
    Lb0, Db0 = oracle.selinv_adjoint(sym, L0, D0, Z0, W)
    Ab0 = oracle.ldlt_adjoint(sym, L0, D0, Lb0, Db0)
    pos = a_positions(sym, p)
    g0 = np.zeros_like(g)
    np.add.at(g0, meta["asm_edge"], meta["asm_sign"] * Ab0[pos[meta["asm_entry"]]])
    assert rel(g, g0) <= 1e-10
    assert abs(loss.item() - float((W * Z0).sum())) <= 1e-10 * abs(float((W * Z0).sum()))
    # central differences on a few edges
    rng = np.random.default_rng(3)
    h = 1e-5
    for e in rng.choice(g.size, size=6, replace=False):
        vals = []
        for sg in (+1, -1):
            th = meta["theta"].copy(); th[e] += sg * h
            q = synth.diffusion_3d(10, theta=th)
            Lq, Dq = oracle.ldlt(q, sym)
            vals.append(float((W * oracle.selinv(sym, Lq, Dq)).sum()))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[e]) <= 1e-6 * max(1.0, abs(g[e]))


def test_autograd_unmasked_loss_reads_whole_diagonal_blocks(native, cuda_device):
    """The forward returns whole diagonal blocks (upper part = mirrored lower
    entries).  A loss over every returned slot (Z.sum() and an unmasked W)
    must give the gradient of that loss: on the oracle side the upper slots'
    weights are added to their lower mirrors (same value of Z)."""
    import torch
    from paper_1604_02528_gb300.api import SelInvContext
    from paper_1604_02528_gb300.autograd import SelInv
    p = synth.random_sparse_spd(120, 0.05, 91, supernodes=synth.problems.RELAXED_128)
    sym = oracle.symbolic_for(p)
    low = oracle.lower_mask(sym)
    r, c, _ = oracle.panel_entries(sym)
    rng = np.random.default_rng(92)
    ctx = SelInvContext.from_problem(p)
    L0, D0 = oracle.ldlt(p, sym)
    Z0 = oracle.selinv(sym, L0, D0)
    pos = a_positions(sym, p)
    # mirror slot of each upper diagonal-block slot (same supernode, same panel)
    off = sym.panel_offsets()
    sp = sym.super_ptr
    col2s = np.repeat(np.arange(sym.nsuper), np.diff(sp))
    mirror = np.arange(low.size)
    up = np.nonzero(~low)[0]
    for e in up:
        i, j = int(r[e]), int(c[e])          # row i < column j, both columns of one supernode
        K = col2s[j]
        ld = sym.rowptr[K + 1] - sym.rowptr[K]
        mirror[e] = off[K] + (i - sp[K]) * ld + (j - sp[K])
    for kind in ("sum", "unmasked"):
        W = np.ones(low.size) if kind == "sum" else rng.standard_normal(low.size)
        A = torch.from_numpy(p.values).cuda().requires_grad_(True)
        Z = SelInv.apply(ctx, A)
        loss = (torch.from_numpy(W).cuda() * Z).sum()
        loss.backward()
        g = A.grad.cpu().numpy()
        Wf = np.where(low, W, 0.0)
        np.add.at(Wf, mirror[up], W[up])
        Lb0, Db0 = oracle.selinv_adjoint(sym, L0, D0, Z0, Wf)
        Ab0 = oracle.ldlt_adjoint(sym, L0, D0, Lb0, Db0)
        assert rel(g, Ab0[pos]) <= 1e-10, kind
        assert abs(loss.item() - float((W * Z0).sum())) <= 1e-10 * abs(float((W * Z0).sum()))


def test_autograd_raises_on_zero_pivot(native, cuda_device):
    """A zero pivot in the forward factorization is reported, not returned."""
    import torch
    from paper_1604_02528_gb300.api import SelInvContext
    from paper_1604_02528_gb300.autograd import SelInv
    # [[0, 1], [1, 0]]: the first pivot is exactly zero
    colptr = np.array([0, 2, 3], np.int64)
    rowind = np.array([0, 1, 1], np.int32)
    ctx = SelInvContext(2, colptr, rowind)
    A = torch.tensor([0.0, 1.0, 0.0], dtype=torch.float64, device="cuda").requires_grad_(True)
    with pytest.raises(native.SelinvError):
        SelInv.apply(ctx, A)
