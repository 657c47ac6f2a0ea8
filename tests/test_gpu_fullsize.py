"""Parity at the full sizes of the configured workloads, in the launch
configuration the benchmark times (level schedule, CUDA graph, tensor-core
contraction for real supernodes with s >= 16).

* 40^3 Laplacian (N = 64000): every block against the oracle's selected
  inversion of the oracle's own factors, plus the GPU factorization.
* DFT-like complex sheet (N = 16384) and the pole-shifted 40^3 pattern:
  sampled columns computed one by one by the oracle's substitution solve,
  and the row-times-column invariant sum_k A_jk Ainv_kj = 1 on every j.
* 24^3 diffusion: the gradient of the selected-entry loss against the
  oracle's reverse mode.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = 1e-10


def a_positions(sym, p):
    off = sym.panel_offsets()
    sp = sym.super_ptr
    col2s = np.repeat(np.arange(sym.nsuper), np.diff(sp))
    cols = np.repeat(np.arange(p.n), np.diff(p.colptr))
    K = col2s[cols]
    pos = np.empty(p.rowind.size, dtype=np.int64)
    for k in range(p.rowind.size):
        R = sym.rows[sym.rowptr[K[k]]:sym.rowptr[K[k] + 1]]
        pos[k] = off[K[k]] + (cols[k] - sp[K[k]]) * R.size + np.searchsorted(R, p.rowind[k])
    return pos


def invariant_residual(p, sym, Z, pos):
    cols = np.repeat(np.arange(p.n), np.diff(p.colptr))
    acc = np.zeros(p.n, dtype=Z.dtype)
    prod = p.values * Z[pos]
    np.add.at(acc, cols, prod)
    off = p.rowind != cols
    np.add.at(acc, p.rowind[off], prod[off])
    return np.abs(acc - 1).max()


def sampled_columns_error(sym, L, D, Z, js):
    """max relative error of the stored lower entries of columns js."""
    off = sym.panel_offsets()
    sp = sym.super_ptr
    col2s = np.repeat(np.arange(sym.nsuper), np.diff(sp))
    worst = 0.0
    for j in js:
        x = oracle.selected_column(sym, L, D, int(j))
        K = col2s[j]
        R = sym.rows[sym.rowptr[K]:sym.rowptr[K + 1]]
        jj = j - sp[K]
        got = Z[off[K] + jj * R.size + jj: off[K] + (jj + 1) * R.size]
        want = x[R[jj:]]
        worst = max(worst, float(np.linalg.norm(got - want) / np.linalg.norm(want)))
    return worst


def test_lap3d_40_all_blocks(native, cuda_device):
    import torch
    from paper_1604_02528_gb300.api import SelInvContext
    p = synth.make_config(2)
    sym = oracle.symbolic_for(p)
    L0, D0 = oracle.ldlt(p, sym)
    Z0 = oracle.selinv(sym, L0, D0)
    ctx = SelInvContext.from_problem(p)
    G = ctx.selinv(torch.from_numpy(L0).cuda(), torch.from_numpy(D0).cuda(),
                   stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert ctx.status() == 0
    err = oracle.block_errors(sym, G.cpu().numpy(), Z0)
    assert err.max() <= TOL, err.max()
    # GPU factorization -> GPU selected inversion, end to end
    L, D = ctx.factor(torch.from_numpy(p.values).cuda())
    Z = ctx.selinv(L, D)
    torch.cuda.synchronize()
    assert oracle.block_errors(sym, Z.cpu().numpy(), Z0).max() <= TOL
    assert invariant_residual(p, sym, Z.cpu().numpy(), a_positions(sym, p)) <= 1e-10


def test_dft_sheet_sampled_columns(native, cuda_device):
    import torch
    from paper_1604_02528_gb300.api import SelInvContext
    p = synth.make_config(3)
    ctx = SelInvContext.from_problem(p)
    L, D = ctx.factor(torch.from_numpy(p.values).cuda())
    Z = ctx.selinv(L, D)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    sym = oracle.symbolic_for(p)
    Zh = Z.cpu().numpy()
    assert invariant_residual(p, sym, Zh, a_positions(sym, p)) <= 1e-9
    # sampled columns from the GPU factors (isolates the selected inversion)
    js = np.random.default_rng(9).choice(p.n, size=12, replace=False)
    assert sampled_columns_error(sym, L.cpu().numpy(), D.cpu().numpy(), Zh, js) <= TOL


def test_pole_shifts_batched_sampled(native, cuda_device):
    """Four pole shifts of the 40^3 pattern plus two uneven Laplacians in one
    batched launch sequence; invariant on every column, sampled columns."""
    import torch
    from paper_1604_02528_gb300.api import SelInvContext
    base = synth.make_config(4)
    e, eta = synth.pole_shifts()
    probs = [base.with_values(synth.problems.shifted_values(base, complex(e[l], eta[l])))
             for l in (0, 13, 26, 39)]
    probs += [synth.laplacian_2d(45), synth.laplacian_3d(22, seed=42)]
    ctxs, Ls, Ds, Zs, dts = [], [], [], [], []
    base_ctx = SelInvContext.from_problem(base)
    for q in probs:
        c = base_ctx if q.n == base.n else SelInvContext.from_problem(q)
        L, D = c.factor(torch.from_numpy(q.values).cuda())
        torch.cuda.synchronize()
        ctxs.append(c); Ls.append(L); Ds.append(D); Zs.append(torch.empty_like(L))
        dts.append(native.SELINV_C128 if q.values.dtype.kind == "c" else native.SELINV_F64)
    native.selinv_numeric_batched([c.plan for c in ctxs], dts, Ls, Ds, Zs, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert ctxs[0].status() == 0
    for q, c, L, D, Z in zip(probs, ctxs, Ls, Ds, Zs):
        sym = oracle.symbolic_for(q)
        Zh = Z.cpu().numpy()
        assert invariant_residual(q, sym, Zh, a_positions(sym, q)) <= 1e-8
        js = np.random.default_rng(q.n).choice(q.n, size=4, replace=False)
        assert sampled_columns_error(sym, L.cpu().numpy(), D.cpu().numpy(), Zh, js) <= TOL


def test_diffusion_24_gradient(native, cuda_device):
    import torch
    from paper_1604_02528_gb300.api import SelInvContext
    from paper_1604_02528_gb300.autograd import SelInv
    p = synth.make_config(5)
    meta = p.meta
    sym = oracle.symbolic_for(p)
    low = oracle.lower_mask(sym)
    W = np.where(low, synth.lower_pattern_weights(low.size), 0.0)
    ctx = SelInvContext.from_problem(p)
    ent = torch.from_numpy(meta["asm_entry"]).cuda()
    edg = torch.from_numpy(meta["asm_edge"]).cuda()
    sgn = torch.from_numpy(meta["asm_sign"]).cuda()
    theta = torch.from_numpy(meta["theta"]).cuda().requires_grad_(True)
    A = torch.zeros(p.nnz_lower, dtype=torch.float64, device="cuda").index_add(0, ent, sgn * theta[edg])
    Z = SelInv.apply(ctx, A)
    (torch.from_numpy(W).cuda() * Z).sum().backward()
    g = theta.grad.cpu().numpy()
    L0, D0 = oracle.ldlt(p, sym)
    Z0 = oracle.selinv(sym, L0, D0)
    assert oracle.block_errors(sym, Z.detach().cpu().numpy(), Z0).max() <= TOL
    Lb0, Db0 = oracle.selinv_adjoint(sym, L0, D0, Z0, W)
    Ab0 = oracle.ldlt_adjoint(sym, L0, D0, Lb0, Db0)
    pos = a_positions(sym, p)
    g0 = np.zeros_like(g)
    np.add.at(g0, meta["asm_edge"], meta["asm_sign"] * Ab0[pos[meta["asm_entry"]]])
    assert np.linalg.norm(g - g0) / np.linalg.norm(g0) <= TOL
