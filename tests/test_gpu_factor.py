"""GPU LDL^T (the prerequisite factorization) against the CPU oracle, and the
end-to-end path (GPU factor -> GPU selected inversion) against the oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

CASES = [
    ("rand80", lambda: synth.random_sparse_spd(80, 0.08, 1)),
    ("rand300-relaxed", lambda: synth.random_sparse_spd(300, 0.02, 2, supernodes=synth.problems.RELAXED_128)),
    ("rand100-c128", lambda: synth.random_sparse_spd(100, 0.1, 3, complex_values=True)),
    ("dense160", lambda: synth.random_sparse_spd(160, 1.0, 4, supernodes=synth.problems.RELAXED_128)),
    ("lap2d-63", lambda: synth.make_config(1)),
    ("lap3d-14-relaxed", lambda: synth.laplacian_3d(14, seed=6)),
    ("dft-8x8", lambda: synth.dft_sheet(side=8, nbasis=16)),
    ("diffusion-12", lambda: synth.diffusion_3d(12)),
]


def _ctx(p):
    from paper_1604_02528_gb300.api import SelInvContext
    return SelInvContext.from_problem(p)


@pytest.mark.parametrize("name,make", CASES)
def test_factor_matches_oracle(native, cuda_device, name, make):
    import torch
    p = make()
    ctx = _ctx(p)
    sym = oracle.symbolic_for(p)
    L0, D0 = oracle.ldlt(p, sym)
    A = torch.from_numpy(p.values).cuda()
    L, D = ctx.factor(A)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    Lg, Dg = L.cpu().numpy(), D.cpu().numpy()
    r, c, _ = oracle.panel_entries(sym)
    strict = r > c
    assert np.abs(Dg - D0).max() <= 1e-12 * np.abs(D0).max()
    assert oracle.block_errors(sym, np.where(strict, Lg, 0), np.where(strict, L0, 0)).max() <= 1e-10
    # end to end: GPU factor -> GPU selinv vs oracle factor -> oracle selinv
    Z = ctx.selinv(L, D)
    torch.cuda.synchronize()
    Z0 = oracle.selinv(sym, L0, D0)
    assert oracle.block_errors(sym, Z.cpu().numpy(), Z0).max() <= 1e-10


def test_factor_zero_pivot_is_reported(native, cuda_device):
    import torch
    # [[0, 1], [1, 0]]: the first pivot is exactly zero
    colptr = np.array([0, 2, 3], np.int64)
    rowind = np.array([0, 1, 1], np.int32)
    p = synth.Problem("zero-pivot", 2, colptr, rowind, np.array([0.0, 1.0, 0.0]), np.arange(2))
    ctx = _ctx(p)
    ctx.factor(torch.from_numpy(p.values).cuda())
    torch.cuda.synchronize()
    assert ctx.status() == native.SelinvError(-4).code
    assert ctx.status() == 0  # the status word is cleared after reading
