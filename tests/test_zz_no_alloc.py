"""The allocation-free entry point (selinv_dinv_noalloc) against the regular
path.

Callers that cannot allocate device memory (latency-critical loops, memory
owned by another allocator, contexts where allocation is not permitted) use
selinv_dinv_noalloc, whose scratch is a static device array.  For a matrix
that is a single supernode, Dinv of its only diagonal block is the whole
inverse, which selinv_numeric also returns: the two must agree.  Two calls
in a row (different sizes and values) check that the shared static scratch
carries nothing over from one call to the next.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10
MAX_S = 128   # SELINV_NOALLOC_MAX_S


def one_supernode_problem(n, seed):
    p = synth.random_sparse_spd(n, 1.0, seed, permute=False)
    p.supernodes = {"kind": "fundamental", "cap": 128, "fill": 0.0}
    return p


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_selinv_numeric_two_calls(native, cuda_device):
    import torch
    from paper_1604_02528_gb300.api import SelInvContext
    for n, seed in ((100, 301), (37, 302)):
        p = one_supernode_problem(n, seed)
        ctx = SelInvContext.from_problem(p)
        assert ctx.nsuper == 1
        L, D = ctx.factor(torch.from_numpy(p.values).cuda())
        Z = ctx.selinv(L, D)                                    # existing entry point
        out = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        native.selinv_dinv_noalloc(n, L, n, D, out, n)          # ld = s + c = n for one supernode
        torch.cuda.synchronize()
        assert ctx.status() == 0
        ref = Z.cpu().numpy().reshape(n, n).T                   # column-major panel -> [row, col]
        got = out.cpu().numpy().T
        assert np.all(np.isfinite(got))
        assert rel(got, ref) <= TOL
        assert rel(got, np.linalg.inv(p.dense())) <= TOL


def test_noalloc_rejects_blocks_beyond_the_static_scratch(native, cuda_device):
    import torch
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(native.SelinvError) as e:
        native.selinv_dinv_noalloc(MAX_S + 1, t, 200, t, t, 200)
    assert e.value.code == -1

