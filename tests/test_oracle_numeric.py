"""Pins for the oracle's numeric part (CPU only).

Each check is independent of the recursion it pins:
  * dense inverse (numpy.linalg.inv) on small random real and complex
    symmetric matrices, for several supernode rules;
  * closed form of tridiag(-1, 2, -1)^{-1};
  * the 2D Dirichlet Laplacian's sine eigen-expansion (63 x 63 grid, the
    63^2 workload) and its trace sum 1/(lambda_pq + 0.1);
  * the 2 x 2 block inverse with a Schur complement (Sec. II-A) for a matrix
    of exactly two supernodes;
  * selected columns from sparse LU solves (scipy.sparse.linalg.splu);
  * the invariant sum_k A_jk Ainv_kj = 1 for every j (needs only entries on
    the pattern);
  * Alg. 1 (pull) against Alg. 2 (push), two summation orders;
  * LDL^T residual;
  * adjoints against the dense gradient -(Z Wbar Z) and central differences,
    real and complex symmetric (plain transposes: the loss is bilinear in Z,
    so the gradient is the holomorphic derivative and central differences
    along the real and the imaginary axis must give the same value).
"""
import numpy as np
import pytest
import scipy.sparse as sps
import scipy.sparse.linalg as spla

import oracle
import synth


def full_sparse(p):
    """Symmetric scipy CSC matrix of the permuted problem."""
    cols = np.repeat(np.arange(p.n), np.diff(p.colptr))
    low = sps.csc_matrix((p.values, (p.rowind, cols)), shape=(p.n, p.n))
    return (low + low.T - sps.diags(low.diagonal())).tocsc()


def a_positions(sym, p):
    """Panel position of every stored lower entry of A (format lookup)."""
    off = sym.panel_offsets()
    sp = sym.super_ptr
    col2s = np.repeat(np.arange(sym.nsuper), np.diff(sp))
    cols = np.repeat(np.arange(p.n), np.diff(p.colptr))
    pos = np.empty(p.rowind.size, dtype=np.int64)
    for k, (i, j) in enumerate(zip(p.rowind, cols)):
        K = col2s[j]
        R = sym.rows[sym.rowptr[K]:sym.rowptr[K + 1]]
        r = np.searchsorted(R, i)
        assert R[r] == i
        pos[k] = off[K] + (j - sp[K]) * R.size + r
    return pos


def run(p, symmetrize=True):
    sym = oracle.symbolic_for(p)
    L, D = oracle.ldlt(p, sym)
    Z = oracle.selinv(sym, L, D, symmetrize)
    return sym, L, D, Z


CASES = [
    ("real-fund", lambda: synth.random_sparse_spd(60, 0.08, 11)),
    ("real-dense", lambda: synth.random_sparse_spd(40, 1.0, 12)),
    ("real-relaxed", lambda: synth.random_sparse_spd(90, 0.04, 13, supernodes=synth.problems.RELAXED_128)),
    ("real-cap1", lambda: synth.random_sparse_spd(50, 0.1, 14, supernodes={"kind": "fundamental", "cap": 1, "fill": 0})),
    ("cplx-fund", lambda: synth.random_sparse_spd(60, 0.08, 15, complex_values=True)),
    ("cplx-relaxed", lambda: synth.random_sparse_spd(80, 0.05, 16, complex_values=True, supernodes=synth.problems.RELAXED_128)),
    ("lap3d-6", lambda: synth.laplacian_3d(6, seed=17)),
    ("dft-small", lambda: synth.dft_sheet(side=4, nbasis=4)),
]


@pytest.mark.parametrize("name,make", CASES)
def test_selinv_matches_dense_inverse(name, make):
    p = make()
    sym, L, D, Z = run(p)
    ref = oracle.dense_to_panels(sym, np.linalg.inv(p.dense()))
    err = oracle.block_errors(sym, Z, ref)
    assert err.max() < 1e-12, (name, err.max())


@pytest.mark.parametrize("name,make", CASES)
def test_ldlt_residual(name, make):
    p = make()
    sym = oracle.symbolic_for(p)
    L, D = oracle.ldlt(p, sym)
    r, c, _ = oracle.panel_entries(sym)
    m = r > c
    Ld = np.eye(p.n, dtype=L.dtype)
    Ld[r[m], c[m]] = L[m]
    A = p.dense()
    res = np.abs(Ld @ np.diag(D) @ Ld.T - A).max() / np.abs(A).max()
    assert res < 1e-13


@pytest.mark.parametrize("name,make", CASES)
def test_pull_and_push_agree(name, make):
    p = make()
    sym, L, D, Z = run(p)
    Zp = oracle.selinv_push(sym, L, D)
    assert oracle.block_errors(sym, Zp, Z).max() < 1e-13


@pytest.mark.parametrize("n", [1, 2, 7, 64, 200])
@pytest.mark.parametrize("nd", [False, True])
def test_tridiagonal_closed_form(n, nd):
    p = synth.tridiagonal(n, nd=nd)
    sym, L, D, Z = run(p)
    i = p.perm[:, None] + 1
    j = p.perm[None, :] + 1
    exact = np.minimum(i, j) * (n + 1 - np.maximum(i, j)) / (n + 1)
    ref = oracle.dense_to_panels(sym, exact)
    kappa = 4.0 * (n + 1) ** 2 / np.pi ** 2        # condition number of tridiag(-1,2,-1)
    assert oracle.block_errors(sym, Z, ref).max() < 1e-14 + 1e-15 * kappa


def laplacian_2d_inverse_by_eigen(m, shift):
    """Dense inverse of the m x m Dirichlet 5-point Laplacian + shift I from
    its sine eigenvectors (no linear solve)."""
    h = m + 1
    x = np.arange(1, m + 1)
    S = np.sqrt(2.0 / h) * np.sin(np.pi * np.outer(x, x) / h)   # S[x, p], orthonormal
    lam1 = 2 - 2 * np.cos(np.pi * x / h)
    lam = lam1[:, None] + lam1[None, :] + shift                  # [p, q]
    # node id = ix + m * iy, mode id = p + m * q
    Phi = np.kron(S, S)                                           # [(y,x),(q,p)]
    Z = (Phi / lam.T.ravel()[None, :]) @ Phi.T
    return Z, (1.0 / lam).sum()


def test_laplacian_2d_eigen_expansion_63():
    p = synth.make_config(1)
    sym, L, D, Z = run(p)
    Zd, trace = laplacian_2d_inverse_by_eigen(63, 0.1)
    Zperm = Zd[np.ix_(p.perm, p.perm)]
    ref = oracle.dense_to_panels(sym, Zperm)
    err = oracle.block_errors(sym, Z, ref)
    assert err.max() < 1e-12
    # trace from the selected diagonal = sum of reciprocal eigenvalues
    r, c, _ = oracle.panel_entries(sym)
    tr = Z[r == c].sum()
    assert abs(tr - trace) / trace < 1e-13


def test_two_supernode_block_formula():
    rng = np.random.default_rng(21)
    n1, n2 = 4, 4
    n = n1 + n2
    B = rng.standard_normal((n, n))
    A = B @ B.T + n * np.eye(n)
    rows, cols = np.tril_indices(n)
    order = np.lexsort((rows, cols))
    colptr = np.concatenate([[0], np.cumsum(np.bincount(cols[order], minlength=n))]).astype(np.int64)
    p = synth.Problem("dense8", n, colptr, rows[order].astype(np.int32), A[rows[order], cols[order]],
                      np.arange(n), {"kind": "fundamental", "cap": n1, "fill": 0.0})
    sym, L, D, Z = run(p)
    assert sym.super_ptr.tolist() == [0, n1, n]      # exactly two supernodes
    A11, A12, A21, A22 = A[:n1, :n1], A[:n1, n1:], A[n1:, :n1], A[n1:, n1:]
    A11i = np.linalg.inv(A11)
    S = A22 - A21 @ A11i @ A12                      # Schur complement
    Si = np.linalg.inv(S)
    Lh = A21 @ A11i                                 # Lhat_21 = L21 L11^{-1}
    Uh = A11i @ A12                                 # Uhat_12 = U11^{-1} U12
    Zref = np.block([[A11i + Uh @ Si @ Lh, -Uh @ Si], [-Si @ Lh, Si]])
    ref = oracle.dense_to_panels(sym, Zref)
    assert oracle.block_errors(sym, Z, ref).max() < 1e-13


@pytest.mark.parametrize("make", [lambda: synth.laplacian_3d(16, seed=2),
                                  lambda: synth.dft_sheet(side=8, nbasis=8)])
def test_selected_columns_by_sparse_lu(make):
    p = make()
    sym, L, D, Z = run(p)
    lu = spla.splu(full_sparse(p), permc_spec="NATURAL")
    off = sym.panel_offsets()
    sp = sym.super_ptr
    col2s = np.repeat(np.arange(sym.nsuper), np.diff(sp))
    rng = np.random.default_rng(5)
    for j in rng.choice(p.n, size=24, replace=False):
        e = np.zeros(p.n, dtype=p.values.dtype); e[j] = 1
        x = lu.solve(e)
        K = col2s[j]
        R = sym.rows[sym.rowptr[K]:sym.rowptr[K + 1]]
        jj = j - sp[K]
        got = Z[off[K] + jj * R.size + jj: off[K] + (jj + 1) * R.size]
        want = x[R[jj:]]
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("make", [lambda: synth.make_config(1), lambda: synth.laplacian_3d(16, seed=2),
                                  lambda: synth.diffusion_3d(10), lambda: synth.dft_sheet(side=8, nbasis=8)])
def test_row_times_column_invariant(make):
    p = make()
    sym, L, D, Z = run(p)
    pos = a_positions(sym, p)
    cols = np.repeat(np.arange(p.n), np.diff(p.colptr))
    acc = np.zeros(p.n, dtype=Z.dtype)
    prod = p.values * Z[pos]
    np.add.at(acc, cols, prod)
    off = p.rowind != cols
    np.add.at(acc, p.rowind[off], prod[off])
    assert np.abs(acc - 1).max() < 1e-11


def test_no_symmetrize_still_inverse_for_exact_input():
    p = synth.random_sparse_spd(50, 0.1, 31)
    sym, L, D, Z = run(p, symmetrize=False)
    ref = oracle.dense_to_panels(sym, np.linalg.inv(p.dense()))
    assert oracle.block_errors(sym, Z, ref).max() < 1e-12


# ----------------------------------------------------------------- adjoints

def loss_and_grad_dense(p, sym, W):
    """l = sum_stored W_ij Z_ij and dl/da (stored lower entries of A on the
    L pattern) from the dense formula -(M + M^T) off the diagonal, -M_ii on
    it, with M = Z Wbar Z and Wbar = W scattered to the lower triangle."""
    Zd = np.linalg.inv(p.dense())
    r, c, low = oracle.panel_entries(sym)
    Wb = np.zeros((p.n, p.n), dtype=Zd.dtype)
    Wb[r[low], c[low]] = W[low]
    M = Zd @ Wb @ Zd
    G = -(M + M.T)
    G[np.diag_indices(p.n)] = -np.diag(M)
    grad = np.zeros(r.size, dtype=Zd.dtype)
    grad[low] = G[r[low], c[low]]
    loss = (W[low] * oracle.dense_to_panels(sym, Zd)[low]).sum()
    loss = complex(loss) if np.iscomplexobj(loss) else float(loss)
    return loss, grad


@pytest.mark.parametrize("make", [lambda: synth.random_sparse_spd(60, 0.08, 41),
                                  lambda: synth.random_sparse_spd(70, 0.06, 42, supernodes=synth.problems.RELAXED_128),
                                  lambda: synth.diffusion_3d(5),
                                  lambda: synth.laplacian_3d(6, seed=43)])
def test_adjoint_chain_matches_dense_gradient(make):
    p = make()
    sym, L, D, Z = run(p)
    low = oracle.lower_mask(sym)
    W = np.where(low, np.random.default_rng(44).standard_normal(low.size), 0.0)
    Lb, Db = oracle.selinv_adjoint(sym, L, D, Z, W)
    Ab = oracle.ldlt_adjoint(sym, L, D, Lb, Db)
    _, grad = loss_and_grad_dense(p, sym, W)
    assert np.abs(Ab - grad)[low].max() <= 1e-10 * np.abs(grad).max()
    # nothing leaks into the unused strictly-upper slots of diagonal blocks
    assert np.all(Ab[~low] == 0)


def test_adjoint_central_differences_on_theta():
    p = synth.diffusion_3d(5)
    sym, L, D, Z = run(p)
    low = oracle.lower_mask(sym)
    W = np.where(low, np.random.default_rng(45).standard_normal(low.size), 0.0)
    Lb, Db = oracle.selinv_adjoint(sym, L, D, Z, W)
    Ab = oracle.ldlt_adjoint(sym, L, D, Lb, Db)
    pos = a_positions(sym, p)
    meta = p.meta
    # chain through the edge assembly: dl/dtheta_e = sum sign * Abar[entry]
    gth = np.zeros(meta["theta"].size)
    np.add.at(gth, meta["asm_edge"], meta["asm_sign"] * Ab[pos[meta["asm_entry"]]])

    def loss(theta):
        q = synth.diffusion_3d(5, theta=theta)
        Lq, Dq = oracle.ldlt(q, sym)
        Zq = oracle.selinv(sym, Lq, Dq)
        return float((W * Zq)[low].sum())

    rng = np.random.default_rng(46)
    h = 1e-5
    for e in rng.choice(gth.size, size=12, replace=False):
        tp = meta["theta"].copy(); tp[e] += h
        tm = meta["theta"].copy(); tm[e] -= h
        fd = (loss(tp) - loss(tm)) / (2 * h)
        assert abs(fd - gth[e]) <= 1e-6 * max(1.0, abs(gth[e]))


def test_selinv_adjoint_central_differences_on_L():
    p = synth.random_sparse_spd(40, 0.12, 47)
    sym, L, D, Z = run(p)
    low = oracle.lower_mask(sym)
    W = np.where(low, np.random.default_rng(48).standard_normal(low.size), 0.0)
    Lb, Db = oracle.selinv_adjoint(sym, L, D, Z, W)
    r, c, _ = oracle.panel_entries(sym)
    strict = np.nonzero(r > c)[0]
    rng = np.random.default_rng(49)
    h = 1e-6
    f = lambda LL, DD: float((W * oracle.selinv(sym, LL, DD))[low].sum())
    for e in rng.choice(strict, size=10, replace=False):
        Lp = L.copy(); Lp[e] += h
        Lm = L.copy(); Lm[e] -= h
        fd = (f(Lp, D) - f(Lm, D)) / (2 * h)
        assert abs(fd - Lb[e]) <= 1e-6 * max(1.0, abs(Lb[e]))
    for k in rng.choice(p.n, size=6, replace=False):
        Dp = D.copy(); Dp[k] += h
        Dm = D.copy(); Dm[k] -= h
        fd = (f(L, Dp) - f(L, Dm)) / (2 * h)
        assert abs(fd - Db[k]) <= 1e-6 * max(1.0, abs(Db[k]))


@pytest.mark.parametrize("make", [lambda: synth.random_sparse_spd(70, 0.1, 51),
                                  lambda: synth.random_sparse_spd(60, 0.1, 52, complex_values=True),
                                  lambda: synth.laplacian_3d(7, seed=53)])
def test_solve_matches_dense_solve(make):
    """The oracle's substitution solve (used for sampled columns at full size)."""
    p = make()
    sym = oracle.symbolic_for(p)
    L, D = oracle.ldlt(p, sym)
    rng = np.random.default_rng(54)
    b = rng.standard_normal(p.n).astype(p.values.dtype)
    x = oracle.solve(sym, L, D, b)
    ref = np.linalg.solve(p.dense(), b)
    assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max()


# ------------------------------------------------- complex symmetric adjoints
#
# A = A^T with complex values: Z = A^{-1} is a holomorphic function of the
# stored entries and the loss l = sum W_ij Z_ij is bilinear, so dl/da is the
# complex derivative, dZ = -Z dA Z with plain transposes (Sec. II-C), and the
# dense gradient is the same expression as in the real case.

CPLX_ADJ = [
    ("rand-fund", lambda: synth.random_sparse_spd(60, 0.08, 61, complex_values=True)),
    ("rand-relaxed", lambda: synth.random_sparse_spd(70, 0.06, 62, complex_values=True,
                                                     supernodes=synth.problems.RELAXED_128)),
    ("dft-small", lambda: synth.dft_sheet(side=4, nbasis=4, seed=63)),
]


def complex_weights(low, seed):
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(low.size) + 1j * rng.standard_normal(low.size)
    return np.where(low, w, 0.0)


@pytest.mark.parametrize("name,make", CPLX_ADJ)
def test_complex_adjoint_chain_matches_dense_gradient(name, make):
    p = make()
    assert np.iscomplexobj(p.values)
    sym, L, D, Z = run(p)
    low = oracle.lower_mask(sym)
    W = complex_weights(low, 64)
    Lb, Db = oracle.selinv_adjoint(sym, L, D, Z, W)
    Ab = oracle.ldlt_adjoint(sym, L, D, Lb, Db)
    loss, grad = loss_and_grad_dense(p, sym, W)
    assert abs(loss - (W * Z)[low].sum()) <= 1e-10 * abs(loss)
    assert np.abs(Ab - grad)[low].max() <= 1e-10 * np.abs(grad).max(), name
    assert np.all(Ab[~low] == 0)
    # a conjugating (Hermitian-style) chain would be a different, wrong answer here
    assert np.abs(Ab.conj() - grad)[low].max() > 1e-3 * np.abs(grad).max()


def test_complex_selinv_adjoint_central_differences_on_L_and_D():
    """Central differences of the complex loss along the real and the
    imaginary direction of single entries of L and D: for a holomorphic
    function both quotients equal the derivative."""
    p = synth.random_sparse_spd(40, 0.12, 65, complex_values=True)
    sym, L, D, Z = run(p)
    low = oracle.lower_mask(sym)
    W = complex_weights(low, 66)
    Lb, Db = oracle.selinv_adjoint(sym, L, D, Z, W)
    r, c, _ = oracle.panel_entries(sym)
    strict = np.nonzero(r > c)[0]
    rng = np.random.default_rng(67)
    h = 1e-6
    f = lambda LL, DD: complex((W * oracle.selinv(sym, LL, DD))[low].sum())
    for e in rng.choice(strict, size=8, replace=False):
        for step in (h, 1j * h):
            Lp = L.copy(); Lp[e] += step
            Lm = L.copy(); Lm[e] -= step
            fd = (f(Lp, D) - f(Lm, D)) / (2 * step)
            assert abs(fd - Lb[e]) <= 1e-6 * max(1.0, abs(Lb[e]))
    for k in rng.choice(p.n, size=5, replace=False):
        for step in (h, 1j * h):
            Dp = D.copy(); Dp[k] += step
            Dm = D.copy(); Dm[k] -= step
            fd = (f(L, Dp) - f(L, Dm)) / (2 * step)
            assert abs(fd - Db[k]) <= 1e-6 * max(1.0, abs(Db[k]))


def test_complex_ldlt_adjoint_central_differences_on_A():
    """dl/da for single stored entries of a complex symmetric A, through the
    factorization and Alg. 1, by central differences of the whole chain."""
    p = synth.random_sparse_spd(36, 0.15, 68, complex_values=True)
    sym, L, D, Z = run(p)
    low = oracle.lower_mask(sym)
    W = complex_weights(low, 69)
    Lb, Db = oracle.selinv_adjoint(sym, L, D, Z, W)
    Ab = oracle.ldlt_adjoint(sym, L, D, Lb, Db)
    pos = a_positions(sym, p)

    def loss(vals):
        q = synth.problems.Problem(p.name, p.n, p.colptr, p.rowind, vals, p.perm, p.supernodes, p.meta)
        Lq, Dq = oracle.ldlt(q, sym)
        return complex((W * oracle.selinv(sym, Lq, Dq))[low].sum())

    rng = np.random.default_rng(70)
    h = 1e-6
    for k in rng.choice(p.values.size, size=10, replace=False):
        for step in (h, 1j * h):
            vp = p.values.copy(); vp[k] += step
            vm = p.values.copy(); vm[k] -= step
            fd = (loss(vp) - loss(vm)) / (2 * step)
            g = Ab[pos[k]]
            assert abs(fd - g) <= 1e-6 * max(1.0, abs(g))


# ------------------------------------------------- level-parallel oracle

@pytest.mark.parametrize("name,make,herm", [
    ("lap3d-9", lambda: synth.laplacian_3d(9, seed=71), False),
    ("rand-cplx-relaxed", lambda: synth.random_sparse_spd(150, 0.04, 72, complex_values=True,
                                                          supernodes=synth.problems.RELAXED_128), False),
    ("hpd", lambda: synth.random_sparse_hpd(120, 0.05, 73), True),
])
def test_level_parallel_oracle_is_bitwise_serial(name, make, herm):
    """Supernodes of one tree level share no output and read only earlier
    levels: the threaded traversal reproduces the serial one bit for bit,
    for any thread count, and also on a root-side subset."""
    p = make()
    sym = oracle.symbolic_for(p)
    L, D = oracle.ldlt(p, sym)     # the Hermitian factorization for a Hermitian problem
    Z = oracle.selinv(sym, L, D, hermitian=herm)
    for nt in (1, 3, 8):
        Zp = oracle.selinv_levels(sym, L, D, nt, hermitian=herm)
        assert np.array_equal(Zp, Z), (name, nt)
    if not herm:
        kmin = sym.nsuper // 2
        assert np.array_equal(oracle.selinv_levels(sym, L, D, 4, kmin=kmin), oracle.selinv_top(sym, L, D, kmin))
