"""Seeded synthetic sparse symmetric matrices and their orderings.

Every matrix is returned as the lower triangle (row >= column) of the
symmetrically permuted matrix P A P^T in compressed-sparse-column form, with
the rows of each column ascending (diagonal first).  The permutation is a
geometric nested dissection, the stand-in for the unspecified fill-reducing
ordering the paper applies before its factorization (Sec. IV).

The workloads stand in for the paper's Table I matrices (Sec. IV): 2D/3D mesh
Laplacians for the ND-mesh matrices and a dense-block atomic sheet for the
DFT (DGDFT/SIESTA) matrices.  Nothing here computes any part of the selected
inversion.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "Problem", "grid_nd_order", "laplacian_2d", "laplacian_3d", "dft_sheet",
    "diffusion_3d", "pole_shifts", "batch_laplacians", "random_sparse_spd",
    "tridiagonal", "make_config", "lower_pattern_weights", "random_sparse_hpd",
    "magnetic_laplacian_3d", "random_sparse_nonsym", "symmetric_scaling",
]

FUNDAMENTAL_64 = {"kind": "fundamental", "cap": 64, "fill": 0.0}
RELAXED_128 = {"kind": "relaxed", "cap": 128, "fill": 0.10}


@dataclass
class Problem:
    """A permuted sparse symmetric (or complex symmetric) matrix.

    ``colptr``/``rowind``/``values`` hold the lower triangle of P A P^T (CSC,
    rows ascending, diagonal first).  ``perm[new] = old`` maps a permuted
    index back to the original node.  ``supernodes`` gives the supernode rule
    to use for this workload (kind, column cap, relaxed fill fraction).
    """

    name: str
    n: int
    colptr: np.ndarray
    rowind: np.ndarray
    values: np.ndarray
    perm: np.ndarray
    supernodes: Dict[str, object] = field(default_factory=lambda: dict(FUNDAMENTAL_64))
    meta: Dict[str, object] = field(default_factory=dict)

    @property
    def dtype(self):
        return self.values.dtype

    @property
    def hermitian(self) -> bool:
        """Complex Hermitian (A = A^H; stored lower values, the upper part is
        their conjugate) rather than symmetric."""
        return bool(self.meta.get("hermitian", False))

    @property
    def nnz_lower(self) -> int:
        return int(self.colptr[-1])

    def with_values(self, values: np.ndarray, name: Optional[str] = None) -> "Problem":
        return Problem(name or self.name, self.n, self.colptr, self.rowind, values,
                       self.perm, dict(self.supernodes), dict(self.meta))

    @property
    def nonsymmetric(self) -> bool:
        """Nonsymmetric values on the symmetric pattern: ``meta["upper"]``
        holds a_ji on the positions of the lower CSC."""
        return "upper" in self.meta

    def dense(self) -> np.ndarray:
        """Full dense matrix (small n only)."""
        a = np.zeros((self.n, self.n), dtype=self.values.dtype)
        cols = np.repeat(np.arange(self.n), np.diff(self.colptr))
        if self.nonsymmetric:
            a[cols, self.rowind] = self.meta["upper"]
        else:
            a[cols, self.rowind] = np.conj(self.values) if self.hermitian else self.values
        a[self.rowind, cols] = self.values
        return a

    def diag_positions(self) -> np.ndarray:
        """Index into ``values`` of every diagonal entry (first in its column)."""
        return self.colptr[:-1].copy()


# ---------------------------------------------------------------------------
# assembly of a permuted lower CSC from (old-index) entries
# ---------------------------------------------------------------------------

def _lower_csc(n: int, perm: np.ndarray, diag: np.ndarray, ei: np.ndarray, ej: np.ndarray,
               ev: np.ndarray) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    """Lower CSC of P A P^T from diagonal values and off-diagonal pairs.

    Returns (colptr, rowind, values, src) where ``src[k]`` is the index of the
    input entry that produced stored entry k (diagonal entries are numbered
    0..n-1 by old index, off-diagonals n + pair index).
    """
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n, dtype=np.int64)
    a = iperm[np.asarray(ei, dtype=np.int64)]
    b = iperm[np.asarray(ej, dtype=np.int64)]
    rows = np.concatenate([iperm[np.arange(n)], np.maximum(a, b)])
    cols = np.concatenate([iperm[np.arange(n)], np.minimum(a, b)])
    vals = np.concatenate([np.asarray(diag), np.asarray(ev)])
    src = np.arange(rows.size, dtype=np.int64)
    order = np.lexsort((rows, cols))
    rows, cols, vals, src = rows[order], cols[order], vals[order], src[order]
    key = cols * n + rows
    if np.any(key[1:] == key[:-1]):
        raise ValueError("duplicate entry in the matrix description")
    colptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(colptr, cols + 1, 1)
    colptr = np.cumsum(colptr)
    return colptr, rows.astype(np.int32), vals, src


# ---------------------------------------------------------------------------
# geometric nested dissection on a box grid
# ---------------------------------------------------------------------------

def _lex_ids(lo: Sequence[int], hi: Sequence[int], dims: Sequence[int]) -> np.ndarray:
    """Node ids of the sub-box [lo, hi) in lexicographic order, x fastest."""
    axes = [np.arange(l, h) for l, h in zip(lo, hi)]
    if any(a.size == 0 for a in axes):
        return np.zeros(0, dtype=np.int64)
    mesh = np.meshgrid(*axes[::-1], indexing="ij")  # slowest axis first
    coords = [m.ravel() for m in mesh[::-1]]        # back to x, y, z order
    ids = np.zeros(coords[0].size, dtype=np.int64)
    stride = 1
    for d, c in enumerate(coords):
        ids += c * stride
        stride *= dims[d]
    return ids


def grid_nd_order(dims: Sequence[int], leaf: int = 32) -> np.ndarray:
    """Nested-dissection order of a box grid (x fastest node numbering).

    Recursive bisection along the longest extent (ties: x, then y, then z);
    the separator is the plane at ``lo + len // 2``; the order is left half,
    right half, separator.  Recursion stops at ``<= leaf`` nodes or when the
    longest extent is below 3; leaves and separators are numbered
    lexicographically with x fastest.  Returns ``perm`` with perm[new] = old.
    """
    dims = list(dims)
    out: List[np.ndarray] = []

    def rec(lo, hi):
        lens = [h - l for l, h in zip(lo, hi)]
        count = int(np.prod(lens))
        if count == 0:
            return
        if count <= leaf or max(lens) < 3:
            out.append(_lex_ids(lo, hi, dims))
            return
        d = int(np.argmax(lens))  # first maximum: x before y before z
        mid = lo[d] + lens[d] // 2
        lhi = list(hi); lhi[d] = mid
        rlo = list(lo); rlo[d] = mid + 1
        slo = list(lo); slo[d] = mid
        shi = list(hi); shi[d] = mid + 1
        rec(list(lo), lhi)
        rec(rlo, list(hi))
        out.append(_lex_ids(slo, shi, dims))

    rec([0] * len(dims), dims)
    perm = np.concatenate(out)
    assert perm.size == int(np.prod(dims)) and np.unique(perm).size == perm.size
    return perm


def _grid_edges(dims: Sequence[int]) -> Tuple[np.ndarray, np.ndarray]:
    """All nearest-neighbour pairs (i, j), j = i + stride_d, in a fixed order."""
    n = int(np.prod(dims))
    ids = np.arange(n, dtype=np.int64)
    coords = []
    rem = ids.copy()
    for d in dims:
        coords.append(rem % d)
        rem //= d
    ei, ej = [], []
    stride = 1
    for d, dim in enumerate(dims):
        m = coords[d] < dim - 1
        ei.append(ids[m])
        ej.append(ids[m] + stride)
        stride *= dim
    return np.concatenate(ei), np.concatenate(ej)


def laplacian_2d(nx: int, ny: Optional[int] = None, shift: float = 0.1,
                 name: Optional[str] = None) -> Problem:
    """2D 5-point Laplacian (diagonal 4 + shift, off-diagonal -1, Dirichlet)."""
    ny = nx if ny is None else ny
    dims = (nx, ny)
    n = nx * ny
    perm = grid_nd_order(dims)
    ei, ej = _grid_edges(dims)
    colptr, rowind, vals, _ = _lower_csc(n, perm, np.full(n, 4.0 + shift), ei, ej,
                                         np.full(ei.size, -1.0))
    return Problem(name or f"lap2d_{nx}x{ny}", n, colptr, rowind, vals.astype(np.float64), perm,
                   dict(FUNDAMENTAL_64), {"dims": dims, "shift": shift})


def laplacian_3d(nx: int, seed: int, name: Optional[str] = None,
                 supernodes: Optional[Dict[str, object]] = None, shift: float = 0.0) -> Problem:
    """3D 7-point Laplacian, diagonal 6 + shift + U(0,1) (seeded, by original
    node id).  A large shift makes A^{-1} decay fast away from the diagonal."""
    dims = (nx, nx, nx)
    n = nx ** 3
    rng = np.random.default_rng(seed)
    diag = 6.0 + shift + rng.uniform(0.0, 1.0, n)
    perm = grid_nd_order(dims)
    ei, ej = _grid_edges(dims)
    colptr, rowind, vals, _ = _lower_csc(n, perm, diag, ei, ej, np.full(ei.size, -1.0))
    return Problem(name or f"lap3d_{nx}", n, colptr, rowind, vals.astype(np.float64), perm,
                   dict(supernodes or RELAXED_128), {"dims": dims, "seed": seed, "shift": shift})


# ---------------------------------------------------------------------------
# DFT-like complex symmetric sheet (dense 16 x 16 atom blocks)
# ---------------------------------------------------------------------------

def _atom_nd(pos: np.ndarray, nbrs: List[np.ndarray], leaf: int = 4) -> np.ndarray:
    """Coordinate-bisection nested dissection over atoms.

    Split at the median of the longest extent (stable sort by coordinate,
    then atom id); separator = atoms of the left half with a neighbour in the
    right half; leaves hold <= ``leaf`` atoms; leaves and separators are
    numbered by ascending atom id.  Order: left, right, separator.
    """
    natoms = pos.shape[0]
    in_right = np.zeros(natoms, dtype=bool)
    out: List[np.ndarray] = []

    def rec(ids: np.ndarray):
        if ids.size == 0:
            return
        if ids.size <= leaf:
            out.append(np.sort(ids))
            return
        ext = pos[ids].max(axis=0) - pos[ids].min(axis=0)
        d = int(np.argmax(ext))
        order = np.lexsort((ids, pos[ids, d]))
        srt = ids[order]
        half = srt.size // 2
        left, right = srt[:half], srt[half:]
        in_right[right] = True
        sep_mask = np.array([bool(in_right[nbrs[a]].any()) for a in left], dtype=bool)
        in_right[right] = False
        sep = np.sort(left[sep_mask])
        rest = left[~sep_mask]
        rec(rest)
        rec(right)
        if sep.size:
            out.append(sep)

    rec(np.arange(natoms, dtype=np.int64))
    order = np.concatenate(out)
    assert np.unique(order).size == natoms
    return order


def dft_sheet(side: int = 32, nbasis: int = 16, cutoff: float = 2.5,
              z: complex = complex(-0.2, 0.05), seed: int = 3) -> Problem:
    """Complex symmetric A = H - z S on a jittered 2D atomic lattice.

    H: dense nbasis x nbasis blocks N(0,1) exp(-r) between atoms within
    ``cutoff`` lattice units (H_JI = H_IJ^T), symmetric on-site blocks (r=0).
    S = I + 0.1 B, B with H's block pattern, off-diagonal N(0,1) exp(-r),
    symmetric, diagonal = row sum of |off-diagonal| + 1, scaled by
    1 / max row sum.  Draw order: jitter, H on-site, H pairs, B on-site, B pairs.
    """
    rng = np.random.default_rng(seed)
    natoms = side * side
    ix, iy = np.meshgrid(np.arange(side), np.arange(side), indexing="xy")
    base = np.stack([ix.ravel(), iy.ravel()], axis=1).astype(np.float64)  # id = ix + side*iy
    pos = base + rng.uniform(-0.1, 0.1, size=(natoms, 2))
    diff = pos[:, None, :] - pos[None, :, :]
    dist = np.sqrt((diff ** 2).sum(-1))
    ii, jj = np.nonzero(np.triu(dist <= cutoff, k=1))
    r = dist[ii, jj]
    npair = ii.size
    nb = nbasis
    tri = np.triu_indices(nb)
    # H on-site blocks: symmetric, upper triangle drawn
    h_on = np.zeros((natoms, nb, nb))
    draws = rng.standard_normal((natoms, tri[0].size))
    h_on[:, tri[0], tri[1]] = draws
    h_on[:, tri[1], tri[0]] = draws
    h_off = rng.standard_normal((npair, nb, nb)) * np.exp(-r)[:, None, None]
    # B on-site off-diagonal entries (strict upper drawn), B pair blocks
    stri = np.triu_indices(nb, k=1)
    b_on = np.zeros((natoms, nb, nb))
    draws = rng.standard_normal((natoms, stri[0].size))
    b_on[:, stri[0], stri[1]] = draws
    b_on[:, stri[1], stri[0]] = draws
    b_off = rng.standard_normal((npair, nb, nb)) * np.exp(-r)[:, None, None]
    # row sums of |B| off-diagonal part, per (atom, basis)
    rowsum = np.abs(b_on).sum(axis=2)
    np.add.at(rowsum, ii, np.abs(b_off).sum(axis=2))
    np.add.at(rowsum, jj, np.abs(b_off).sum(axis=1))
    b_diag = rowsum + 1.0
    scale = 1.0 / float((rowsum + b_diag).max())
    n = natoms * nb
    # atom ordering, expanded to basis functions
    nbrs: List[List[int]] = [[] for _ in range(natoms)]
    for a, b in zip(ii, jj):
        nbrs[a].append(b); nbrs[b].append(a)
    nbrs_arr = [np.array(x, dtype=np.int64) for x in nbrs]
    aorder = _atom_nd(pos, nbrs_arr)
    perm = (aorder[:, None] * nb + np.arange(nb)[None, :]).ravel()
    # entries (old indices): on-site strict lower, pair blocks, diagonal
    zc = complex(z)
    s_on = 0.1 * scale * b_on
    a_on = h_on - zc * s_on
    a_diag = np.array([a_on[a].diagonal() for a in range(natoms)])  # h_ii - z*0 (s_on diag = 0)
    a_diag = a_diag - zc * (1.0 + 0.1 * scale * b_diag)
    sl = np.tril_indices(nb, k=-1)
    on_i = (np.arange(natoms)[:, None] * nb + sl[0][None, :]).ravel()
    on_j = (np.arange(natoms)[:, None] * nb + sl[1][None, :]).ravel()
    on_v = a_on[:, sl[0], sl[1]].ravel()
    a_off = h_off - zc * 0.1 * scale * b_off            # rows of atom ii, cols of atom jj
    pi = (ii[:, None, None] * nb + np.arange(nb)[None, :, None]) * np.ones((1, 1, nb), dtype=np.int64)
    pj = (jj[:, None, None] * nb + np.arange(nb)[None, None, :]) * np.ones((1, nb, 1), dtype=np.int64)
    ei = np.concatenate([on_i, pi.ravel()])
    ej = np.concatenate([on_j, pj.ravel()])
    ev = np.concatenate([on_v, a_off.ravel()])
    diag_old = a_diag.ravel()
    colptr, rowind, vals, _ = _lower_csc(n, perm, diag_old, ei, ej, ev)
    return Problem(f"dft_sheet_{natoms}x{nb}", n, colptr, rowind, vals.astype(np.complex128), perm,
                   dict(FUNDAMENTAL_64),
                   {"natoms": natoms, "nbasis": nb, "cutoff": cutoff, "z": zc, "seed": seed,
                    "npairs": int(npair)})


# ---------------------------------------------------------------------------
# 3D variable-coefficient diffusion (parameters: edge conductances)
# ---------------------------------------------------------------------------

def diffusion_3d(nx: int = 24, seed: int = 5, sigma: float = 0.5,
                 theta: Optional[np.ndarray] = None) -> Problem:
    """A = sum_e theta_e u_e u_e^T over grid edges and Dirichlet ghost edges.

    Interior edge (i, j): u_e = e_i - e_j.  Ghost edge at boundary node i:
    u_e = e_i (six faces, order -x, +x, -y, +y, -z, +z).  theta_e =
    exp(sigma N(0,1)) drawn in edge order (interior, then ghost).  ``meta``
    carries the edge list and an assembly map (stored entry, edge, sign) so
    that values = sum over the map of sign * theta[edge].
    """
    dims = (nx, nx, nx)
    n = nx ** 3
    ei, ej = _grid_edges(dims)
    ids = np.arange(n, dtype=np.int64)
    cx, cy, cz = ids % nx, (ids // nx) % nx, ids // (nx * nx)
    ghosts = np.concatenate([ids[cx == 0], ids[cx == nx - 1], ids[cy == 0], ids[cy == nx - 1],
                             ids[cz == 0], ids[cz == nx - 1]])
    nint, ngh = ei.size, ghosts.size
    if theta is None:
        rng = np.random.default_rng(seed)
        theta = np.exp(sigma * rng.standard_normal(nint + ngh))
    theta = np.asarray(theta, dtype=np.float64)
    perm = grid_nd_order(dims)
    colptr, rowind, _, src = _lower_csc(n, perm, np.zeros(n), ei, ej, np.zeros(nint))
    # stored position of each input entry
    pos_of_src = np.empty(src.size, dtype=np.int64)
    pos_of_src[src] = np.arange(src.size)
    diag_pos = pos_of_src[:n]          # by old node id
    off_pos = pos_of_src[n:]           # by interior edge
    m_entry = np.concatenate([diag_pos[ei], diag_pos[ej], off_pos, diag_pos[ghosts]])
    m_edge = np.concatenate([np.arange(nint), np.arange(nint), np.arange(nint),
                             nint + np.arange(ngh)])
    m_sign = np.concatenate([np.ones(nint), np.ones(nint), -np.ones(nint), np.ones(ngh)])
    vals = np.zeros(colptr[-1])
    np.add.at(vals, m_entry, m_sign * theta[m_edge])
    meta = {"dims": dims, "seed": seed, "edges_i": ei, "edges_j": ej, "ghosts": ghosts,
            "theta": theta, "asm_entry": m_entry, "asm_edge": m_edge, "asm_sign": m_sign}
    return Problem(f"diffusion3d_{nx}", n, colptr, rowind, vals, perm, dict(RELAXED_128), meta)


def lower_pattern_weights(nnz: int, seed: int = 5) -> np.ndarray:
    """Loss weights W ~ N(0,1), one per stored lower entry of the L pattern."""
    return np.random.default_rng(1000 + seed).standard_normal(nnz)


# ---------------------------------------------------------------------------
# batches: pole shifts on one pattern, uneven Laplacians
# ---------------------------------------------------------------------------

def pole_shifts(npoles: int = 40, seed: int = 4) -> Tuple[np.ndarray, np.ndarray]:
    """Pole shifts z_l = E_l + i eta_l, E_l ~ U(-1,1), eta_l log-spaced 1e-3..1e-1."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(-1.0, 1.0, npoles)
    eta = np.logspace(-3, -1, npoles)
    return e, eta


def shifted_values(base: Problem, z: complex) -> np.ndarray:
    """Values of base - z I on base's stored pattern (complex128)."""
    v = base.values.astype(np.complex128)
    v[base.diag_positions()] -= z
    return v


def batch_laplacians(scale: float = 1.0) -> List[Problem]:
    """Eight uneven Laplacians: 2D 45^2, 100^2, 160^2, 245^2 (+0.1 shift) and
    3D 13^3, 22^3, 30^3, 39^3 (diagonal 6 + U(0,1), seeds 41..44).

    ``scale`` < 1 shrinks every side (for quick tests)."""
    out = []
    for k in (45, 100, 160, 245):
        m = max(3, int(round(k * scale)))
        out.append(laplacian_2d(m))
    for t, k in enumerate((13, 22, 30, 39)):
        m = max(3, int(round(k * scale)))
        out.append(laplacian_3d(m, seed=41 + t))
    return out


# ---------------------------------------------------------------------------
# small test matrices
# ---------------------------------------------------------------------------

def tridiagonal(n: int, diag: float = 2.0, off: float = -1.0, nd: bool = False) -> Problem:
    """tridiag(off, diag, off) in natural order, or a 1D nested-dissection order."""
    perm = grid_nd_order((n,), leaf=1) if nd else np.arange(n)
    ei = np.arange(n - 1)
    colptr, rowind, vals, _ = _lower_csc(n, perm, np.full(n, diag), ei, ei + 1,
                                         np.full(n - 1, off))
    return Problem(f"tridiag_{n}{'_nd' if nd else ''}", n, colptr, rowind, vals.astype(np.float64),
                   perm, dict(FUNDAMENTAL_64), {})


def random_sparse_spd(n: int, density: float, seed: int, complex_values: bool = False,
                      supernodes: Optional[Dict[str, object]] = None,
                      permute: bool = True) -> Problem:
    """Random symmetric pattern with diagonally dominant values.

    Off-diagonal values N(0,1) (complex: real and imaginary parts N(0,1));
    diagonal = row sum of |off-diagonal| + 1 (+ 1i for complex), so that the
    no-pivot LDL^T exists.  ``permute`` applies a random symmetric permutation.
    """
    rng = np.random.default_rng(seed)
    m = int(round(density * n * (n - 1) / 2))
    iu = rng.choice(n * (n - 1) // 2, size=min(m, n * (n - 1) // 2), replace=False)
    # map linear index of strict upper triangle to (i, j)
    iu = np.sort(iu)
    r = np.floor((np.sqrt(8.0 * iu + 1) - 1) / 2).astype(np.int64) + 1
    c = iu - r * (r - 1) // 2
    ei, ej = r, c                      # ei > ej
    if complex_values:
        ev = rng.standard_normal(ei.size) + 1j * rng.standard_normal(ei.size)
    else:
        ev = rng.standard_normal(ei.size)
    rs = np.zeros(n)
    np.add.at(rs, ei, np.abs(ev)); np.add.at(rs, ej, np.abs(ev))
    diag = rs + 1.0 + (1j if complex_values else 0.0)
    perm = rng.permutation(n) if permute else np.arange(n)
    colptr, rowind, vals, _ = _lower_csc(n, perm, diag, ei, ej, ev)
    dt = np.complex128 if complex_values else np.float64
    return Problem(f"rand_{n}_{seed}", n, colptr, rowind, vals.astype(dt), perm,
                   dict(supernodes or FUNDAMENTAL_64), {"seed": seed})


def _hermitian_lower(n: int, perm: np.ndarray, diag: np.ndarray, ei: np.ndarray, ej: np.ndarray,
                     ev: np.ndarray):
    """Lower CSC of P A P^T for a Hermitian A given A[ei, ej] = ev (old
    indices): the stored lower entry is ev where ei lands below ej after the
    permutation, conj(ev) where it lands above."""
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n, dtype=np.int64)
    ev = np.where(iperm[ei] > iperm[ej], ev, np.conj(ev))
    return _lower_csc(n, perm, diag, ei, ej, ev)


def symmetric_scaling(p: Problem, decades: float, seed: int) -> Problem:
    """S A S with S = diag(10^u), u ~ U(-decades/4, decades/4) per original
    node: still symmetric (positive definite if A is), its diagonal spread
    over about `decades` orders of magnitude, and the entries of A^{-1}
    (= S^{-1} A^{-1} S^{-1}) spread over as many within each row."""
    rng = np.random.default_rng(seed)
    u = 10.0 ** rng.uniform(-decades / 4.0, decades / 4.0, p.n)
    sc = u[p.perm]                                  # by permuted index
    cols = np.repeat(np.arange(p.n), np.diff(p.colptr))
    vals = p.values * sc[p.rowind] * sc[cols]
    meta = dict(p.meta)
    meta["scaling_decades"] = decades
    return Problem(p.name + f"_scaled{decades:g}", p.n, p.colptr, p.rowind, vals, p.perm,
                   dict(p.supernodes), meta)


def random_sparse_hpd(n: int, density: float, seed: int,
                      supernodes: Optional[Dict[str, object]] = None) -> Problem:
    """Random Hermitian positive definite matrix: off-diagonal entries with
    real and imaginary parts N(0,1), real diagonal = row sum of |off-diagonal|
    + 1, a random symmetric permutation."""
    rng = np.random.default_rng(seed)
    m = int(round(density * n * (n - 1) / 2))
    iu = np.sort(rng.choice(n * (n - 1) // 2, size=min(m, n * (n - 1) // 2), replace=False))
    r = np.floor((np.sqrt(8.0 * iu + 1) - 1) / 2).astype(np.int64) + 1
    c = iu - r * (r - 1) // 2
    ev = rng.standard_normal(r.size) + 1j * rng.standard_normal(r.size)
    rs = np.zeros(n)
    np.add.at(rs, r, np.abs(ev)); np.add.at(rs, c, np.abs(ev))
    perm = rng.permutation(n)
    colptr, rowind, vals, _ = _hermitian_lower(n, perm, rs + 1.0, r, c, ev)
    return Problem(f"hpd_{n}_{seed}", n, colptr, rowind, vals.astype(np.complex128), perm,
                   dict(supernodes or FUNDAMENTAL_64), {"seed": seed, "hermitian": True})


def random_sparse_nonsym(n: int, density: float, seed: int, complex_values: bool = False,
                         supernodes: Optional[Dict[str, object]] = None) -> Problem:
    """Random symmetric pattern with independent values above and below the
    diagonal (N(0,1); complex: both parts), diagonal = sum of |a_ij| + |a_ji|
    over the row + 1 (diagonally dominant by rows and columns: LU without
    pivoting exists), a random symmetric permutation."""
    rng = np.random.default_rng(seed)
    m = int(round(density * n * (n - 1) / 2))
    iu = np.sort(rng.choice(n * (n - 1) // 2, size=min(m, n * (n - 1) // 2), replace=False))
    r = np.floor((np.sqrt(8.0 * iu + 1) - 1) / 2).astype(np.int64) + 1
    c = iu - r * (r - 1) // 2
    if complex_values:
        draw = lambda k: rng.standard_normal(k) + 1j * rng.standard_normal(k)
    else:
        draw = rng.standard_normal
    below, above = draw(r.size), draw(r.size)       # A[r, c] and A[c, r]
    rs = np.zeros(n)
    for v in (below, above):
        np.add.at(rs, r, np.abs(v))
        np.add.at(rs, c, np.abs(v))
    diag = rs + 1.0
    perm = rng.permutation(n)
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    low_first = iperm[r] > iperm[c]                  # A[r, c] lands below the diagonal
    lo_in = np.where(low_first, below, above)
    up_in = np.where(low_first, above, below)
    colptr, rowind, vals, src = _lower_csc(n, perm, diag, r, c, lo_in)
    up_all = np.concatenate([diag, up_in])
    dt = np.complex128 if complex_values else np.float64
    return Problem(f"nonsym_{n}_{seed}", n, colptr, rowind, vals.astype(dt), perm,
                   dict(supernodes or FUNDAMENTAL_64), {"seed": seed, "upper": up_all[src].astype(dt)})


def magnetic_laplacian_3d(nx: int, seed: int, flux: float = 0.25,
                          supernodes: Optional[Dict[str, object]] = None) -> Problem:
    """3D 7-point Laplacian with complex hopping -exp(i theta_e) on every edge
    (theta_e = 2 pi flux U(-1, 1), a random magnetic-phase field), diagonal
    6 + U(0,1): Hermitian positive definite, nested-dissection order."""
    dims = (nx, nx, nx)
    n = nx ** 3
    rng = np.random.default_rng(seed)
    diag = 6.0 + rng.uniform(0.0, 1.0, n)
    perm = grid_nd_order(dims)
    ei, ej = _grid_edges(dims)
    theta = 2.0 * np.pi * flux * rng.uniform(-1.0, 1.0, ei.size)
    colptr, rowind, vals, _ = _hermitian_lower(n, perm, diag, ei, ej, -np.exp(1j * theta))
    return Problem(f"maglap3d_{nx}", n, colptr, rowind, vals.astype(np.complex128), perm,
                   dict(supernodes or RELAXED_128), {"dims": dims, "seed": seed, "hermitian": True})


# ---------------------------------------------------------------------------
# the five configured workloads
# ---------------------------------------------------------------------------

def make_config(i: int) -> Problem:
    """Workload i (1..5).

    1: 2D 5-point Laplacian 63x63 + 0.1 I, f64, fundamental supernodes <= 64.
    2: 3D 7-point Laplacian 40^3, diagonal 6 + U(0,1), relaxed supernodes
       (<= 128 columns, <= 10% explicit zeros).
    3: DFT-like complex symmetric sheet, 1024 atoms x 16, c128, fundamental <= 64.
    4: the pattern of 2 with pole shifts (see ``pole_shifts``) -- returns the
       base problem; the shifts and the extra Laplacians come separately.
    5: 3D variable-coefficient diffusion 24^3, relaxed supernodes.
    """
    if i == 1:
        return laplacian_2d(63, shift=0.1, name="cfg1_lap2d_63")
    if i == 2:
        return laplacian_3d(40, seed=2, name="cfg2_lap3d_40")
    if i == 3:
        return dft_sheet()
    if i == 4:
        return laplacian_3d(40, seed=2, name="cfg4_base_lap3d_40")
    if i == 5:
        return diffusion_3d(24, seed=5)
    raise ValueError(f"no workload {i}")
