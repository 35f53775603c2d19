"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module only *generates* inputs: sparse symmetric test matrices in CSR form and
the i.i.d. Gaussian start block that Algorithm 8 ("initialize an i.i.d. Gaussian random
matrix X") draws.  It holds none of the eigensolver's arithmetic, so that the CUDA path
and the CPU oracle can both be fed from it without sharing any of the method.

Workloads (the paper's test matrices are not available; these stand in for them, with
comparable n, nnz/n and k):

* ``laplacian_2d(m)`` - 5-point Dirichlet Laplacian on an m x m grid (diag 4, off -1).
* ``laplacian_3d(m)`` - 7-point Dirichlet Laplacian on an m^3 grid (diag 6, off -1).
* ``gaussian_block(n, p, seed)`` - row-major n x p block of N(0,1) samples from a
  counter-based generator (Philox4x32-10, Salmon, Moraes, Dror & Shaw, SC'11) with a
  Box-Muller transform, so any element can be regenerated from (seed, index) alone.

CSR convention everywhere: ``rowptr`` int32[n+1], ``col`` int32[nnz] sorted within each
row, ``val`` float64[nnz]; rows in natural lexicographic grid order.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """A sparse matrix in compressed-sparse-row form (host arrays)."""

    n: int
    rowptr: np.ndarray  # int32[n+1]
    col: np.ndarray  # int32[nnz]
    val: np.ndarray  # float64[nnz] (or float32)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def to_dense(self) -> np.ndarray:
        """Dense copy (small n only)."""
        a = np.zeros((self.n, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        a[rows, self.col] = self.val
        return a


def _stencil_csr(shape: tuple[int, ...], diag: float) -> CSR:
    """Dirichlet nearest-neighbour Laplacian on a tensor grid of the given shape.

    Grid point (i0, i1, ...) maps to row i0 + shape[0]*(i1 + shape[1]*(...)), so
    the first axis is the fastest-varying one.  Every row holds the diagonal plus one
    -1 per in-grid neighbour, columns sorted ascending.
    """
    dims = len(shape)
    n = int(np.prod(shape))
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for s in shape:
        coords.append(rem % s)
        rem //= s
    strides = [int(np.prod(shape[:a])) for a in range(dims)]
    # candidate neighbours in ascending column order: -stride_{d-1} ... -stride_0, self, +stride_0 ...
    offs = []
    for a in reversed(range(dims)):
        offs.append((a, -1))
    offs.append((None, 0))
    for a in range(dims):
        offs.append((a, +1))
    cols = []
    vals = []
    valid = []
    for a, s in offs:
        if a is None:
            cols.append(idx)
            vals.append(np.full(n, diag))
            valid.append(np.ones(n, dtype=bool))
        else:
            c = coords[a] + s
            ok = (c >= 0) & (c < shape[a])
            cols.append(idx + s * strides[a])
            vals.append(np.full(n, -1.0))
            valid.append(ok)
    cols = np.stack(cols, axis=1)
    vals = np.stack(vals, axis=1)
    valid = np.stack(valid, axis=1)
    counts = valid.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    col = cols[valid].astype(np.int32)
    val = vals[valid].astype(np.float64)
    return CSR(n=n, rowptr=rowptr.astype(np.int32), col=col, val=val)


def laplacian_2d(m: int) -> CSR:
    """5-point Dirichlet Laplacian on an m x m grid: n = m^2, nnz = 5m^2 - 4m."""
    return _stencil_csr((m, m), 4.0)


def laplacian_3d(m: int) -> CSR:
    """7-point Dirichlet Laplacian on an m^3 grid: n = m^3, nnz = 7m^3 - 6m^2."""
    return _stencil_csr((m, m, m), 6.0)


# ---------------------------------------------------------------------------------
# Counter-based Gaussian generator (Philox4x32-10 + Box-Muller)
# ---------------------------------------------------------------------------------
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint32(0x9E3779B9)
_PHILOX_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: tuple[int, int]) -> np.ndarray:
    """Philox4x32 with 10 rounds on a batch of 128-bit counters.

    ``ctr`` is uint32[..., 4]; ``key`` two 32-bit words.  Each round multiplies words 0
    and 2 by the two Philox constants (full 64-bit products split into hi/lo halves),
    permutes, and xors the high halves with words 1/3 and the round key; the key is
    bumped by the two Weyl constants between rounds.
    """
    c = [ctr[..., i].astype(np.uint64) for i in range(4)]
    k0 = np.uint32(key[0] & 0xFFFFFFFF)
    k1 = np.uint32(key[1] & 0xFFFFFFFF)
    with np.errstate(over="ignore"):
        for r in range(10):
            if r > 0:
                k0 = np.uint32((int(k0) + int(_PHILOX_W0)) & 0xFFFFFFFF)
                k1 = np.uint32((int(k1) + int(_PHILOX_W1)) & 0xFFFFFFFF)
            p0 = _PHILOX_M0 * c[0]
            p1 = _PHILOX_M1 * c[2]
            hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
            hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
            c = [
                hi1 ^ c[1] ^ np.uint64(k0),
                lo1,
                hi0 ^ c[3] ^ np.uint64(k1),
                lo0,
            ]
    return np.stack([x.astype(np.uint32) for x in c], axis=-1)


def gaussian_from_counter(first: int, count: int, seed: int) -> np.ndarray:
    """N(0,1) samples number ``first`` .. ``first+count-1`` of the stream ``seed``.

    Sample e uses Philox counter (e//2 low word, e//2 high word, 0, 0) and key
    (seed low word, seed high word).  The four output words give two 53-bit uniforms
    u1 in (0,1) and u2 in [0,1); Box-Muller turns them into sqrt(-2 ln u1) * cos(2 pi u2)
    for even e and sqrt(-2 ln u1) * sin(2 pi u2) for odd e.
    """
    if count <= 0:
        return np.zeros(0, dtype=np.float64)
    e0 = first // 2
    e1 = (first + count - 1) // 2 + 1
    pair = np.arange(e0, e1, dtype=np.uint64)
    ctr = np.zeros((pair.shape[0], 4), dtype=np.uint32)
    ctr[:, 0] = (pair & _MASK32).astype(np.uint32)
    ctr[:, 1] = (pair >> np.uint64(32)).astype(np.uint32)
    out = philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)).astype(np.float64)
    two53 = 9007199254740992.0
    u1 = (np.floor(out[:, 0] / 32.0) * 67108864.0 + np.floor(out[:, 1] / 64.0) + 0.5) / two53
    u2 = (np.floor(out[:, 2] / 32.0) * 67108864.0 + np.floor(out[:, 3] / 64.0)) / two53
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * pair.shape[0], dtype=np.float64)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    off = first - 2 * e0
    return z[off:off + count]


def gaussian_block(n: int, p: int, seed: int) -> np.ndarray:
    """Row-major n x p start block, element (i, j) = sample i*p + j of stream ``seed``."""
    return gaussian_from_counter(0, n * p, seed).reshape(n, p)


# ---------------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------------
@dataclass
class Workload:
    """A benchmark / parity problem: matrix, wanted count and solver parameters."""

    name: str
    A: CSR
    k: int
    which: str  # "smallest" | "largest"
    p: int
    q: int
    degree: int
    tol: float
    seed: int


def workload_2d64() -> Workload:
    """2D 64x64 Dirichlet Laplacian, n=4096, nnz=20224; 20 smallest; p=30, d=10, q=1."""
    return Workload("laplace2d_64x64_k20_p30_d10_q1", laplacian_2d(64), 20, "smallest",
                    30, 1, 10, 1e-10, 20150722)


def workload_3d128() -> Workload:
    """3D 128^3 Dirichlet Laplacian, n=2097152, nnz=14581760; 200 smallest; p=240, d=20, q=2."""
    return Workload("laplace3d_128^3_k200_p240_d20_q2", laplacian_3d(128), 200, "smallest",
                    240, 2, 20, 1e-8, 20150723)


def workload_3d(m: int, k: int, p: int, degree: int = 20, q: int = 2, tol: float = 1e-8,
                seed: int = 20150723) -> Workload:
    """Scaled-down member of the 3D Laplacian family (same stencil, smaller grid)."""
    return Workload(f"laplace3d_{m}^3_k{k}_p{p}_d{degree}_q{q}", laplacian_3d(m), k,
                    "smallest", p, q, degree, tol, seed)


# ---------------------------------------------------------------------------------
# Normalised graph Laplacian of a Chung-Lu random graph
# ---------------------------------------------------------------------------------
def chung_lu_weights(n: int, beta: float = 2.5, mean: float = 16.0, wmax: float = 5000.0) -> np.ndarray:
    """Expected degrees w_i = c (i + i0)^(-1/(beta-1)), i = 0..n-1, with c and i0 chosen so
    that the mean is `mean` and the largest (w_0) is `wmax` (bisection on i0)."""
    g = 1.0 / (beta - 1.0)
    i = np.arange(n, dtype=np.float64)

    def mean_for(i0):
        w = (i + i0) ** (-g)
        return wmax * w.mean() / i0 ** (-g)

    lo, hi = 1e-6, 1e12
    for _ in range(200):
        mid = np.sqrt(lo * hi)
        if mean_for(mid) > mean:  # the mean grows with i0
            hi = mid
        else:
            lo = mid
    i0 = np.sqrt(lo * hi)
    return wmax * ((i + i0) / i0) ** (-g)


def chung_lu_laplacian(n: int, seed: int = 1507, beta: float = 2.5, mean: float = 16.0,
                       wmax: float = 5000.0) -> tuple[CSR, np.ndarray]:
    """L = I - D^{-1/2} W D^{-1/2} of the largest connected component of a Chung-Lu graph.

    Edges: about sum(w)/2 endpoint pairs drawn independently with probability proportional
    to w (a pair u != v is then present with probability 1 - exp(-w_u w_v / sum w), the
    expected-degree model); duplicates and self-loops are dropped, the graph is symmetric
    and unweighted.  Values -1/sqrt(d_u d_v) are computed in FP64 with the operands in a
    fixed order and rounded to FP32 once (stored widened to float64).  Returns the CSR
    matrix and the original vertex ids of the component.
    """
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    w = chung_lu_weights(n, beta, mean, wmax)
    S = w.sum()
    rng = np.random.Generator(np.random.Philox(seed))
    m = rng.poisson(S / 2.0)
    cdf = np.cumsum(w / S)
    cdf[-1] = 1.0
    u = np.searchsorted(cdf, rng.random(m), side="right")
    v = np.searchsorted(cdf, rng.random(m), side="right")
    keep = u != v
    u, v = u[keep], v[keep]
    a, b = np.minimum(u, v), np.maximum(u, v)
    key = np.unique(a.astype(np.int64) * n + b)
    a, b = (key // n).astype(np.int64), (key % n).astype(np.int64)
    W = sp.coo_matrix((np.ones(a.size), (a, b)), shape=(n, n)).tocsr()
    W = (W + W.T).tocsr()
    ncomp, lab = connected_components(W, directed=False)
    big = np.argmax(np.bincount(lab))
    ids = np.nonzero(lab == big)[0]
    W = W[ids][:, ids].tocsr()
    W.sort_indices()
    deg = np.asarray(W.sum(axis=1)).ravel()
    rows = np.repeat(np.arange(W.shape[0]), np.diff(W.indptr))
    cols = W.indices
    du, dv = deg[np.minimum(rows, cols)], deg[np.maximum(rows, cols)]
    off = (-1.0 / np.sqrt(du * dv)).astype(np.float32).astype(np.float64)
    nn = W.shape[0]
    L = sp.csr_matrix((off, cols, W.indptr), shape=(nn, nn)) + sp.identity(nn, format="csr")
    L = L.tocsr()
    L.sort_indices()
    return CSR(nn, L.indptr.astype(np.int32), L.indices.astype(np.int32), L.data.astype(np.float64)), ids


def rcm_permuted(A: CSR) -> tuple[CSR, np.ndarray]:
    """P A P^T for the reverse Cuthill-McKee order of A's graph (scipy.sparse.csgraph), the
    locality ordering for matrices whose nonzeros gather rows at random (power-law graphs):
    neighbouring rows then gather nearby rows.  The spectrum is unchanged and eigenvectors
    come back by the returned permutation (row i of the result is row perm[i] of A)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import reverse_cuthill_mckee
    M = sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n))
    perm = reverse_cuthill_mckee(M, symmetric_mode=True).astype(np.int64)
    R = M[perm][:, perm].tocsr()
    R.sort_indices()
    return CSR(A.n, R.indptr.astype(np.int32), R.indices.astype(np.int32), R.data.astype(np.float64)), perm


def diffusion_2d(side: int, seed: int) -> CSR:
    """5-point variable-coefficient diffusion on a side x side grid with Dirichlet ghost
    nodes: every grid edge (interior and boundary) gets a conductance exp(N(0,1))
    (lognormal, mu = 0, sigma = 1); A_ii = sum of the 4 conductances at node i,
    A_ij = -kappa_ij for the interior edge ij.  Symmetric positive definite."""
    rng = np.random.Generator(np.random.Philox(seed))
    kx = np.exp(rng.standard_normal((side + 1, side)))  # edges between x-1 and x, per row y
    ky = np.exp(rng.standard_normal((side, side + 1)))  # edges between y-1 and y, per column x
    n = side * side
    idx = np.arange(n).reshape(side, side)  # [y, x]
    diag = kx[:-1, :].T + kx[1:, :].T + ky[:, :-1].T + ky[:, 1:].T  # [y, x]
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [diag.ravel()]
    # x-neighbours: (y, x) - (y, x+1) through kx[x+1, y]
    rows += [idx[:, :-1].ravel(), idx[:, 1:].ravel()]
    cols += [idx[:, 1:].ravel(), idx[:, :-1].ravel()]
    kxi = -kx[1:-1, :].T.ravel()
    vals += [kxi, kxi]
    # y-neighbours: (y, x) - (y+1, x) through ky[x, y+1]
    rows += [idx[:-1, :].ravel(), idx[1:, :].ravel()]
    cols += [idx[1:, :].ravel(), idx[:-1, :].ravel()]
    kyi = -ky[:, 1:-1].T.ravel()
    vals += [kyi, kyi]
    import scipy.sparse as sp
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    M.sort_indices()
    return CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))


def batched_diffusion_instances(count: int = 256, base_seed: int = 30000, side_range=(32, 512),
                                k_range=(8, 64)) -> list[Workload]:
    """Instance i: side ~ U{side_range}, k ~ U{k_range}, p = round(1.5 k), smallest
    eigenpairs to relative residual 1e-8; the grid and the coefficients come from seed
    base_seed + i."""
    out = []
    for i in range(count):
        rng = np.random.Generator(np.random.Philox(base_seed + i))
        side = int(rng.integers(side_range[0], side_range[1] + 1))
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        p = int(round(1.5 * k))
        A = diffusion_2d(side, base_seed + i)
        out.append(Workload(f"diffusion2d_{side}x{side}_k{k}", A, k, "smallest", p, 1, 10, 1e-8, base_seed + i))
    return out
