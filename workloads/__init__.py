"""Seeded synthetic inputs for the arrow-decomposition SpMM.

This module only *generates* inputs: sparse matrices with the structure of
the paper's workloads (bounded-degree meshes standing in for OSM Europe /
GenBank, power-law graphs standing in for GAP-twitter / WebBase / sk-2005,
random-geometric graphs for the batched workload) and dense feature blocks.
It holds none of the method's arithmetic (no decomposition, no product), so
both the oracle and the CUDA path may import it.

Every matrix is returned as a :class:`Csr` with int64 row pointers, int32
column indices sorted strictly ascending inside each row, and float64 values.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Csr:
    n: int
    rowptr: np.ndarray  # int64[n+1]
    colidx: np.ndarray  # int32[nnz]
    values: np.ndarray  # float64[nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.values, self.colidx, self.rowptr), shape=(self.n, self.n))


def _round_values(vals: np.ndarray, round_to) -> np.ndarray:
    if round_to is None:
        return vals
    return vals.astype(round_to).astype(np.float64)


def _row_of_entry(rowptr: np.ndarray) -> np.ndarray:
    n = rowptr.shape[0] - 1
    counts = np.diff(rowptr)
    return np.repeat(np.arange(n, dtype=np.int64), counts)


def row_normalise(rowptr: np.ndarray, vals: np.ndarray) -> np.ndarray:
    """Divide each row by its sum (input recipe: 'values ... row-normalised')."""
    sums = np.add.reduceat(vals, rowptr[:-1]) if vals.size else np.zeros(0)
    empty = rowptr[1:] == rowptr[:-1]
    sums = np.where(empty, 1.0, sums)
    return vals / np.repeat(sums, np.diff(rowptr))


def grid_stencil(dims, seed: int | None = 1, value_range=(0.5, 1.5), row_normalised=True,
                 round_to=np.float32, unit_weights=False, diag_value=None) -> Csr:
    """2D 5-point / 3D 7-point stencil adjacency on a Dirichlet grid, diagonal included.

    ``dims`` is (N0, N1) or (N0, N1, N2); vertex id = row-major index (last
    axis fastest).  With ``unit_weights`` every off-diagonal entry is 1 and the
    diagonal is ``diag_value`` (the textbook Laplacian-type stencil used for
    closed-form eigenvector checks); otherwise values are U(value_range) drawn
    from numpy PCG64(seed) in CSR order, then optionally row-normalised and
    rounded to ``round_to`` (float32 by default, the workloads' storage type).
    """
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    strides = []
    s = 1
    for d in reversed(dims):
        strides.append(s)
        s *= d
    strides = list(reversed(strides))  # stride of each axis
    # candidate offsets in ascending column order: -s0, -s1, ..., -1, 0, +1, ..., +s0
    neg = [(ax, -1) for ax in range(len(dims))]          # -s0 < -s1 < ... (s0 largest)
    pos = [(ax, +1) for ax in reversed(range(len(dims)))]  # +last < ... < +s0
    offs = neg + [(None, 0)] + pos
    v = np.arange(n, dtype=np.int64)
    coords = []
    rem = v.copy()
    for ax in range(len(dims)):
        coords.append(rem // strides[ax])
        rem = rem % strides[ax]
    cand = np.empty((n, len(offs)), dtype=np.int32)
    mask = np.empty((n, len(offs)), dtype=bool)
    for j, (ax, sgn) in enumerate(offs):
        if ax is None:
            cand[:, j] = v
            mask[:, j] = True
        else:
            c = coords[ax] + sgn
            ok = (c >= 0) & (c < dims[ax])
            cand[:, j] = v + sgn * strides[ax]
            mask[:, j] = ok
    del coords, rem
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colidx = cand[mask]
    is_diag = (np.broadcast_to(np.arange(len(offs)) == len(dims), mask.shape))[mask]
    del cand, mask
    if unit_weights:
        vals = np.ones(colidx.shape[0], dtype=np.float64)
        if diag_value is not None:
            vals[is_diag] = float(diag_value)
        return Csr(n, rowptr, colidx, vals)
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = value_range
    vals = lo + (hi - lo) * rng.random(colidx.shape[0])
    if row_normalised:
        vals = row_normalise(rowptr, vals)
    return Csr(n, rowptr, colidx, _round_values(vals, round_to))


def _sorted_unique(a: np.ndarray) -> np.ndarray:
    """np.unique of a 1-D integer array by sort + neighbour test (the same result; np.unique's
    own path is far slower on arrays of hundreds of millions of keys)."""
    a = np.sort(a)
    if a.size < 2:
        return a
    m = np.empty(a.size, dtype=bool)
    m[0] = True
    np.not_equal(a[1:], a[:-1], out=m[1:])
    return a[m]


def _csr_from_pairs(n: int, rows: np.ndarray, cols: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Pattern CSR (rowptr int64, colidx int32) from (row, col) pairs; duplicates removed."""
    key = rows.astype(np.int64) * n + cols.astype(np.int64)
    key = _sorted_unique(key)
    r = key // n
    c = (key % n).astype(np.int32)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=rowptr[1:])
    return rowptr, c


def rmat_edges(scale: int, edge_factor: int, abcd=(0.57, 0.19, 0.19, 0.05), seed: int = 5):
    """R-MAT edge list (Chakrabarti et al.): ``edge_factor * 2**scale`` directed edges.

    Each edge picks one quadrant per bit level with probabilities (a, b, c, d);
    uniform draws come from PCG64(seed), one float32 array per level.
    """
    a, b, c, d = abcd
    n = 1 << scale
    m = edge_factor * n
    rng = np.random.Generator(np.random.PCG64(seed))
    wide = np.int64 if scale > 31 else np.uint32
    u = np.zeros(m, dtype=wide)
    v = np.zeros(m, dtype=wide)
    ab = a + b
    abc = a + b + c
    for lvl in range(scale):
        r = rng.random(m, dtype=np.float32)
        bit = wide(1 << (scale - 1 - lvl))
        # quadrant: [0,a) -> (0,0); [a,a+b) -> (0,1); [a+b,a+b+c) -> (1,0); else (1,1)
        row_bit = r >= ab
        col_bit = ((r >= a) & (r < ab)) | (r >= abc)
        u += row_bit * bit
        v += col_bit * bit
    return n, u.astype(np.int64), v.astype(np.int64)


def rmat_gcn(scale: int, edge_factor: int = 16, abcd=(0.57, 0.19, 0.19, 0.05), seed: int = 5,
             round_to=None) -> Csr:
    """Symmetrised R-MAT graph with self-loops, GCN-normalised D^-1/2 (A+I) D^-1/2.

    Directed edges are symmetrised and deduplicated, self-loops of the draw are
    dropped and one self-loop per vertex added; d_v is the number of entries
    in row v of A+I and entry (u, v) gets 1/sqrt(d_u d_v).
    """
    n, u, v = rmat_edges(scale, edge_factor, abcd, seed)
    keep = u != v
    u, v = u[keep], v[keep]
    ar = np.arange(n, dtype=np.int64)
    rows = np.concatenate([u, v, ar])
    cols = np.concatenate([v, u, ar])
    del u, v
    rowptr, colidx = _csr_from_pairs(n, rows, cols)
    del rows, cols
    deg = np.diff(rowptr).astype(np.float64)
    rs = 1.0 / np.sqrt(deg)
    vals = rs[_row_of_entry(rowptr)] * rs[colidx]
    return Csr(n, rowptr, colidx, _round_values(vals, round_to))


def rgg(n: int, seed: int, mean_degree: float = 8.0, value_range=(0.5, 1.5),
        row_normalised=True, round_to=np.float16) -> Csr:
    """2D random-geometric graph: n points U[0,1]^2, edge when distance < r.

    r = sqrt(mean_degree / (pi n)) gives the stated mean degree away from the
    boundary.  Self-loops added; values U(value_range) from PCG64(seed+1)
    row-normalised, rounded to ``round_to`` (float16 by default).
    """
    from scipy.spatial import cKDTree
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = rng.random((n, 2))
    r = math.sqrt(mean_degree / (math.pi * n))
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray").astype(np.int64)
    ar = np.arange(n, dtype=np.int64)
    rows = np.concatenate([pairs[:, 0], pairs[:, 1], ar])
    cols = np.concatenate([pairs[:, 1], pairs[:, 0], ar])
    rowptr, colidx = _csr_from_pairs(n, rows, cols)
    vrng = np.random.Generator(np.random.PCG64(seed + 1))
    lo, hi = value_range
    vals = lo + (hi - lo) * vrng.random(colidx.shape[0])
    if row_normalised:
        vals = row_normalise(rowptr, vals)
    return Csr(n, rowptr, colidx, _round_values(vals, round_to))


def random_csr(n: int, density: float, seed: int, symmetric=False, diag=False) -> Csr:
    """Uniform random sparsity pattern with U(-1, 1) values (small test matrices)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = max(1, int(density * n * n))
    r = rng.integers(0, n, m)
    c = rng.integers(0, n, m)
    if symmetric:
        r, c = np.concatenate([r, c]), np.concatenate([c, r])
    if diag:
        ar = np.arange(n)
        r, c = np.concatenate([r, ar]), np.concatenate([c, ar])
    rowptr, colidx = _csr_from_pairs(n, r, c)
    vals = rng.uniform(-1.0, 1.0, colidx.shape[0])
    return Csr(n, rowptr, colidx, vals)


def features(n: int, k: int, seed: int, dtype=np.float32) -> np.ndarray:
    """Dense n x k feature block, N(0, 1) from PCG64(seed), row-major, cast to ``dtype``.

    For 16-bit types the float32 draw is rounded by the caller's tensor
    library (round-to-nearest-even); this returns float32 in that case.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.standard_normal((n, k), dtype=np.float32)
    if dtype in (np.float32, "float32"):
        return x
    if dtype in (np.float64, "float64"):
        return x.astype(np.float64)
    return x


# Named workloads with the shapes of the paper's inputs (full size and a
# scaled-down twin that the oracle finishes in seconds).
def grid2d_64(seed=1) -> Csr:
    """2D 64x64 grid, 5-point stencil (n=4096, nnz=20,224), U(0.5,1.5) row-normalised f32."""
    return grid_stencil((64, 64), seed=seed)


def grid3d(N: int, seed=3) -> Csr:
    """3D NxNxN grid, 7-point stencil, U(0.5,1.5) row-normalised f32 (N=400: n=64M)."""
    return grid_stencil((N, N, N), seed=seed)


def log_uniform_sizes(count: int, lo: float, hi: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(rng.uniform(math.log(lo), math.log(hi), count)).astype(np.int64)
