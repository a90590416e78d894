"""FP64 value oracle: the plain product Y = A X and its iteration (test infrastructure only).

Eq. 1 (Section 3) states A X = sum_i P_{pi_i} (B_i (P_{pi_i}^T X)): an
identity, so the arrow-decomposed product reaches exactly (up to rounding
order) the plain sparse-times-dense product.  That plain product, in FP64, is
the value oracle.  The iteration X_{t+1} = sigma(A X_t) is the one of
Section 2 ("Matrices").  Section 2 leaves sigma to the application; the ones
restated here are the per-column L2 normalisation of power/Lanczos-style runs
(reduced in FP64) and, for the graph-neural-network use the introduction
motivates (a layer applies a non-linearity to A X), the rectifier max(0, y)
and the per-row L2 normalisation.  They compose in one fixed order:
sigma(Y) = column_normalise(row_normalise(relu(Y))), each part optional.

Pinned by tests/test_oracle_spmm.py (closed-form stencil eigenvectors,
row-normalised and GCN-normalised invariants, dense brute force, and the fixed
points and identities of the three sigma parts).
"""
from __future__ import annotations

import numpy as np


def spmm(A, X: np.ndarray) -> np.ndarray:
    """Y = A X in FP64 via scipy's CSR product (Section 2: Y = A X)."""
    S = A.to_scipy()
    return np.asarray(S @ np.asarray(X, dtype=np.float64))


def spmm_dense(A, X: np.ndarray) -> np.ndarray:
    """Brute force Y = A X for tiny n: densify A entry by entry, then a dense product."""
    n = A.n
    D = np.zeros((n, n), dtype=np.float64)
    for r in range(n):
        for j in range(int(A.rowptr[r]), int(A.rowptr[r + 1])):
            D[r, int(A.colidx[j])] += float(A.values[j])
    return D @ np.asarray(X, dtype=np.float64)


def column_normalise(Y: np.ndarray) -> np.ndarray:
    """sigma of Section 2 as used here: divide every column by its FP64 L2 norm."""
    Y = np.asarray(Y, dtype=np.float64)
    norms = np.sqrt(np.sum(Y * Y, axis=0))
    return Y / norms


def relu(Y: np.ndarray) -> np.ndarray:
    """The rectifier applied entry by entry: y if y > 0, else 0."""
    Y = np.asarray(Y, dtype=np.float64)
    return np.where(Y > 0.0, Y, 0.0)


def row_normalise(Y: np.ndarray) -> np.ndarray:
    """Every row divided by its FP64 L2 norm; a row of zeros stays zero."""
    Y = np.asarray(Y, dtype=np.float64)
    norms = np.sqrt(np.sum(Y * Y, axis=1))
    out = np.zeros_like(Y)
    nz = norms > 0.0
    out[nz] = Y[nz] / norms[nz][:, None]
    return out


def iterate(A, X: np.ndarray, iters: int, rescale: bool = False, rectify: bool = False,
            rownorm: bool = False) -> np.ndarray:
    """X_T of X_{t+1} = sigma(A X_t), X_0 = X (Section 2).

    sigma = column_normalise (if ``rescale``) after row_normalise (if ``rownorm``) after
    relu (if ``rectify``); the identity when all are false.  Returns X_T in FP64.
    """
    S = A.to_scipy()
    Y = np.asarray(X, dtype=np.float64)
    for _ in range(iters):
        Y = np.asarray(S @ Y)
        if rectify:
            Y = relu(Y)
        if rownorm:
            Y = row_normalise(Y)
        if rescale:
            Y = column_normalise(Y)
    return Y


def decomposed_product(levels, X: np.ndarray) -> np.ndarray:
    """Eq. 1 written out: Y = sum_i P_{pi_i} (B_i (P_{pi_i}^T X)), in FP64.

    Each level carries ``iperm`` (position -> vertex) and its B_i in CSR over
    positions.  (P^T X)[p] = X[iperm[p]]; P Z puts row p of Z at vertex iperm[p].
    """
    X = np.asarray(X, dtype=np.float64)
    Y = np.zeros_like(X)
    for lv in levels:
        Xp = X[lv.iperm]                      # P_{pi_i}^T X
        Zi = lv.to_scipy() @ Xp               # B_i (P_{pi_i}^T X)
        Yi = np.zeros_like(X)
        Yi[lv.iperm] = Zi                     # P_{pi_i} (...)
        Y += Yi
    return Y


def iterate_rows(A, X: np.ndarray, iters: int, rows: np.ndarray) -> np.ndarray:
    """Rows ``rows`` of A^iters X, exactly, without touching the whole matrix.

    Row s of A^T X depends only on the vertices within T hops of s.  With
    R_j the vertices within j hops of ``rows``, the restriction of A to R_T
    iterated T times is exact on R_{T-t} after t steps, hence on ``rows`` at
    the end.  ``X`` is any object indexable by an int64 array of vertices
    (an ndarray, or a callable returning those rows).
    """
    import scipy.sparse as sp
    S = A.to_scipy()
    cur = np.unique(np.asarray(rows, dtype=np.int64))
    ball = cur
    for _ in range(iters):
        nb = np.unique(S[cur].indices.astype(np.int64))
        cur = np.setdiff1d(nb, ball)
        ball = np.union1d(ball, nb)
    sub = S[ball][:, ball]
    Xb = X(ball) if callable(X) else np.asarray(X)[ball]
    Y = np.asarray(Xb, dtype=np.float64)
    for _ in range(iters):
        Y = np.asarray(sub @ Y)
    pos = np.searchsorted(ball, np.asarray(rows, dtype=np.int64))
    return Y[pos]
