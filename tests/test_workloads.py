"""CPU tests of the seeded input generators (workloads/): structure the recipes promise.

The generators hold none of the method's arithmetic; these tests check that the inputs
have the stated shape (sorted, duplicate-free CSR, symmetric patterns, self-loops, degree
and normalisation rules) and that the fast dedupe equals np.unique.
"""
import numpy as np
import pytest

import workloads as w


def _check_csr(A):
    assert A.rowptr.dtype == np.int64 and A.colidx.dtype == np.int32
    assert A.rowptr[0] == 0 and A.rowptr[-1] == A.nnz == A.colidx.size == A.values.size
    assert np.all(np.diff(A.rowptr) >= 0)
    for r in range(A.n):
        c = A.colidx[A.rowptr[r]:A.rowptr[r + 1]]
        assert np.all(np.diff(c) > 0)                       # sorted, no duplicates
    assert A.nnz == 0 or (A.colidx.min() >= 0 and A.colidx.max() < A.n)


def _dense(A):
    D = np.zeros((A.n, A.n))
    for r in range(A.n):
        D[r, A.colidx[A.rowptr[r]:A.rowptr[r + 1]]] = A.values[A.rowptr[r]:A.rowptr[r + 1]]
    return D


@pytest.mark.parametrize("a", [np.zeros(0, np.int64), np.array([7], np.int64), np.array([3, 3, 3], np.int64),
                               np.random.default_rng(1).integers(0, 50, 1000),
                               np.random.default_rng(2).integers(-(1 << 40), 1 << 40, 10000)])
def test_sorted_unique_equals_numpy(a):
    assert np.array_equal(w._sorted_unique(a), np.unique(a))


def test_rmat_gcn_structure_and_normalisation():
    A = w.rmat_gcn(9, 8, seed=3)
    _check_csr(A)
    D = _dense(A)
    assert np.array_equal(D != 0, (D != 0).T)               # symmetric pattern
    assert np.all(np.diag(D) > 0)                           # one self-loop per vertex
    deg = np.diff(A.rowptr).astype(np.float64)
    # GCN normalisation: entry (u, v) = 1 / sqrt(d_u d_v), d = entries of the row of A + I
    r, c = np.nonzero(D)
    assert np.allclose(D[r, c], 1.0 / np.sqrt(deg[r] * deg[c]), rtol=0, atol=1e-15)
    # the power-law draw: the largest degree is far above the mean
    assert deg.max() > 8 * deg.mean()


def test_rmat_edges_seeded_and_in_range():
    n, u, v = w.rmat_edges(10, 4, seed=11)
    n2, u2, v2 = w.rmat_edges(10, 4, seed=11)
    assert n == 1024 and u.size == v.size == 4 * n and u.dtype == np.int64
    assert np.array_equal(u, u2) and np.array_equal(v, v2)
    assert u.min() >= 0 and u.max() < n and v.min() >= 0 and v.max() < n
    # quadrant probabilities: the top bit of u is set with probability c + d = 0.24
    top = (u >> 9) & 1
    assert abs(top.mean() - 0.24) < 0.05


def test_grid_stencils_row_normalised():
    for A, per_row in ((w.grid2d_64(), 5), (w.grid3d(6), 7)):
        _check_csr(A)
        deg = np.diff(A.rowptr)
        assert deg.max() == per_row and deg.min() >= 3      # diagonal + neighbours, fewer on the boundary
        sums = np.add.reduceat(A.values, A.rowptr[:-1])
        assert np.allclose(sums, 1.0, atol=1e-6)            # rows sum to one (values rounded to f32)


def test_rgg_symmetric_with_self_loops():
    A = w.rgg(2000, seed=4)
    _check_csr(A)
    D = _dense(A)
    assert np.array_equal(D != 0, (D != 0).T) and np.all(np.diag(D) > 0)
    assert 5 < A.nnz / A.n - 1 < 11                         # mean degree about 8 (fewer at the border)


def test_features_and_sizes_seeded():
    X = w.features(100, 16, seed=3)
    assert X.shape == (100, 16) and X.dtype == np.float32
    assert np.array_equal(X, w.features(100, 16, seed=3)) and not np.array_equal(X, w.features(100, 16, seed=4))
    s = w.log_uniform_sizes(1000, 1e3, 2e6, seed=1)
    assert s.min() >= 1e3 and s.max() <= 2e6
    assert abs(np.median(np.log(s)) - 0.5 * (np.log(1e3) + np.log(2e6))) < 0.3
