"""Pins of the FP64 value oracle (oracle/spmm.py) against facts fixed by mathematics.

* closed-form eigenpairs of the Dirichlet 5-point / 7-point stencils;
* row-normalised matrices fix the all-ones vector; GCN-normalised ones fix d^{1/2};
* brute force (dense, entry by entry) on tiny inputs;
* the iteration equals the dense matrix power, and with per-column rescaling it
  equals the normalised matrix power (scalars commute with A);
* Eq. 1 (Section 3): sum_i P_i B_i P_i^T X equals A X for the oracle's own decomposition.
"""
import math

import numpy as np
import pytest

import workloads as w
from oracle import decompose as D
from oracle import spmm as S


def _eig_2d(N0, N1, pairs):
    V = np.zeros((N0 * N1, len(pairs)))
    lam = np.zeros(len(pairs))
    i = np.arange(N0)[:, None]
    j = np.arange(N1)[None, :]
    for t, (p, q) in enumerate(pairs):
        V[:, t] = (np.sin(math.pi * p * (i + 1) / (N0 + 1)) * np.sin(math.pi * q * (j + 1) / (N1 + 1))).ravel()
        lam[t] = 2 * math.cos(math.pi * p / (N0 + 1)) + 2 * math.cos(math.pi * q / (N1 + 1))
    return V, lam


def test_stencil_2d_closed_form_eigenpairs():
    N0, N1, d = 13, 9, -4.0
    A = w.grid_stencil((N0, N1), unit_weights=True, diag_value=d)
    pairs = [(1, 1), (2, 5), (13, 9), (7, 3)]
    V, lam = _eig_2d(N0, N1, pairs)
    Y = S.spmm(A, V)
    assert np.max(np.abs(Y - V * (lam + d))) < 1e-12
    # the same through the decomposed product of Eq. 1
    lv = D.la_decompose(A, b=4, seed=7)
    Yd = S.decomposed_product(lv, V)
    assert np.max(np.abs(Yd - V * (lam + d))) < 1e-12


def test_stencil_3d_closed_form_eigenpairs():
    N, d = 7, 1.5
    A = w.grid_stencil((N, N, N), unit_weights=True, diag_value=d)
    idx = np.arange(N)
    pqr = [(1, 1, 1), (2, 3, 4), (7, 1, 6)]
    V = np.zeros((N ** 3, len(pqr)))
    lam = np.zeros(len(pqr))
    for t, (p, q, r) in enumerate(pqr):
        f = [np.sin(math.pi * m * (idx + 1) / (N + 1)) for m in (p, q, r)]
        V[:, t] = np.einsum("i,j,k->ijk", *f).ravel()
        lam[t] = d + sum(2 * math.cos(math.pi * m / (N + 1)) for m in (p, q, r))
    assert np.max(np.abs(S.spmm(A, V) - V * lam)) < 1e-12
    lv = D.la_decompose(A, b=8, seed=1)
    assert np.max(np.abs(S.decomposed_product(lv, V) - V * lam)) < 1e-12


def test_row_normalised_fixes_ones():
    A = w.grid_stencil((20, 17), seed=11, round_to=None)
    one = np.ones((A.n, 2))
    assert np.max(np.abs(S.spmm(A, one) - 1.0)) < 1e-14
    A3 = w.grid_stencil((6, 5, 4), seed=12, round_to=None)
    assert np.max(np.abs(S.iterate(A3, np.ones((A3.n, 1)), 9) - 1.0)) < 1e-13


def test_gcn_normalised_fixes_sqrt_degree():
    A = w.rmat_gcn(9, 8, seed=3)
    d = np.diff(A.rowptr).astype(np.float64)            # degree of A + I (self-loops included)
    s = np.sqrt(d)[:, None]
    assert np.max(np.abs(S.spmm(A, s) - s) / s) < 1e-13
    assert np.max(np.abs(S.iterate(A, s, 5) - s) / s) < 1e-12


@pytest.mark.parametrize("seed,density,sym", [(1, 0.05, False), (2, 0.2, True), (3, 0.01, False)])
def test_spmm_matches_dense_brute_force(seed, density, sym):
    A = w.random_csr(60, density, seed, symmetric=sym)
    X = np.random.default_rng(seed).standard_normal((60, 5))
    assert np.allclose(S.spmm(A, X), S.spmm_dense(A, X), rtol=0, atol=1e-13)


def test_iterate_is_matrix_power():
    A = w.random_csr(40, 0.1, 5, diag=True)
    X = np.random.default_rng(0).standard_normal((40, 3))
    M = S.spmm_dense(A, np.eye(40))
    ref = np.linalg.matrix_power(M, 6) @ X
    assert np.allclose(S.iterate(A, X, 6), ref, rtol=1e-12, atol=1e-12)
    # sigma = per-column L2 normalisation: X_T = N(A^T X), columns of unit norm
    Yr = S.iterate(A, X, 6, rescale=True)
    assert np.allclose(np.linalg.norm(Yr, axis=0), 1.0, atol=1e-14)
    assert np.allclose(Yr, ref / np.linalg.norm(ref, axis=0), rtol=1e-12, atol=1e-13)
    assert np.array_equal(S.iterate(A, X, 0), X.astype(np.float64))


def test_decomposed_product_equals_plain_product():
    for A, b in ((w.rmat_gcn(8, 8, seed=4), 6), (w.random_csr(100, 0.03, 9), 3), (w.grid2d_64(), 64)):
        X = np.random.default_rng(1).standard_normal((A.n, 4))
        lv = D.la_decompose(A, b, seed=2)
        assert np.allclose(S.decomposed_product(lv, X), S.spmm(A, X), rtol=1e-13, atol=1e-13)


def test_iterate_rows_equals_full_iteration():
    for A, T in ((w.grid_stencil((9, 8, 7), seed=2), 4), (w.rmat_gcn(9, 8, seed=8), 3),
                 (w.random_csr(200, 0.01, 3), 5)):
        X = np.random.default_rng(T).standard_normal((A.n, 3))
        rows = np.array([0, 5, A.n - 1, A.n // 2])
        full = S.iterate(A, X, T)[rows]
        assert np.allclose(S.iterate_rows(A, X, T, rows), full, rtol=1e-13, atol=1e-13)
        assert np.allclose(S.iterate_rows(A, lambda r: X[r], T, rows), full, rtol=1e-13, atol=1e-13)
