"""Pins of the FP64 value oracle (oracle/spmm.py) against facts fixed by mathematics.

* closed-form eigenpairs of the Dirichlet 5-point / 7-point stencils;
* row-normalised matrices fix the all-ones vector; GCN-normalised ones fix d^{1/2};
* brute force (dense, entry by entry) on tiny inputs;
* the iteration equals the dense matrix power, and with per-column rescaling it
  equals the normalised matrix power (scalars commute with A);
* Eq. 1 (Section 3): sum_i P_i B_i P_i^T X equals A X for the oracle's own decomposition;
* the sigma parts: the rectifier is the identity on non-negative data and zero on
  non-positive data and splits y = relu(y) - relu(-y); row normalisation gives unit rows, is
  blind to positive row scales and maps a rank-one u v^T to sign(u) v / |v|; a row-normalised
  A keeps the all-ones block fixed under row normalisation, a GCN-normalised A keeps
  d^{1/2} fixed under the rectifier and column normalisation.
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


def test_relu_definition_and_fixed_points():
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((50, 6))
    R = S.relu(Y)
    assert np.all(R >= 0.0) and np.array_equal(S.relu(R), R)
    assert np.array_equal(R - S.relu(-Y), Y)                    # y = max(0, y) - max(0, -y)
    assert np.array_equal(R[Y > 0], Y[Y > 0]) and np.all(R[Y <= 0] == 0.0)
    # a matrix with positive values: non-negative data stays as it was, non-positive data vanishes
    A = w.grid_stencil((9, 7), seed=2)
    Xp = np.abs(rng.standard_normal((A.n, 3)))
    assert np.allclose(S.iterate(A, Xp, 4, rectify=True), S.iterate(A, Xp, 4), rtol=1e-14, atol=0)
    assert np.count_nonzero(S.iterate(A, -Xp, 1, rectify=True)) == 0


def test_row_normalise_definition_and_fixed_points():
    rng = np.random.default_rng(4)
    Y = rng.standard_normal((40, 5))
    Y[7] = 0.0
    N = S.row_normalise(Y)
    nrm = np.linalg.norm(N, axis=1)
    assert np.allclose(np.delete(nrm, 7), 1.0, atol=1e-15) and nrm[7] == 0.0
    c = np.exp(rng.standard_normal(40))[:, None]
    assert np.allclose(S.row_normalise(c * Y), N, rtol=1e-14, atol=1e-15)
    u, v = rng.standard_normal(30), rng.standard_normal(4)
    assert np.allclose(S.row_normalise(np.outer(u, v)), np.sign(u)[:, None] * v / np.linalg.norm(v), atol=1e-15)
    # row-normalised A maps the all-ones block to itself, so 1 / sqrt(k) is a fixed point
    A = w.grid3d(6, seed=3)
    X1 = np.ones((A.n, 4))
    assert np.allclose(S.iterate(A, X1, 5, rownorm=True), 0.5, atol=1e-14)


def test_sigma_composition_on_gcn_fixed_point():
    # GCN-normalised A fixes d^{1/2}; it is positive, so the rectifier keeps it and the
    # column normalisation returns d^{1/2} / |d^{1/2}| after every step
    A = w.rmat_gcn(9, 8, seed=8)
    d = np.sqrt(np.diff(A.rowptr).astype(np.float64))
    X = np.stack([d, 2 * d], axis=1)
    Y = S.iterate(A, X, 6, rescale=True, rectify=True)
    assert np.allclose(Y, (d / np.linalg.norm(d))[:, None], rtol=1e-12, atol=1e-14)
    # the order is column(row(relu(.))): on the same data row normalisation makes each row
    # (d_r, 2 d_r) / |.| = (1, 2) / sqrt(5), then the columns are normalised
    Z = S.iterate(A, X, 1, rescale=True, rectify=True, rownorm=True)
    ref = np.tile(np.array([1.0, 2.0]) / math.sqrt(5.0), (A.n, 1))
    assert np.allclose(Z, ref / np.linalg.norm(ref, axis=0), rtol=1e-12)
