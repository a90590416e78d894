"""Pins of the multi-core C form of the value oracle (oracle/cspmm.py) against mathematics:
closed-form stencil eigenpairs, dense brute force, the matrix power, and the scipy form."""
import math

import numpy as np
import pytest

import workloads as w
from oracle import cspmm as C
from oracle import spmm as S


def test_closed_form_eigenpairs():
    N0, N1, d = 11, 7, -4.0
    A = w.grid_stencil((N0, N1), unit_weights=True, diag_value=d)
    i = np.arange(N0)[:, None]
    j = np.arange(N1)[None, :]
    for p, q in ((1, 1), (4, 6), (11, 7)):
        v = (np.sin(math.pi * p * (i + 1) / (N0 + 1)) * np.sin(math.pi * q * (j + 1) / (N1 + 1))).ravel()
        lam = d + 2 * math.cos(math.pi * p / (N0 + 1)) + 2 * math.cos(math.pi * q / (N1 + 1))
        assert np.max(np.abs(C.spmm(A, v)[:, 0] - lam * v)) < 1e-12


@pytest.mark.parametrize("seed,density,sym", [(1, 0.05, False), (2, 0.2, True), (5, 0.01, False)])
def test_dense_brute_force_and_scipy_form(seed, density, sym):
    A = w.random_csr(70, density, seed, symmetric=sym)
    X = np.random.default_rng(seed).standard_normal((70, 6))
    Y = C.spmm(A, X)
    assert np.allclose(Y, S.spmm_dense(A, X), rtol=0, atol=1e-13)
    assert np.allclose(Y, S.spmm(A, X), rtol=1e-14, atol=1e-14)


def test_iteration_is_the_matrix_power_and_normalises():
    A = w.random_csr(40, 0.1, 5, diag=True)
    X = np.random.default_rng(0).standard_normal((40, 3))
    P = np.linalg.matrix_power(S.spmm_dense(A, np.eye(40)), 5) @ X
    assert np.allclose(C.iterate(A, X, 5), P, rtol=1e-12, atol=1e-12)
    assert np.allclose(C.iterate(A, X, 5, rescale=True), P / np.linalg.norm(P, axis=0), rtol=1e-12, atol=1e-13)


def test_rows_independent_of_thread_count():
    # every row is summed in entry order by one thread: the bits match the 1-core ordering,
    # which is also what a row-by-row Python loop gives
    A = w.rmat_gcn(11, 8, seed=2)
    X = np.random.default_rng(3).standard_normal((A.n, 4))
    Y = C.spmm(A, X)
    for r in (0, 1, 7, A.n // 2, A.n - 1):
        acc = np.zeros(4)
        for jj in range(A.rowptr[r], A.rowptr[r + 1]):
            acc = acc + A.values[jj] * X[A.colidx[jj]]
        assert np.array_equal(Y[r], acc)
    assert C.threads() >= 1


def test_empty_and_row_normalised_fixed_point():
    E = w.Csr(5, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0))
    assert np.array_equal(C.spmm(E, np.ones((5, 2))), np.zeros((5, 2)))
    A = w.grid_stencil((9, 8, 7), seed=4, round_to=None)
    assert np.max(np.abs(C.iterate(A, np.ones((A.n, 1)), 6) - 1.0)) < 1e-13


def test_column_normalise_unit_columns_and_direction():
    Y = np.random.default_rng(4).standard_normal((10_000, 5)) * np.array([1e-3, 1.0, 7.0, 1e3, 2.0])
    Z = C.column_normalise(Y)
    assert np.allclose(np.linalg.norm(Z, axis=0), 1.0, rtol=0, atol=1e-14)
    assert np.allclose(Z * np.linalg.norm(Y, axis=0), Y, rtol=1e-14, atol=0)
    assert np.allclose(Z, S.column_normalise(Y), rtol=1e-14, atol=1e-16)
