"""Multi-core FP64 form of the value oracle (test infrastructure only).

The same plain product as :func:`oracle.spmm.spmm` -- Y = A X in FP64 (Section 2; Eq. 1
makes the decomposed product equal to it) -- computed by a plain C loop (oracle/c/csr_spmm.c)
whose rows are spread over the host cores.  Each row is summed in CSR order by one thread,
so results do not depend on the thread count.  Pinned by tests/test_oracle_cspmm.py against
the closed-form stencil eigenpairs, dense brute force and the scipy form.
"""
from __future__ import annotations

import ctypes

import numpy as np

import os

_lib = None
LIB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "liboracle_c.so")


def lib():
    """The compiled C loop.  It is compiled (host C compiler, OpenMP when available) by the
    project's build step, __graft_entry__.build(), which the test session runs first."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: run __graft_entry__.build() to compile the oracle's C part")
        _lib = ctypes.CDLL(LIB)
        _lib.oracle_threads.restype = ctypes.c_int
        _lib.oracle_csr_spmm_f64.restype = None
        _lib.oracle_csr_spmm_f64.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        _lib.oracle_column_normalise_f64.restype = ctypes.c_int
        _lib.oracle_column_normalise_f64.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
    return _lib


def threads() -> int:
    """Host threads the C loop runs on."""
    return int(lib().oracle_threads())


def spmm(A, X: np.ndarray) -> np.ndarray:
    """Y = A X in FP64, rows in parallel, each row in CSR order."""
    rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int64)
    colidx = np.ascontiguousarray(A.colidx, dtype=np.int32)
    vals = np.ascontiguousarray(A.values, dtype=np.float64)
    Xc = np.ascontiguousarray(X, dtype=np.float64)
    if Xc.ndim == 1:
        Xc = Xc[:, None]
    Y = np.empty((A.n, Xc.shape[1]), dtype=np.float64)
    if A.n and Xc.shape[1]:
        lib().oracle_csr_spmm_f64(A.n, rowptr.ctypes.data, colidx.ctypes.data, vals.ctypes.data,
                                  Xc.ctypes.data, Xc.shape[1], Y.ctypes.data)
    return Y


def column_normalise(Y: np.ndarray) -> np.ndarray:
    """sigma of Section 2 as used here, in place on a fresh FP64 copy: every column divided by
    its FP64 L2 norm (squares summed in fixed 4096-row blocks, then over the blocks in order)."""
    Z = np.array(Y, dtype=np.float64, order="C", copy=True)
    if Z.ndim == 1:
        Z = Z[:, None]
    if Z.size and lib().oracle_column_normalise_f64(Z.shape[0], Z.shape[1], Z.ctypes.data) != 0:
        raise MemoryError("oracle_column_normalise_f64: allocation failed")
    return Z


def iterate(A, X: np.ndarray, iters: int, rescale: bool = False) -> np.ndarray:
    """X_{t+1} = sigma(A X_t) of Section 2, sigma = identity or per-column FP64 L2 normalisation."""
    Y = np.asarray(X, dtype=np.float64)
    for _ in range(iters):
        Y = spmm(A, Y)
        if rescale:
            Y = column_normalise(Y)
    return Y
