"""Randomised comparison of the library's host decomposer with the oracle (CPU, no GPU).

Small random matrices -- symmetric or not, with or without diagonal, of random density --
decomposed with random widths, seeds and both arrow predicates: the permutations, per-level
CSR structure and values, active rows and level shapes must agree bit for bit with the
oracle's LA-Decompose, and the fused row program the kernels run (block predicate) must
reproduce the FP64 product.
"""
import numpy as np
import pytest

import workloads as w
from oracle import decompose as D
from oracle import spmm as S

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402


def _matrix(n, density, seed, sym, diag):
    if density == 0:
        return w.Csr(n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    return w.random_csr(n, density, seed, symmetric=sym, diag=diag)


_arrow_pkg = None


def _pkg():
    global _arrow_pkg
    if _arrow_pkg is None:
        from paper_2402_19364_gb300 import build
        build.build()
        import paper_2402_19364_gb300 as pkg
        _arrow_pkg = pkg
    return _arrow_pkg


@settings(max_examples=150, deadline=None)
@given(n=st.integers(1, 70), density=st.sampled_from([0.0, 0.02, 0.06, 0.15, 0.4]), seed=st.integers(0, 10_000),
       sym=st.booleans(), diag=st.booleans(), b=st.integers(2, 40), dseed=st.integers(0, 2 ** 32),
       band=st.booleans(), long_row=st.sampled_from([0, 2, 4, 8]), segment=st.sampled_from([0, 2, 3, 16]))
def test_library_matches_oracle(n, density, seed, sym, diag, b, dseed, band, long_row, segment):
    arrow = _pkg()
    A = _matrix(n, density, seed, sym, diag)
    pred = "band" if band else "block"
    M = arrow.ArrowMatrix(A, b, seed=dseed, predicate=pred, host_only=True, long_row=long_row, segment=segment)
    L = D.la_decompose(A, b, seed=dseed, predicate=D.pred_band if band else D.pred_block)
    assert M.num_levels == len(L)
    for i, lv in enumerate(L):
        assert np.array_equal(M.level_perm(i), lv.perm)
        rp, ci, vv = M.level_csr(i)
        assert np.array_equal(rp, lv.rowptr) and np.array_equal(ci, lv.colidx) and np.array_equal(vv, lv.values)
        sh = M.level_shape(i)
        assert (sh["n_active"], sh["nnz"]) == (lv.n_active, lv.nnz)
        assert (sh["head_nnz"], sh["band_nnz"], sh["tiles"]) == D.level_shape(lv)
    # the fused program evaluated as the kernels do equals the FP64 product (either predicate)
    pg = M.program()
    perm0 = M.level_perm(0).astype(np.int64) if M.num_levels else np.arange(n)
    iperm0 = np.empty(n, np.int64)
    iperm0[perm0] = np.arange(n)
    X = np.random.default_rng(seed).standard_normal((n, 2))
    Xh = X[iperm0]
    Yh = np.zeros_like(Xh)
    rp = pg["rowptr"].astype(np.int64)
    prow = np.repeat(np.arange(n), np.diff(rp))
    np.add.at(Yh, prow, A.values[pg["src"]][:, None] * Xh[pg["col"]])
    for li, p in enumerate(pg["long_rows"]):
        for g in range(pg["long_segptr"][li], pg["long_segptr"][li + 1]):
            s0, s1 = pg["seg_begin"][g], pg["seg_end"][g]
            Yh[p] += (A.values[pg["lsrc"][s0:s1]][:, None] * Xh[pg["lcol"][s0:s1]]).sum(axis=0)
    assert np.allclose(Yh[perm0], S.spmm(A, X), rtol=1e-12, atol=1e-12)
    M.close()
