"""CPU checks of the fused row program the device kernels run (arrow_get_program).

The GPU kernels read this program; here it is evaluated with numpy (no GPU) and checked
against the FP64 oracle product, and its layout invariants are checked entry by entry:
every entry of A appears exactly once; each entry sits in the row of its vertex's pi_0
position and names the pi_0 position of its column; inside a row the levels come in order
and, inside a level, the columns in increasing level position (Alg. 2's write-back with
destinations fixed at preprocessing); split rows are cut into contiguous segments of at
most `segment` entries; tiles cover the short rows in order within their size limits.
"""
import numpy as np
import pytest

import workloads as w
from oracle import decompose as D
from oracle import spmm as S


@pytest.fixture(scope="module")
def arrow():
    from paper_2402_19364_gb300 import build
    build.build()
    import paper_2402_19364_gb300 as pkg
    return pkg


def _star(n=300):
    rows = np.r_[np.zeros(n - 1, np.int64), np.arange(1, n), np.arange(n)]
    cols = np.r_[np.arange(1, n), np.zeros(n - 1, np.int64), np.arange(n)]
    rp, ci = w._csr_from_pairs(n, rows, cols)
    return w.Csr(n, rp, ci, np.linspace(0.5, 1.5, ci.size))


CASES = {
    "grid2d_64": (lambda: w.grid2d_64(), 64, {}),
    "grid3d_12": (lambda: w.grid3d(12), 144, {}),
    "rmat10_split": (lambda: w.rmat_gcn(10, 16, seed=4), 32, {"long_row": 16, "segment": 64}),
    "rgg": (lambda: w.rgg(3000, seed=7), 55, {}),
    "nonsym": (lambda: w.random_csr(300, 0.02, 8), 4, {}),
    "star": (lambda: _star(), 2, {"long_row": 8, "segment": 32}),
    "empty": (lambda: w.Csr(100, np.zeros(101, np.int64), np.zeros(0, np.int32), np.zeros(0)), 8, {}),
    "b_ge_n": (lambda: w.random_csr(50, 0.1, 1, symmetric=True, diag=True), 64, {}),
}


def _entry_levels(A, b, seed=0, pred="block"):
    """Level of every entry of A and its level-position column, from the oracle's decomposition."""
    lv = D.la_decompose(A, b, seed=seed, predicate=D.pred_band if pred == "band" else D.pred_block) if A.nnz else []
    key = {}
    for i, L in enumerate(lv):
        rows = np.repeat(np.arange(L.n), np.diff(L.rowptr))
        for p, q in zip(rows, L.colidx):
            key[(int(L.iperm[p]), int(L.iperm[q]))] = (i, int(q))
    arow = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    return [key[(int(r), int(c))] for r, c in zip(arow, A.colidx)]


@pytest.mark.parametrize("pred", ["block", "band"])
@pytest.mark.parametrize("case", list(CASES))
def test_program_layout_and_value(arrow, case, pred):
    make, b, kw = CASES[case]
    A = make()
    M = arrow.ArrowMatrix(A, b, host_only=True, predicate=pred, **kw)
    pg = M.program()
    n, nnz = A.n, A.nnz
    perm0 = M.level_perm(0).astype(np.int64) if M.num_levels else np.arange(n)
    iperm0 = np.empty(n, np.int64)
    iperm0[perm0] = np.arange(n)
    arow = np.repeat(np.arange(n), np.diff(A.rowptr))
    rp, col, src = pg["rowptr"].astype(np.int64), pg["col"].astype(np.int64), pg["src"].astype(np.int64)
    lcol, lsrc = pg["lcol"].astype(np.int64), pg["lsrc"].astype(np.int64)
    long_rows, segptr = pg["long_rows"].astype(np.int64), pg["long_segptr"].astype(np.int64)
    sb, se = pg["seg_begin"].astype(np.int64), pg["seg_end"].astype(np.int64)

    # every entry of A exactly once, in the row of its vertex, reading its column's pi_0 row
    assert np.array_equal(np.sort(np.r_[src, lsrc]), np.arange(nnz))
    prow = np.repeat(np.arange(n), np.diff(rp))
    assert np.array_equal(arow[src], iperm0[prow])
    assert np.array_equal(col, perm0[A.colidx[src]])
    assert np.array_equal(lcol, perm0[A.colidx[lsrc]])

    # short rows hold at most long_row entries; split rows none, and more than long_row in the long stream
    lens = np.diff(rp)
    assert lens.max(initial=0) <= pg["long_row"]
    assert np.all(np.diff(long_rows) > 0) and np.all(lens[long_rows] == 0)
    full = np.diff(A.rowptr)[iperm0]
    assert np.all(full[long_rows] > pg["long_row"])
    short = np.ones(n, bool)
    short[long_rows] = False
    assert np.array_equal(lens[short], full[short])

    # segments: each split row's range cut in order into non-empty pieces of at most `segment`
    seg = kw.get("segment", 512)
    pos = 0
    for li, p in enumerate(long_rows):
        g0, g1 = segptr[li], segptr[li + 1]
        assert g1 > g0 and sb[g0] == pos
        assert np.all(sb[g0 + 1:g1] == se[g0:g1 - 1]) and np.all(se[g0:g1] - sb[g0:g1] <= seg)
        assert np.all(se[g0:g1] > sb[g0:g1])
        pos = se[g1 - 1]
        assert np.all(arow[lsrc[sb[g0]:pos]] == iperm0[p]) and pos - sb[g0] == full[p]
    assert pos == lcol.size and segptr[-1] == sb.size

    # tiles: consecutive rows from 0 to n within the handle's limits
    tr, te = pg["tile_row"].astype(np.int64), pg["tile_ent"].astype(np.int64)
    tune = M.tuning
    if n:
        assert tr[0] == 0 and tr[-1] == n and np.all(np.diff(tr) > 0)
        assert np.array_equal(te, rp[tr])
        assert np.diff(tr).max() <= tune["tile_rows"] and np.diff(te).max() <= tune["tile_nnz"]

    # inside a short row: levels in order, inside a level increasing level position
    if nnz:
        lvpos = _entry_levels(A, b, pred=pred)
        keys = [lvpos[int(e)] for e in src]
        for p in range(n):
            k = keys[rp[p]:rp[p + 1]]
            assert k == sorted(k) and len(set(k)) == len(k)

    # evaluate the program as the kernels do and compare with the FP64 oracle product
    X = np.random.default_rng(1).standard_normal((n, 3))
    Xh = X[iperm0]
    Yh = np.zeros_like(Xh)
    np.add.at(Yh, prow, A.values[src][:, None] * Xh[col])
    for li, p in enumerate(long_rows):
        for g in range(segptr[li], segptr[li + 1]):
            Yh[p] += (A.values[lsrc[sb[g]:se[g]]][:, None] * Xh[lcol[sb[g]:se[g]]]).sum(axis=0)
    Y = Yh[perm0]
    R = S.spmm(A, X)
    assert np.allclose(Y, R, rtol=1e-12, atol=1e-12)
