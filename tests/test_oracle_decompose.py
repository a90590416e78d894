"""Pins of the LA-Decompose oracle (oracle/decompose.py).

Each test fixes a part of the decomposition with something other than the
oracle itself: the paper's worked example (Fig. 3) and tile picture (Fig. 2),
published SplitMix64 outputs, scipy's minimum spanning tree, hand-derived
layouts of small trees, Lemma 4.3's band count, Lemma 4.1's Markov bound,
and exact reconstruction A = sum_i P_i B_i P_i^T (Eq. 1) with every entry in
exactly one level.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import minimum_spanning_tree

import workloads as w
from oracle import decompose as D

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _csr_from_edges(n, edges, diag=False, value=None):
    rows, cols = [], []
    for u, v in edges:
        rows += [u, v]
        cols += [v, u]
    if diag:
        rows += list(range(n))
        cols += list(range(n))
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    rowptr, colidx = w._csr_from_pairs(n, rows, cols) if rows.size else (np.zeros(n + 1, np.int64), np.zeros(0, np.int32))
    vals = np.arange(1, colidx.size + 1, dtype=np.float64) if value is None else np.full(colidx.size, value)
    return w.Csr(n, rowptr, colidx, vals)


def _dense(n, rows, cols, vals):
    M = np.zeros((n, n))
    M[rows, cols] = vals
    return M


def _reconstruct(levels, n):
    M = np.zeros((n, n))
    for lv in levels:
        r = np.repeat(np.arange(n), np.diff(lv.rowptr))
        # P B P^T: entry (p, q) of B_i sits at (iperm[p], iperm[q]) of A
        M[lv.iperm[r], lv.iperm[lv.colidx]] += lv.values
    return M


def test_splitmix64_published_outputs():
    vals = []
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                i, h = line.split()
                vals.append((int(i), int(h, 16)))
    gamma = 0x9E3779B97F4A7C15
    states = np.array([(i * gamma) % 2 ** 64 for i, _ in vals], dtype=np.uint64)
    out = D.splitmix64(states)
    assert [int(x) for x in out] == [h for _, h in vals]


def test_edge_keys_distinct_and_seeded():
    rng = np.random.default_rng(0)
    u = rng.integers(0, 1 << 20, 200000)
    v = u + 1 + rng.integers(0, 1 << 20, 200000)
    key = np.unique(u * (1 << 22) + v)
    u, v = key >> 22, key & ((1 << 22) - 1)
    k0 = D.edge_keys(u, v, seed=0, level=0)
    assert np.unique(k0).size == k0.size            # bijection: distinct edges, distinct keys
    assert not np.array_equal(k0, D.edge_keys(u, v, seed=0, level=1))
    assert not np.array_equal(k0, D.edge_keys(u, v, seed=1, level=0))


def test_pred_block_is_fig2_tile_pattern():
    # Fig. 2: a 4x4-tile arrow matrix owns row tile 0, column tile 0 and the diagonal tiles
    b = 3
    r, c = np.meshgrid(np.arange(4 * b), np.arange(4 * b), indexing="ij")
    I, J = r // b, c // b
    assert np.array_equal(D.pred_block(r, c, b), (I == 0) | (J == 0) | (I == J))
    # the band predicate is the definition of arrow width in Section 1 (0-based)
    assert np.array_equal(D.pred_band(r, c, b), (r < b) | (c < b) | (np.abs(r - c) <= b))


def _fig3():
    edges = {}
    with open(os.path.join(GOLDEN, "fig3_split.txt")) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "n":
                n = int(t[1])
            elif t[0] == "b":
                b = int(t[1])
            else:
                edges[(int(t[0]), int(t[1]))] = t[2]
    return n, b, edges


def test_fig3_split_step_band_predicate():
    n, b, edges = _fig3()
    A = _csr_from_edges(n, list(edges))
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    (rp, ci, vv), n_act, take = D.split_step(n, rows, A.colidx.astype(np.int64), A.values, np.arange(n), b,
                                             D.pred_band)
    got = {(int(r), int(c)) for r, c in zip(np.repeat(np.arange(n), np.diff(rp)), ci)}
    want = {(u, v) for (u, v), k in edges.items() if k != "outside"}
    want |= {(v, u) for u, v in want}
    assert len(got) == 14 and got == want
    rest = {(int(r), int(c)) for r, c in zip(rows[~take], A.colidx[~take])}
    assert rest == {(2, 5), (5, 2)}
    # block predicate: the tiles {0,1},{2,3},{4,5},{6}; {3,4} and {5,6} leave B_0 as well
    _, _, take_b = D.split_step(n, rows, A.colidx.astype(np.int64), A.values, np.arange(n), b, D.pred_block)
    rest_b = {(int(r), int(c)) for r, c in zip(rows[~take_b], A.colidx[~take_b])}
    assert rest_b == {(2, 5), (5, 2), (3, 4), (4, 3), (5, 6), (6, 5)}


def test_fig3_remainder_becomes_head_of_b1():
    # Fig. 3's B_1: the single remaining edge {2,5} is moved into the head (positions 0, 1)
    A = _csr_from_edges(7, [(2, 5)])
    lv = D.la_decompose(A, b=2)
    assert len(lv) == 1
    B = lv[0]
    assert list(B.iperm[:2]) == [2, 5]
    assert _dense(7, np.repeat(np.arange(7), np.diff(B.rowptr)), B.colidx, B.values)[0, 1] != 0
    assert B.nnz == 2 and B.n_active == 2


def test_head_selection_hand_example():
    # degrees: 0:1 1:3 2:2 3:3 4:1 5:0 -> by (deg desc, id asc): 1, 3, 2, 0, 4, 5
    deg = np.array([1, 3, 2, 3, 1, 0])
    assert list(D.select_head(deg, 3)) == [1, 3, 2]
    assert list(D.select_head(deg, 10)) == [1, 3, 2, 0, 4, 5]


def test_kruskal_matches_scipy_mst():
    A = w.random_csr(400, 0.01, 4, symmetric=True)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    eu, ev = D.undirected_edges(rows, A.colidx.astype(np.int64), A.n)
    key = D.edge_keys(eu, ev, seed=3, level=0)
    forest = D.kruskal_msf(A.n, eu, ev, key)
    rank = np.empty(key.size)
    rank[np.argsort(key)] = np.arange(1, key.size + 1, dtype=np.float64)
    G = sp.coo_matrix((rank, (eu, ev)), shape=(A.n, A.n)).tocsr()
    T = minimum_spanning_tree(G).tocoo()
    want = {(min(a, c), max(a, c)) for a, c in zip(T.row, T.col)}
    assert {(min(a, c), max(a, c)) for a, c in forest} == want


def test_smallest_first_hand_example():
    # root 0; children 1 (subtree {1,4,5,6}), 2 (leaf), 3 (subtree {3,7}); 4 has leaves 5, 6
    edges = [(0, 1), (0, 2), (0, 3), (1, 4), (4, 5), (4, 6), (3, 7)]
    adj = [[] for _ in range(8)]
    for a, c in edges:
        adj[a].append(c)
        adj[c].append(a)
    assert D.smallest_first_preorder(adj, 0) == [0, 2, 3, 7, 1, 4, 5, 6]


def test_forest_arrangement_hand_example():
    # non-head vertices 1..8: trees {1,2,3}, {4}, {5,6}, {7}, {8}; head {0}
    # 4 and 8 touched (edges to the head), 7 untouched.
    is_head = np.zeros(9, dtype=bool)
    is_head[0] = True
    touched = np.ones(9, dtype=bool)
    touched[7] = False
    order = D.forest_arrangement(9, is_head, [(1, 2), (2, 3), (5, 6)], touched)
    assert list(order) == [1, 2, 3, 5, 6, 4, 8, 7]


def _random_tree(n, rng):
    parent = [int(rng.integers(0, v)) for v in range(1, n)]
    return [(p, v + 1) for v, p in enumerate(parent)]


@pytest.mark.parametrize("n,x", [(60, 2), (200, 3), (500, 4), (1000, 2)])
def test_lemma_4_3_band_count(n, x):
    rng = np.random.default_rng(n + x)
    edges = _random_tree(n, rng)
    adj = [[] for _ in range(n)]
    for a, c in edges:
        adj[a].append(c)
        adj[c].append(a)
    delta = max(len(a) for a in adj)
    order = D.smallest_first_preorder(adj, 0)
    pos = np.empty(n, dtype=np.int64)
    pos[order] = np.arange(n)
    within = sum(abs(pos[a] - pos[c]) <= x * delta for a, c in edges)
    assert within >= min(n - 1, math.ceil((x - 1) * (n - 1) / x) + 1)


def test_lemma_4_1_markov_bound_band():
    # under the band predicate the entries of G_i' left over have stretch > b, so
    # their count is at most lambda_{pi'}(G_i') / b
    A = w.grid_stencil((24, 24), seed=3)
    b = 6
    n = A.n
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    cols = A.colidx.astype(np.int64)
    lv = D.la_decompose(A, b, seed=5, predicate=D.pred_band)
    eu, ev = D.undirected_edges(rows, cols, n)
    head = lv[0].iperm[:b]
    keep = ~np.isin(eu, head) & ~np.isin(ev, head)
    stretch = np.abs(lv[0].perm[eu[keep]] - lv[0].perm[ev[keep]])
    lam = stretch.sum()
    left = (stretch > b).sum()
    assert left <= lam / b
    nxt = sum(l.nnz for l in lv[1:]) // 2
    assert nxt == left


def _matrices():
    yield w.grid_stencil((16, 16), seed=1), 4
    yield w.random_csr(200, 0.02, 1, symmetric=True, diag=True), 5
    yield w.random_csr(150, 0.03, 2), 3                       # nonsymmetric
    yield w.rmat_gcn(8, 8, seed=2), 6
    yield _csr_from_edges(50, [(0, v) for v in range(1, 50)]), 2  # star
    yield _csr_from_edges(64, [(v, v + 1) for v in range(63)], diag=True), 2  # path
    yield _csr_from_edges(20, [], diag=True), 3               # diagonal only
    yield w.Csr(10, np.zeros(11, np.int64), np.zeros(0, np.int32), np.zeros(0)), 2   # empty
    yield w.random_csr(30, 0.1, 3, symmetric=True), 64        # b >= n: one level


@pytest.mark.parametrize("case", range(9))
def test_exact_reconstruction_and_arrow_shape(case):
    A, b = list(_matrices())[case]
    n = A.n
    lv = D.la_decompose(A, b, seed=case)
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    want = _dense(n, rows, A.colidx, A.values)
    assert np.array_equal(_reconstruct(lv, n), want)                  # exact: no arithmetic
    assert sum(l.nnz for l in lv) == A.nnz                            # every entry exactly once
    seen = np.zeros((n, n), dtype=np.int64)
    for i, l in enumerate(lv):
        r = np.repeat(np.arange(n), np.diff(l.rowptr))
        assert D.pred_block(r, l.colidx, b).all()                     # arrow shape of every B_i
        assert np.array_equal(np.sort(l.perm), np.arange(n))           # pi_i is a permutation
        assert np.array_equal(l.perm[l.iperm], np.arange(n))
        seen[l.iperm[r], l.iperm[l.colidx]] += 1
        if l.nnz:
            touched = np.zeros(n, dtype=bool)
            touched[r] = True
            touched[l.colidx] = True
            assert l.n_active == np.nonzero(touched)[0].max() + 1
        # vertices that still hold an entry of A_i sit, past the head, in a prefix of
        # pi_i (the non-zero rows are collected at the top)
        alive = np.zeros(n, dtype=bool)
        for m in lv[i:]:
            rm = np.repeat(np.arange(n), np.diff(m.rowptr))
            alive[m.iperm[rm]] = True
            alive[m.iperm[m.colidx]] = True
        pos_alive = alive[l.iperm]
        if pos_alive[b:].any():
            last = np.nonzero(pos_alive[b:])[0].max() + b
            assert pos_alive[b:last + 1].all()
    assert seen.max() <= 1 and seen.sum() == A.nnz
    if b >= n:
        assert len(lv) <= 1


def test_head_vertices_leave_no_entries():
    A = w.rmat_gcn(9, 8, seed=6)
    b = 8
    lv = D.la_decompose(A, b, seed=1)
    assert len(lv) >= 2
    for i, l in enumerate(lv[:-1]):
        head = set(l.iperm[:b].tolist())
        for m in lv[i + 1:]:
            r = np.repeat(np.arange(A.n), np.diff(m.rowptr))
            verts = set(m.iperm[r].tolist()) | set(m.iperm[m.colidx].tolist())
            assert not (head & verts)


def test_b_below_two_rejected():
    with pytest.raises(ValueError):
        D.la_decompose(w.grid2d_64(), 1)


def test_fig3_shape_of_b0_and_b1():
    # Fig. 3 colours B_0's edges: dashed blue = pruned head part, green = band.  Under the
    # band predicate with pi_0 = identity and b = 2: 4 head edges and 3 band edges, each
    # stored twice (symmetric), and the b x b tiles they touch, counted by hand:
    # {0,1}->(0,0); {0,4},{0,5}->(0,2),(2,0); {1,3}->(0,1),(1,0); {2,3}->(1,1);
    # {3,4}->(1,2),(2,1); {5,6}->(2,3),(3,2)  = 10 tiles.
    n, b, edges = _fig3()
    A = _csr_from_edges(n, list(edges))
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    (rp, ci, vv), n_act, take = D.split_step(n, rows, A.colidx.astype(np.int64), A.values, np.arange(n), b,
                                             D.pred_band)
    head = sum(2 for k in edges.values() if k == "head")
    band = sum(2 for k in edges.values() if k == "band")
    assert (head, band) == (8, 6)
    assert D.arrow_shape(np.repeat(np.arange(n), np.diff(rp)), ci, b) == (head, band, 10)
    # B_1: the remaining edge {2, 5} moved to head positions 0 and 1: one tile, all head
    lv = D.la_decompose(_csr_from_edges(7, [(2, 5)]), b=2)
    assert D.level_shape(lv[0]) == (2, 0, 1)


def test_count_tiles_closed_forms():
    # 2D N x N 5-point stencil in natural order, b = N: tile row R holds grid rows R-1, R,
    # R+1 -> 3N - 2 non-zero tiles; one tile when b = N^2
    for N in (8, 13):
        A = w.grid_stencil((N, N), seed=1)
        assert D.count_tiles(A, N) == 3 * N - 2
        assert D.count_tiles(A, N * N) == 1
    # diagonal only, n = 10, b = 3: ceil(10/3) = 4 diagonal tiles; positions 0..2 are head
    n = 10
    A = w.Csr(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n))
    assert D.count_tiles(A, 3) == 4
    assert D.arrow_shape(np.arange(n), np.arange(n), 3) == (3, 7, 4)


def test_level_shapes_partition_the_entries():
    A = w.rmat_gcn(9, 8, seed=2)
    for pred in (D.pred_block, D.pred_band):
        lv = D.la_decompose(A, b=24, predicate=pred)
        for L in lv:
            h, bd, t = D.level_shape(L)
            assert h + bd == L.nnz and t >= 1
            # every B_i entry outside the head lies in a diagonal tile (block) or the band
            rows = np.repeat(np.arange(L.n), np.diff(L.rowptr))
            off = (rows >= L.b) & (L.colidx >= L.b)
            assert np.all(pred(rows[off], L.colidx[off], L.b))
