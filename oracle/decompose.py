"""LA-Decompose, restated step by step (test infrastructure only).

Follows Section 4.1 (LA-Decompose(A, b)): for level i, (1) put the b highest
degree vertices first, (2) lay out the rest with a linear arrangement of the
induced subgraph G_i', (3) B_i = the entries of P^T A_i P inside the arrow
shape, (4) A_{i+1} = A_i - P B_i P^T; repeat.  The arrangement of step (2) is
the random spanning forest scheme of Section 4.3 (random edge weights, a
minimum spanning forest, trees in decreasing size) with each tree laid out in
the smallest-first order of Section 4.4 (root first, then the child subtrees
in increasing size, recursively).

Where the paper leaves a choice open this file takes the following readings
(each also listed with the design notes of the repository):

* positions are 0-based; the head is positions 0..b-1;
* the arrow shape of B_i is the block-diagonal one of Section 3.1 / Fig. 2:
  ``pred_block(r, c) = r < b or c < b or r // b == c // b``; the literal
  band of Section 1 (``|r - c| <= b``) is :func:`pred_band`, used for the
  Fig. 3 check and for Lemma 4.1;
* the graph of A_i is the symmetric pattern of its remaining entries with
  self-loops dropped; deg is the number of distinct neighbours;
* ties: head by (degree desc, id asc); trees by (size desc, vertices
  without remaining entries last, smallest id asc) so that the touched rows
  form a prefix (Section 3, x-compacting: the non-zero rows are collected at
  the top); a tree is rooted at its smallest id; siblings by (subtree size
  asc, id asc);
* the U(0,1) weights of Section 4.3 are replaced by 64-bit keys
  w(u, v) = splitmix64(splitmix64(seed + i) XOR (u * 2^32 + v)) for u < v;
  splitmix64 is a bijection, so distinct edges get distinct keys and the
  minimum spanning forest is unique;
* the stop rule "until nnz(A_i) <= 2b" is read as "until no entry is left";
* every entry of A (diagonal included, values carried with their own (r, c))
  lands in exactly one B_i.

Parity of this module is pinned by tests/test_oracle_decompose.py.
"""
from __future__ import annotations

import dataclasses

import numpy as np

MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea, Flood 2014), vectorised over uint64.

    z = x + 0x9E3779B97F4A7C15; z = (z ^ z>>30) * 0xBF58476D1CE4E5B9;
    z = (z ^ z>>27) * 0x94D049BB133111EB; return z ^ z>>31 (all mod 2^64).
    """
    z = np.asarray(x, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def edge_keys(u: np.ndarray, v: np.ndarray, seed: int, level: int) -> np.ndarray:
    """Random edge weights of Section 4.3 step 1, as distinct 64-bit keys (u < v)."""
    salt = splitmix64(np.array([(seed + level) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
    pair = (np.asarray(u, dtype=np.uint64) << np.uint64(32)) | np.asarray(v, dtype=np.uint64)
    return splitmix64(pair ^ salt)


def pred_block(r, c, b: int):
    """Block-diagonal arrow shape (Section 3.1, Fig. 2): head rows, head columns, diagonal tiles."""
    r = np.asarray(r)
    c = np.asarray(c)
    return (r < b) | (c < b) | ((r // b) == (c // b))


def pred_band(r, c, b: int):
    """Arrow-width b as defined in Section 1 (0-based): r < b or c < b or |r - c| <= b."""
    r = np.asarray(r)
    c = np.asarray(c)
    return (r < b) | (c < b) | (np.abs(r - c) <= b)


def undirected_edges(rows: np.ndarray, cols: np.ndarray, n: int):
    """Edges {u < v} of the symmetric pattern of the entries, self-loops dropped."""
    off = rows != cols
    u = np.minimum(rows[off], cols[off]).astype(np.int64)
    v = np.maximum(rows[off], cols[off]).astype(np.int64)
    key = np.unique(u * n + v)
    return key // n, key % n


def degrees(n: int, eu: np.ndarray, ev: np.ndarray) -> np.ndarray:
    return np.bincount(eu, minlength=n) + np.bincount(ev, minlength=n)


def select_head(deg: np.ndarray, b: int) -> np.ndarray:
    """Step 1 of LA-Decompose: the min(b, n) vertices of highest degree, ties by id."""
    n = deg.shape[0]
    order = np.lexsort((np.arange(n), -deg.astype(np.int64)))
    return order[: min(b, n)]


def kruskal_msf(n: int, eu: np.ndarray, ev: np.ndarray, w: np.ndarray):
    """Minimum spanning forest by Kruskal (edges by increasing key, union-find)."""
    parent = list(range(n))
    size = [1] * n

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    out = []
    for e in np.argsort(w, kind="stable"):
        a, c = int(eu[e]), int(ev[e])
        ra, rc = find(a), find(c)
        if ra == rc:
            continue
        if size[ra] < size[rc]:
            ra, rc = rc, ra
        parent[rc] = ra
        size[ra] += size[rc]
        out.append((a, c))
    return out


def smallest_first_preorder(adj, root: int):
    """Section 4.4: root first, then each child subtree in increasing size (ties by id)."""
    parent = {root: -1}
    order = [root]
    k = 0
    while k < len(order):                      # BFS for parents
        x = order[k]
        k += 1
        for y in adj[x]:
            if y not in parent:
                parent[y] = x
                order.append(y)
    size = {x: 1 for x in order}
    for x in reversed(order[1:]):
        size[parent[x]] += size[x]
    children = {x: [] for x in order}
    for x in order[1:]:
        children[parent[x]].append(x)
    out = []
    stack = [root]
    while stack:
        x = stack.pop()
        out.append(x)
        ch = sorted(children[x], key=lambda y: (size[y], y))
        stack.extend(reversed(ch))
    return out


def forest_arrangement(n: int, is_head: np.ndarray, forest_edges, touched=None):
    """Step 3 of Section 4.3: trees in decreasing size, each smallest-first.

    Ties between trees of equal size: trees whose vertices hold no remaining
    entry go last (Section 3: the non-zero rows can be collected at the top),
    then by smallest id.  Only single-vertex trees can be untouched.
    """
    if touched is None:
        touched = np.ones(n, dtype=bool)
    adj = [[] for _ in range(n)]
    for a, c in forest_edges:
        adj[a].append(c)
        adj[c].append(a)
    seen = np.zeros(n, dtype=bool)
    trees = []
    for s in range(n):                          # ascending scan: s is its tree's smallest id
        if is_head[s] or seen[s]:
            continue
        comp = [s]
        seen[s] = True
        k = 0
        while k < len(comp):
            x = comp[k]
            k += 1
            for y in adj[x]:
                if not seen[y]:
                    seen[y] = True
                    comp.append(y)
        trees.append((len(comp), 0 if touched[s] else 1, s))
    trees.sort(key=lambda t: (-t[0], t[1], t[2]))
    out = []
    for _, _, root in trees:
        out.extend(smallest_first_preorder(adj, root))
    return np.asarray(out, dtype=np.int64)


@dataclasses.dataclass
class Level:
    """One term P_{pi_i} B_i P_{pi_i}^T: B_i in CSR over positions 0..n-1."""
    n: int
    b: int
    perm: np.ndarray      # vertex -> position  (pi_i)
    iperm: np.ndarray     # position -> vertex
    rowptr: np.ndarray    # int64[n+1]
    colidx: np.ndarray    # int64[nnz]
    values: np.ndarray    # float64[nnz]
    n_active: int         # 1 + largest position touched by an entry

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.values, self.colidx, self.rowptr), shape=(self.n, self.n))


def split_step(n: int, rows, cols, vals, perm, b: int, predicate=pred_block):
    """Steps 3-4 of LA-Decompose: entries inside the arrow shape of P^T A_i P form B_i.

    Returns (Level-CSR arrays, n_active, mask of entries taken).
    """
    pr = perm[rows]
    pc = perm[cols]
    take = predicate(pr, pc, b)
    r, c, x = pr[take], pc[take], vals[take]
    o = np.lexsort((c, r))
    r, c, x = r[o], c[o], x[o]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=rowptr[1:])
    n_active = int(max(r.max(), c.max()) + 1) if r.size else 0
    return (rowptr, c.astype(np.int64), x.astype(np.float64)), n_active, take


def la_decompose(A, b: int, seed: int = 0, predicate=pred_block, max_levels: int = 10_000):
    """LA-Decompose(A, b) of Section 4.1 with the arrangement of Sections 4.3-4.4."""
    if b < 2:
        raise ValueError("LA-Decompose needs b >= 2")
    n = A.n
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(A.rowptr))
    cols = np.asarray(A.colidx, dtype=np.int64)
    vals = np.asarray(A.values, dtype=np.float64)
    levels = []
    i = 0
    while rows.size:
        if i >= max_levels:
            raise RuntimeError("too many levels")
        eu, ev = undirected_edges(rows, cols, n)
        deg = degrees(n, eu, ev)
        head = select_head(deg, b)                               # step 1
        is_head = np.zeros(n, dtype=bool)
        is_head[head] = True
        keep = ~is_head[eu] & ~is_head[ev]                       # G_i' = G_i[V \ V^h]
        gu, gv = eu[keep], ev[keep]
        w = edge_keys(gu, gv, seed, i)                           # Section 4.3 step 1
        forest = kruskal_msf(n, gu, gv, w)                       # Section 4.3 step 2
        touched = np.zeros(n, dtype=bool)
        touched[rows] = True
        touched[cols] = True
        rest = forest_arrangement(n, is_head, forest, touched)   # Section 4.3 step 3 + 4.4
        iperm = np.concatenate([head.astype(np.int64), rest])    # step 2: concatenate
        perm = np.empty(n, dtype=np.int64)
        perm[iperm] = np.arange(n, dtype=np.int64)
        (rp, ci, vv), n_act, take = split_step(n, rows, cols, vals, perm, b, predicate)  # step 3
        levels.append(Level(n, b, perm, iperm, rp, ci, vv, n_act))
        rows, cols, vals = rows[~take], cols[~take], vals[~take]  # step 4
        i += 1
    return levels


def arrow_shape(rows, cols, b: int):
    """Where entries at positions (rows, cols) sit under the b x b tiling of Section 3.1 /
    Fig. 2: (entries in a head row or head column, the other entries, distinct non-zero
    b x b tiles).  The first two are the 'pruned' part and the band that Section 6 reads off
    the decompositions (Fig. 1); the tile count is what it compares against 1.5D blocks."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    head = (rows < b) | (cols < b)
    tiles = {(int(r) // b, int(c) // b) for r, c in zip(rows, cols)}
    return int(np.count_nonzero(head)), int(np.count_nonzero(~head)), len(tiles)


def level_shape(L: Level):
    """arrow_shape of the entries of B_i (positions of level i)."""
    rows = np.repeat(np.arange(L.n, dtype=np.int64), np.diff(L.rowptr))
    return arrow_shape(rows, L.colidx, L.b)


def count_tiles(A, b: int) -> int:
    """Distinct non-zero b x b tiles of A in its own order (equally sized 1.5D blocks)."""
    rows = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.rowptr))
    return arrow_shape(rows, A.colidx, b)[2]
