// Host side of the library: LA-Decompose (Section 4.1) with the random spanning forest
// linear arrangement (Section 4.3) and the smallest-first tree layout (Section 4.4),
// followed by the construction of the fused row program that the device kernels run.
//
// Readings of the paper taken here (the same ones the test oracle states):
//   * positions are 0-based, the head is positions 0..b-1;
//   * B_i uses the block-diagonal arrow shape of Section 3.1 / Fig. 2
//     (r < b || c < b || r/b == c/b), or the band of Section 1 (|r-c| <= b) on request;
//   * the graph of A_i is the symmetric pattern of its remaining entries without
//     self-loops, deg(v) = number of distinct remaining neighbours;
//   * head = the b vertices of largest degree, ties by smaller id, in that order;
//   * the U(0,1) weights of Section 4.3 become distinct 64-bit keys
//     w(u,v) = splitmix64(splitmix64(seed + i) ^ (u << 32 | v)), u < v (splitmix64 is a
//     bijection, so the minimum spanning forest is unique);
//   * trees in decreasing size; among single vertices those that still hold an entry
//     (an edge to the head, or a diagonal entry) come first, so the touched rows of
//     every level form a prefix (Section 3: non-zero rows collected at the top); then
//     smallest vertex id; each tree is rooted at its smallest id; siblings in
//     increasing subtree size, ties by id;
//   * levels are built until no entry is left.
//
// The minimum spanning forest is computed with a parallel Boruvka (a component's
// lightest edge is in the unique forest), which agrees with Kruskal because keys are
// distinct.  The arrangement of a tree is computed top-down: a child's position is its
// parent's position + 1 + the sizes of its smaller siblings, which is the smallest-first
// preorder written without recursion.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>
#include <thread>
#include <utility>

#include "arrow_internal.h"

namespace arrow {
namespace {

int g_threads = 1;


// f(begin, end, thread) over [0, n) in g_threads contiguous chunks.
template <class F>
void pfor(int64_t n, F&& f) {
    int T = g_threads;
    if (n < 32768 || T <= 1) {
        if (n > 0) f(int64_t(0), n, 0);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(T);
    for (int t = 0; t < T; ++t) {
        int64_t b = n * t / T, e = n * (t + 1) / T;
        th.emplace_back([&f, b, e, t] { f(b, e, t); });
    }
    for (auto& x : th) x.join();
}

// f(row_begin, row_end, thread) over the rows [0, n) in g_threads chunks of about equal
// entry counts (ptr: entry prefix over the rows, ptr[0] = 0): a power-law matrix keeps most
// of its entries in a few rows, which row-count chunks would hand to one thread.
template <class F>
void pfor_rows(int64_t n, const int64_t* ptr, F&& f) {
    const int64_t total = n > 0 ? ptr[n] : 0;
    const int T = g_threads;
    if (total < 32768 || T <= 1) {
        if (n > 0) f(int64_t(0), n, 0);
        return;
    }
    std::vector<int64_t> cut(T + 1, 0);
    cut[T] = n;
    for (int t = 1; t < T; ++t) {
        const int64_t target = total * t / T;
        const int64_t r = int64_t(std::upper_bound(ptr, ptr + n + 1, target) - ptr) - 1;
        cut[t] = std::min(n, std::max(cut[t - 1], r));
    }
    std::vector<std::thread> th;
    th.reserve(T);
    for (int t = 0; t < T; ++t)
        if (cut[t + 1] > cut[t]) th.emplace_back([&f, &cut, t] { f(cut[t], cut[t + 1], t); });
    for (auto& x : th) x.join();
}

// Order-preserving parallel filter: out receives emit(i) for every i with keep(i).
template <class Vec, class Keep, class Emit>
void pfilter(int64_t n, Vec& out, Keep&& keep, Emit&& emit) {
    int T_ = (n < 32768) ? 1 : g_threads;
    std::vector<int64_t> cnt(T_ + 1, 0);
    auto count = [&](int64_t b, int64_t e, int t) {
        int64_t c = 0;
        for (int64_t i = b; i < e; ++i) c += keep(i) ? 1 : 0;
        cnt[t + 1] = c;
    };
    if (T_ == 1) count(0, n, 0); else pfor(n, count);
    for (int t = 0; t < T_; ++t) cnt[t + 1] += cnt[t];
    out.resize(cnt[T_]);
    auto fill = [&](int64_t b, int64_t e, int t) {
        int64_t o = cnt[t];
        for (int64_t i = b; i < e; ++i)
            if (keep(i)) out[o++] = emit(i);
    };
    if (T_ == 1) fill(0, n, 0); else pfor(n, fill);
}

inline uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <class T>
inline void atomic_min_relaxed(T& slot, T v) {
    std::atomic_ref<T> a(slot);
    T cur = a.load(std::memory_order_relaxed);
    while (v < cur && !a.compare_exchange_weak(cur, v, std::memory_order_relaxed)) {
    }
}

template <class T>
inline T aload(T& slot) { return std::atomic_ref<T>(slot).load(std::memory_order_relaxed); }
template <class T>
inline void astore(T& slot, T v) { std::atomic_ref<T>(slot).store(v, std::memory_order_relaxed); }

inline bool pred_block(int64_t r, int64_t c, int64_t b) { return r < b || c < b || (r / b) == (c / b); }
inline bool pred_band(int64_t r, int64_t c, int64_t b) {
    return r < b || c < b || (r > c ? r - c : c - r) <= b;
}

struct Ent {
    int32_t r, c;  // vertices
    int32_t s;     // index of the entry in the symmetric pattern
};

int validate(const arrow_csr* A) {
    if (!A) { set_error("arrow_decompose: A is NULL"); return ARROW_EINVAL; }
    if (A->n < 0 || A->n >= (int64_t(1) << 31)) { set_error("arrow_decompose: n out of range [0, 2^31)"); return ARROW_EINVAL; }
    if (A->nnz < 0 || A->nnz >= (int64_t(1) << 31)) { set_error("arrow_decompose: nnz out of range [0, 2^31)"); return ARROW_EINVAL; }
    if (A->n > 0 && !A->rowptr) { set_error("arrow_decompose: rowptr is NULL"); return ARROW_EINVAL; }
    if (A->nnz > 0 && (!A->colidx || !A->values)) { set_error("arrow_decompose: colidx/values NULL"); return ARROW_EINVAL; }
    if (A->n == 0) {
        if (A->nnz != 0) { set_error("arrow_decompose: nnz > 0 with n == 0"); return ARROW_EINVAL; }
        return ARROW_OK;
    }
    if (A->rowptr[0] != 0 || A->rowptr[A->n] != A->nnz) {
        set_error("arrow_decompose: rowptr[0] must be 0 and rowptr[n] must be nnz");
        return ARROW_EINVAL;
    }
    std::atomic<int> bad{0};
    pfor(A->n, [&](int64_t b, int64_t e, int) {
        for (int64_t r = b; r < e; ++r) {
            int64_t s = A->rowptr[r], t = A->rowptr[r + 1];
            if (t < s || s < 0 || t > A->nnz) { bad.store(1); return; }
            int64_t prev = -1;
            for (int64_t j = s; j < t; ++j) {
                int64_t c = A->colidx[j];
                if (c < 0 || c >= A->n) { bad.store(2); return; }
                if (c <= prev) { bad.store(3); return; }
                prev = c;
            }
        }
    });
    switch (bad.load()) {
        case 1: set_error("arrow_decompose: rowptr is not non-decreasing within [0, nnz]"); return ARROW_EINVAL;
        case 2: set_error("arrow_decompose: column index out of range"); return ARROW_EINVAL;
        case 3: set_error("arrow_decompose: column indices must be strictly increasing in each row"); return ARROW_EINVAL;
        default: return ARROW_OK;
    }
}

// Symmetric pattern S = pattern(A) U pattern(A^T).  If A is already structurally
// symmetric S is A's pattern (a2s empty = identity).
struct SymPattern {
    const int64_t* ptr = nullptr;
    const int32_t* col = nullptr;
    int64_t nnz = 0;
    std::vector<int64_t> own_ptr;
    std::vector<int32_t> own_col;
    std::vector<int32_t> a2s;  // A entry -> S entry (empty when identity)
};

bool row_has(const int64_t* ptr, const int32_t* col, int64_t r, int32_t c) {
    const int32_t* b = col + ptr[r];
    const int32_t* e = col + ptr[r + 1];
    const int32_t* it = std::lower_bound(b, e, c);
    return it != e && *it == c;
}

void build_sym(const arrow_csr* A, SymPattern& S) {
    const int64_t n = A->n;
    // structurally symmetric iff every entry above the diagonal has its mirror below and
    // both sides hold as many entries (the mirror map is then a bijection); the mirror of
    // (r, c), c > r, is searched in row c, rarely a hub row when hubs have small ids
    // (chunks of entries, not of rows: a power-law matrix keeps most entries in a few rows)
    std::atomic<bool> sym{true};
    std::atomic<int64_t> upper{0}, lower{0};
    pfor(A->nnz, [&](int64_t b, int64_t e, int) {
        int64_t up = 0, lo = 0;
        int64_t r = int64_t(std::upper_bound(A->rowptr, A->rowptr + n + 1, b) - A->rowptr) - 1;
        for (int64_t j = b; j < e; ++j) {
            while (A->rowptr[r + 1] <= j) ++r;
            const int32_t c = A->colidx[j];
            if (c > r) {
                ++up;
                if (!row_has(A->rowptr, A->colidx, c, int32_t(r))) { sym.store(false); return; }
            } else if (c < r) {
                ++lo;
            }
            if ((j & 4095) == 0 && !sym.load(std::memory_order_relaxed)) return;
        }
        upper.fetch_add(up);
        lower.fetch_add(lo);
    });
    if (sym.load() && upper.load() == lower.load()) {
        S.ptr = A->rowptr;
        S.col = A->colidx;
        S.nnz = A->nnz;
        return;
    }
    // transpose pattern (rows ascending inside each column list)
    std::vector<int64_t> tptr(n + 1, 0);
    for (int64_t j = 0; j < A->nnz; ++j) tptr[A->colidx[j] + 1]++;
    for (int64_t i = 0; i < n; ++i) tptr[i + 1] += tptr[i];
    std::vector<int32_t> tcol(A->nnz);
    {
        std::vector<int64_t> pos(tptr.begin(), tptr.end() - 1);
        for (int64_t r = 0; r < n; ++r)
            for (int64_t j = A->rowptr[r]; j < A->rowptr[r + 1]; ++j) tcol[pos[A->colidx[j]]++] = int32_t(r);
    }
    // merge row r of A with row r of A^T
    S.own_ptr.assign(n + 1, 0);
    for (int64_t r = 0; r < n; ++r) {
        int64_t a = A->rowptr[r], ae = A->rowptr[r + 1], t = tptr[r], te = tptr[r + 1], m = 0;
        while (a < ae || t < te) {
            if (t >= te || (a < ae && A->colidx[a] < tcol[t])) ++a;
            else if (a >= ae || tcol[t] < A->colidx[a]) ++t;
            else { ++a; ++t; }
            ++m;
        }
        S.own_ptr[r + 1] = S.own_ptr[r] + m;
    }
    S.nnz = S.own_ptr[n];
    S.own_col.resize(S.nnz);
    S.a2s.resize(A->nnz);
    for (int64_t r = 0; r < n; ++r) {
        int64_t a = A->rowptr[r], ae = A->rowptr[r + 1], t = tptr[r], te = tptr[r + 1], o = S.own_ptr[r];
        while (a < ae || t < te) {
            if (t >= te || (a < ae && A->colidx[a] < tcol[t])) { S.a2s[a] = int32_t(o); S.own_col[o++] = A->colidx[a++]; }
            else if (a >= ae || tcol[t] < A->colidx[a]) { S.own_col[o++] = tcol[t++]; }
            else { S.a2s[a] = int32_t(o); S.own_col[o++] = A->colidx[a++]; ++t; }
        }
    }
    S.ptr = S.own_ptr.data();
    S.col = S.own_col.data();
}

// Step 1 of LA-Decompose: min(b, n) vertices by (degree desc, id asc).
std::vector<int32_t> select_head(const std::vector<int32_t>& deg, int64_t b) {
    const int64_t n = int64_t(deg.size());
    const int64_t hb = std::min<int64_t>(b, n);
    // degree histogram (per-chunk maxima and counts, summed in chunk order)
    std::vector<int32_t> cmax(size_t(g_threads), 0);
    pfor(n, [&](int64_t lo, int64_t hi, int t) {
        int32_t m = 0;
        for (int64_t v = lo; v < hi; ++v) m = std::max(m, deg[v]);
        cmax[size_t(t)] = m;
    });
    const int32_t maxdeg = *std::max_element(cmax.begin(), cmax.end());
    std::vector<std::vector<int64_t>> ccnt(static_cast<size_t>(g_threads));
    pfor(n, [&](int64_t lo, int64_t hi, int t) {
        std::vector<int64_t>& c = ccnt[size_t(t)];
        c.assign(size_t(maxdeg) + 2, 0);
        for (int64_t v = lo; v < hi; ++v) c[size_t(deg[v])]++;
    });
    std::vector<int64_t> cnt(size_t(maxdeg) + 2, 0);
    for (const auto& c : ccnt)
        for (size_t d = 0; d < c.size(); ++d) cnt[d] += c[d];
    // threshold D: #(deg > D) < hb <= #(deg >= D)
    int64_t above = 0;
    int32_t D = maxdeg;
    for (;; --D) {
        if (above + cnt[D] >= hb || D == 0) break;
        above += cnt[D];
    }
    std::vector<int32_t> head;
    pfilter(n, head, [&](int64_t v) { return deg[v] > D; }, [&](int64_t v) { return int32_t(v); });
    std::sort(head.begin(), head.end(), [&](int32_t x, int32_t y) {
        return deg[x] != deg[y] ? deg[x] > deg[y] : x < y;
    });
    if (int64_t(head.size()) < hb) {
        std::vector<int32_t> tie;   // degree exactly D, in id order
        pfilter(n, tie, [&](int64_t v) { return deg[v] == D; }, [&](int64_t v) { return int32_t(v); });
        for (size_t i = 0; i < tie.size() && int64_t(head.size()) < hb; ++i) head.push_back(tie[i]);
    }
    return head;
}

// Minimum spanning forest of the edge set (unique keys) by parallel Boruvka.
// On return comp[v] is the representative of v's tree (every vertex, isolated ones
// are their own representative) and `forest` holds the forest edges (any order).
void boruvka(int64_t n, uvec<int32_t> eu, uvec<int32_t> ev, uvec<uint64_t> ew,
             std::vector<int32_t>& comp, std::vector<std::pair<int32_t, int32_t>>& forest) {
    comp.resize(n);
    std::iota(comp.begin(), comp.end(), 0);
    std::vector<uint64_t> best(n);
    std::vector<int32_t> link(n);
    std::iota(link.begin(), link.end(), 0);
    forest.assign(std::min<int64_t>(n, int64_t(eu.size())), {0, 0});
    std::atomic<int64_t> fcount{0};
    const uint64_t NONE = ~uint64_t(0);
    // the round's edges live in (U, Vv, W)[0, m); the filter moves the survivors to the other
    // buffer of each pair (allocated once, never zero-filled: it is written before it is read)
    const int64_t m0 = int64_t(eu.size());
    std::unique_ptr<int32_t[]> su(new int32_t[size_t(std::max<int64_t>(1, m0))]);
    std::unique_ptr<int32_t[]> sv(new int32_t[size_t(std::max<int64_t>(1, m0))]);
    std::unique_ptr<uint64_t[]> sw(new uint64_t[size_t(std::max<int64_t>(1, m0))]);
    int32_t *U = eu.data(), *Vv = ev.data(), *U2 = su.get(), *V2 = sv.get();
    uint64_t *W = ew.data(), *W2 = sw.get();
    std::vector<int32_t> ecu(static_cast<size_t>(m0)), ecv(static_cast<size_t>(m0));   // edge ends' components this round
    int64_t m = m0;
    while (m > 0) {
        pfor(m, [&](int64_t b, int64_t e, int) {
            for (int64_t i = b; i < e; ++i) {
                int32_t cu = comp[U[i]], cv = comp[Vv[i]];
                ecu[i] = cu; ecv[i] = cv;
                // resets written only where they change something: a large component is the
                // end of many edges, and unconditional stores would bounce its cache line
                // between all threads
                if (aload(best[cu]) != NONE) astore(best[cu], NONE);
                if (aload(best[cv]) != NONE) astore(best[cv], NONE);
                if (aload(link[cu]) != cu) astore(link[cu], cu);
                if (aload(link[cv]) != cv) astore(link[cv], cv);
            }
        });
        pfor(m, [&](int64_t b, int64_t e, int) {
            for (int64_t i = b; i < e; ++i) {
                int32_t cu = ecu[i], cv = ecv[i];
                if (cu == cv) continue;
                atomic_min_relaxed(best[cu], W[i]);
                atomic_min_relaxed(best[cv], W[i]);
            }
        });
        // each chunk keeps its selected edges and appends them in one reservation (one shared
        // counter per chunk, not per edge: the forest is a set, its order is not used)
        std::atomic<int64_t> selected{0};
        pfor(m, [&](int64_t b, int64_t e, int) {
            std::vector<std::pair<int32_t, int32_t>> mine;
            for (int64_t i = b; i < e; ++i) {
                int32_t cu = ecu[i], cv = ecv[i];
                if (cu == cv) continue;
                bool a = aload(best[cu]) == W[i], c = aload(best[cv]) == W[i];
                if (!a && !c) continue;
                mine.push_back({U[i], Vv[i]});
                if (a) astore(link[cu], cv);
                if (c) astore(link[cv], cu);
            }
            if (!mine.empty()) {
                const int64_t at = fcount.fetch_add(int64_t(mine.size()), std::memory_order_relaxed);
                std::copy(mine.begin(), mine.end(), forest.begin() + at);
                selected.fetch_add(int64_t(mine.size()));
            }
        });
        if (selected.load() == 0) break;
        // mutual choices form 2-cycles: the smaller label becomes the root
        pfor(m, [&](int64_t b, int64_t e, int) {
            for (int64_t i = b; i < e; ++i) {
                for (int32_t c : {ecu[i], ecv[i]}) {
                    int32_t l = aload(link[c]);
                    if (l != c && aload(link[l]) == c && c < l) astore(link[c], c);
                }
            }
        });
        // pointer jumping to the roots
        pfor(m, [&](int64_t b, int64_t e, int) {
            for (int64_t i = b; i < e; ++i) {
                for (int32_t c : {ecu[i], ecv[i]}) {
                    for (;;) {
                        int32_t l = aload(link[c]);
                        int32_t ll = aload(link[l]);
                        if (l == ll) break;
                        astore(link[c], ll);
                    }
                }
            }
        });
        // the edge ends take their component's new root (one step after the jumping); the
        // other vertices follow their links once, after the last round
        pfor(m, [&](int64_t b, int64_t e, int) {
            for (int64_t i = b; i < e; ++i) {
                const int32_t ru = aload(link[ecu[i]]), rv = aload(link[ecv[i]]);
                if (aload(comp[U[i]]) != ru) astore(comp[U[i]], ru);
                if (aload(comp[Vv[i]]) != rv) astore(comp[Vv[i]], rv);
            }
        });
        // drop edges inside one component (order kept: per-chunk counts, then each chunk
        // writes its survivors at its offset)
        std::vector<int64_t> cnt(size_t(g_threads) + 1, 0);
        pfor(m, [&](int64_t b, int64_t e, int t) {
            int64_t c = 0;
            for (int64_t i = b; i < e; ++i) c += comp[U[i]] != comp[Vv[i]];
            cnt[size_t(t) + 1] = c;
        });
        for (int t = 0; t < g_threads; ++t) cnt[size_t(t) + 1] += cnt[size_t(t)];
        pfor(m, [&](int64_t b, int64_t e, int t) {
            int64_t o = cnt[size_t(t)];
            for (int64_t i = b; i < e; ++i)
                if (comp[U[i]] != comp[Vv[i]]) { U2[o] = U[i]; V2[o] = Vv[i]; W2[o] = W[i]; ++o; }
        });
        m = cnt[size_t(g_threads)];
        std::swap(U, U2);
        std::swap(Vv, V2);
        std::swap(W, W2);
    }
    // every vertex to its tree's representative: a component's link, once it stopped being a
    // root, points at the root that absorbed it, so the chains end at the final roots
    pfor(n, [&](int64_t b, int64_t e, int) {
        for (int64_t v = b; v < e; ++v) {
            int32_t r = comp[v];
            for (;;) { const int32_t l = link[r]; if (l == r) break; r = l; }
            comp[v] = r;
        }
    });
    forest.resize(fcount.load());
}

// Sections 4.3 step 3 and 4.4: trees in decreasing size, each in smallest-first order,
// after the head.  Writes perm (vertex -> position) and iperm.
void arrange(int64_t n, const std::vector<int32_t>& head, const std::vector<uint8_t>& is_head,
             const std::vector<uint8_t>& touched, const std::vector<int32_t>& comp, const std::vector<std::pair<int32_t, int32_t>>& forest,
             std::vector<int32_t>& perm, std::vector<int32_t>& iperm) {
    const int64_t hb = int64_t(head.size());
    perm.assign(n, -1);
    iperm.assign(n, -1);
    for (int64_t p = 0; p < hb; ++p) { perm[head[p]] = int32_t(p); iperm[p] = head[p]; }

    // tree sizes and smallest ids, keyed by representative
    // (one pass in vertex order: the first vertex seen of a tree is its smallest id; a
    // parallel form with atomics contended on the single counter of a spanning tree)
    std::vector<int32_t> tsize(n, 0), tmin(n, INT32_MAX);
    for (int64_t v = 0; v < n; ++v) {
        if (is_head[v]) continue;
        const int32_t c = comp[v];
        if (tsize[c]++ == 0) tmin[c] = int32_t(v);
    }
    struct Tree { int32_t size, root; int64_t start; };
    std::vector<Tree> multi;
    pfilter(n, multi, [&](int64_t v) { return !is_head[v] && comp[v] == v && tsize[v] >= 2; },
            [&](int64_t v) { return Tree{tsize[v], tmin[v], 0}; });
    std::sort(multi.begin(), multi.end(), [](const Tree& x, const Tree& y) {
        return x.size != y.size ? x.size > y.size : x.root < y.root;
    });
    int64_t pos = hb;
    for (auto& t : multi) { t.start = pos; pos += t.size; }
    // single vertices: those holding an entry first, each group in id order (per-chunk counts,
    // then every chunk writes its own consecutive positions)
    {
        auto single = [&](int64_t v) { return !is_head[v] && tsize[comp[v]] == 1; };
        std::vector<int64_t> c0(g_threads + 1, 0), c1(g_threads + 1, 0);
        pfor(n, [&](int64_t b, int64_t e, int t) {
            int64_t a = 0, z = 0;
            for (int64_t v = b; v < e; ++v)
                if (single(v)) ++(touched[v] ? a : z);
            c0[t + 1] = a;
            c1[t + 1] = z;
        });
        for (int t = 0; t < g_threads; ++t) { c0[t + 1] += c0[t]; c1[t + 1] += c1[t]; }
        const int64_t p0 = pos, p1 = pos + c0[g_threads];
        pfor(n, [&](int64_t b, int64_t e, int t) {
            int64_t a = p0 + c0[t], z = p1 + c1[t];
            for (int64_t v = b; v < e; ++v)
                if (single(v)) {
                    int64_t& q = touched[v] ? a : z;
                    perm[v] = int32_t(q);
                    iperm[q] = int32_t(v);
                    ++q;
                }
        });
        pos = p1 + c1[g_threads];
    }

    // forest adjacency (the order inside a vertex's list does not matter: the tree, its
    // subtree sizes and the sorted child order it yields are the same)
    std::vector<int64_t> fptr(n + 1, 0);
    const int64_t nf = int64_t(forest.size());
    pfor(nf, [&](int64_t b, int64_t e, int) {
        for (int64_t i = b; i < e; ++i) {
            std::atomic_ref<int64_t>(fptr[forest[i].first + 1]).fetch_add(1, std::memory_order_relaxed);
            std::atomic_ref<int64_t>(fptr[forest[i].second + 1]).fetch_add(1, std::memory_order_relaxed);
        }
    });
    {
        std::vector<int64_t> part(g_threads + 1, 0);
        pfor(n, [&](int64_t b, int64_t e, int t) {
            int64_t sum = 0;
            for (int64_t v = b; v < e; ++v) sum += fptr[v + 1];
            part[t + 1] = sum;
        });
        for (int t = 0; t < g_threads; ++t) part[t + 1] += part[t];
        pfor(n, [&](int64_t b, int64_t e, int t) {
            int64_t run = part[t];
            for (int64_t v = b; v < e; ++v) { run += fptr[v + 1]; fptr[v + 1] = run; }
        });
    }
    std::vector<int32_t> fadj(fptr[n]);
    {
        std::vector<int64_t> fill(fptr.begin(), fptr.end() - 1);
        pfor(nf, [&](int64_t b, int64_t e, int) {
            for (int64_t i = b; i < e; ++i) {
                const int32_t u = forest[i].first, v = forest[i].second;
                fadj[std::atomic_ref<int64_t>(fill[u]).fetch_add(1, std::memory_order_relaxed)] = v;
                fadj[std::atomic_ref<int64_t>(fill[v]).fetch_add(1, std::memory_order_relaxed)] = u;
            }
        });
    }
    // Each tree is laid out in its own breadth-first numbering: a vertex's children are
    // appended together, so they form one contiguous range of that numbering, parents come
    // before children, and the subtree sizes and positions are computed over small dense
    // arrays instead of by vertex id (the giant spanning tree of a mesh spans most of n).
    std::atomic<int64_t> next{0};
    auto worker = [&] {
        std::vector<int32_t> order, par, kid0, subq;
        std::vector<int64_t> posq;
        std::vector<int32_t> kids;
        for (;;) {
            int64_t ti = next.fetch_add(1);
            if (ti >= int64_t(multi.size())) return;
            const Tree& t = multi[ti];
            order.assign(1, t.root);
            par.assign(1, -1);
            kid0.clear();
            for (size_t q = 0; q < order.size(); ++q) {
                const int32_t v = order[q];
                const int32_t pv = par[q] >= 0 ? order[size_t(par[q])] : -1;
                kid0.push_back(int32_t(order.size()));
                for (int64_t j = fptr[v]; j < fptr[v + 1]; ++j) {
                    const int32_t u = fadj[j];
                    if (u == pv) continue;
                    order.push_back(u);
                    par.push_back(int32_t(q));
                }
            }
            const size_t sz = order.size();
            kid0.push_back(int32_t(sz));
            subq.assign(sz, 1);
            for (size_t q = sz; q-- > 1;) subq[size_t(par[q])] += subq[q];
            posq.assign(sz, 0);
            posq[0] = t.start;
            for (size_t q = 0; q < sz; ++q) {
                kids.clear();
                for (int32_t c = kid0[q]; c < kid0[q + 1]; ++c) kids.push_back(c);
                std::sort(kids.begin(), kids.end(), [&](int32_t x, int32_t y) {
                    return subq[x] != subq[y] ? subq[x] < subq[y] : order[x] < order[y];
                });
                int64_t run = posq[q] + 1;
                for (int32_t c : kids) { posq[c] = run; run += subq[c]; }
            }
            for (size_t q = 0; q < sz; ++q) {
                perm[order[q]] = int32_t(posq[q]);
                iperm[posq[q]] = order[q];
            }
        }
    };
    int T = std::max(1, std::min<int>(g_threads, int(multi.size())));
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t) th.emplace_back(worker);
    for (auto& x : th) x.join();
}

}  // namespace

void build_tiles(arrow_handle_s* h, int tile_rows, int tile_nnz) {
    // consecutive rows, at most tile_rows rows and tile_nnz entries (short rows only)
    const int64_t n = h->n;
    h->tile_row.assign(1, 0);
    h->tile_ent.assign(1, 0);
    if (h->f_rowptr.empty()) return;
    int64_t r = 0;
    while (r < n) {
        int64_t r1 = r, ent = 0;
        while (r1 < n && r1 - r < tile_rows) {
            int64_t l = h->f_rowptr[r1 + 1] - h->f_rowptr[r1];
            if (ent + l > tile_nnz) break;
            ent += l;
            ++r1;
        }
        h->tile_row.push_back(int32_t(r1));
        h->tile_ent.push_back(h->f_rowptr[r1]);
        r = r1;
    }
    h->tune.tile_rows = tile_rows;
    h->tune.tile_nnz = tile_nnz;
}

// Host fault injection for the tests of the allocation-failure path: with the environment
// variable ARROW_INJECT_HOST_ALLOC_FAILURE=k the decomposition throws std::bad_alloc as it
// starts level k, as a failed allocation there would (arrow_decompose turns it into
// ARROW_ENOMEM and frees the partial handle).  Unset in normal use.
static int injected_alloc_failure_level() {
    const char* s = std::getenv("ARROW_INJECT_HOST_ALLOC_FAILURE");
    return s && *s ? std::atoi(s) : -1;
}

int decompose_host(arrow_handle_s* h, const arrow_csr* A, int64_t b, const arrow_opts& o) {
    auto t0 = std::chrono::steady_clock::now();
    const int fail_level = injected_alloc_failure_level();
    g_threads = o.nthreads > 0 ? o.nthreads : int(std::max(1u, std::thread::hardware_concurrency()));
    g_threads = std::min(g_threads, 256);
    if (b < 2) { set_error("arrow_decompose: b must be >= 2 (Section 4.1)"); return ARROW_EINVAL; }
    if (o.predicate != ARROW_PRED_BLOCK && o.predicate != ARROW_PRED_BAND) {
        set_error("arrow_decompose: unknown predicate");
        return ARROW_EINVAL;
    }
    if (o.value_dtype < ARROW_F32 || o.value_dtype > ARROW_F16) {
        set_error("arrow_decompose: unknown value_dtype");
        return ARROW_EINVAL;
    }
    int rc = validate(A);
    if (rc != ARROW_OK) return rc;
    const int64_t n = A->n, nnz = A->nnz;
    const int max_levels = o.max_levels > 0 ? std::min(o.max_levels, 254) : 254;
    h->n = n; h->nnz = nnz; h->b = b; h->opts = o;
    // the input copy, in parallel chunks (first touch of gigabytes of new pages)
    h->rowptr.resize(n + 1);
    h->colidx.resize(nnz);
    h->values.resize(nnz);
    pfor(n + 1, [&](int64_t bb, int64_t e, int) {
        std::memcpy(h->rowptr.data() + bb, A->rowptr + bb, size_t(e - bb) * sizeof(int64_t));
    });
    pfor(nnz, [&](int64_t bb, int64_t e, int) {
        std::memcpy(h->colidx.data() + bb, A->colidx + bb, size_t(e - bb) * sizeof(int32_t));
        std::memcpy(h->values.data() + bb, A->values + bb, size_t(e - bb) * sizeof(double));
    });

    SymPattern S;
    build_sym(A, S);
    if (S.nnz >= (int64_t(1) << 31)) { set_error("arrow_decompose: symmetric pattern too large"); return ARROW_EINVAL; }

    std::vector<uint8_t> lvlS(S.nnz, 255);
    uvec<Ent> act(S.nnz);
    pfor_rows(n, S.ptr, [&](int64_t bb, int64_t e, int) {
        for (int64_t r = bb; r < e; ++r)
            for (int64_t j = S.ptr[r]; j < S.ptr[r + 1]; ++j) act[j] = {int32_t(r), S.col[j], int32_t(j)};
    });
    const bool band = o.predicate == ARROW_PRED_BAND;
    std::vector<int32_t> deg(n);
    std::vector<uint8_t> is_head(n), touched(n);
    // ARROW_DEVICE_DECOMPOSE: the degrees, the edges of G_i' with their keys, the spanning
    // forest and the split run on the current GPU (decompose_device.cu); the head and the tree
    // layout stay here.  The remaining entries then live on the device.
    const bool on_dev = (o.flags & ARROW_DEVICE_DECOMPOSE) != 0;
    struct DdHold {
        DeviceDecomp* d = nullptr;
        ~DdHold() { dd_free(d); }
    } dd;
    if (on_dev) {
        int drc = dd_begin(&dd.d, n, S.nnz, act.data());
        if (drc != ARROW_OK) return drc;
        uvec<Ent>().swap(act);
    }
    int level = 0;
    while (on_dev ? dd_remaining(dd.d) > 0 : !act.empty()) {
        if (level == fail_level) throw std::bad_alloc();
        if (level >= max_levels) {
            set_error("arrow_decompose: more than max_levels levels");
            return ARROW_EINVAL;
        }
        std::fill(deg.begin(), deg.end(), 0);
        std::fill(touched.begin(), touched.end(), 0);
        if (on_dev) {
            int drc = dd_degrees(dd.d, deg.data(), touched.data());
            if (drc != ARROW_OK) return drc;
        }
        // act stays sorted by row (it is filtered in order), so a chunk counts each row's
        // off-diagonal entries in one run; only the rows cut by a chunk boundary are shared
        if (!on_dev) pfor(int64_t(act.size()), [&](int64_t bb, int64_t e, int) {
            for (int64_t i = bb; i < e;) {
                const int32_t r = act[i].r;
                int32_t cnt = 0;
                int64_t j = i;
                for (; j < e && act[j].r == r; ++j) cnt += act[j].c != r;
                astore(touched[r], uint8_t(1));          // S is symmetric: rows cover columns
                if (i == bb || j == e)
                    std::atomic_ref<int32_t>(deg[r]).fetch_add(cnt, std::memory_order_relaxed);
                else
                    deg[r] = cnt;
                i = j;
            }
        });
        std::vector<int32_t> head = select_head(deg, b);
        std::fill(is_head.begin(), is_head.end(), 0);
        for (int32_t v : head) is_head[v] = 1;

        // edges of G_i' = G_i[V \ V^h], keyed by the level's random weights
        const uint64_t salt = splitmix64(o.seed + uint64_t(level));
        std::vector<int32_t> comp;
        std::vector<std::pair<int32_t, int32_t>> forest;
        if (on_dev) {
            int drc = dd_forest(dd.d, is_head.data(), salt, comp, forest);
            if (drc != ARROW_OK) return drc;
        } else {
        uvec<int32_t> eu, ev;
        uvec<uint64_t> ew;
        {
            uvec<int64_t> idx;
            pfilter(int64_t(act.size()), idx,
                    [&](int64_t i) { const Ent& x = act[i]; return x.r < x.c && !is_head[x.r] && !is_head[x.c]; },
                    [&](int64_t i) { return i; });
            eu.resize(idx.size()); ev.resize(idx.size()); ew.resize(idx.size());
            pfor(int64_t(idx.size()), [&](int64_t bb, int64_t e, int) {
                for (int64_t j = bb; j < e; ++j) {
                    const Ent& x = act[idx[j]];
                    eu[j] = x.r; ev[j] = x.c;
                    ew[j] = splitmix64(salt ^ ((uint64_t(uint32_t(x.r)) << 32) | uint64_t(uint32_t(x.c))));
                }
            });
        }
        boruvka(n, std::move(eu), std::move(ev), std::move(ew), comp, forest);
        }
        Level L;
        std::vector<int32_t> iperm;
        arrange(n, head, is_head, touched, comp, forest, L.perm, iperm);

        // steps 3-4: entries inside the arrow shape go to B_i, the rest stays
        const int32_t* perm = L.perm.data();
        if (on_dev) {
            int drc = dd_split(dd.d, perm, b, band, level);
            if (drc != ARROW_OK) return drc;
            h->levels.push_back(std::move(L));
            ++level;
            continue;
        }
        uvec<Ent> rest;
        pfilter(int64_t(act.size()), rest,
                [&](int64_t i) {
                    const Ent& x = act[i];
                    int64_t p = perm[x.r], q = perm[x.c];
                    bool take = band ? pred_band(p, q, b) : pred_block(p, q, b);
                    if (take) lvlS[x.s] = uint8_t(level);
                    return !take;
                },
                [&](int64_t i) { return act[i]; });
        act.swap(rest);
        h->levels.push_back(std::move(L));
        ++level;
    }
    if (on_dev) {
        int drc = dd_levels(dd.d, lvlS.data());
        if (drc != ARROW_OK) return drc;
    }
    // level of every entry of A, per-level nnz and active rows
    h->entry_level.resize(nnz);
    const int nl = int(h->levels.size());
    std::vector<std::vector<int64_t>> cnt(g_threads, std::vector<int64_t>(nl, 0));
    std::vector<std::vector<int64_t>> mx(g_threads, std::vector<int64_t>(nl, -1));
    pfor_rows(n, A->rowptr, [&](int64_t bb, int64_t e, int t) {
        for (int64_t r = bb; r < e; ++r)
            for (int64_t j = A->rowptr[r]; j < A->rowptr[r + 1]; ++j) {
                uint8_t l = S.a2s.empty() ? lvlS[j] : lvlS[S.a2s[j]];
                h->entry_level[j] = l;
                const int32_t* p = h->levels[l].perm.data();
                cnt[t][l]++;
                mx[t][l] = std::max<int64_t>(mx[t][l], std::max(p[r], p[A->colidx[j]]));
            }
    });
    for (int l = 0; l < nl; ++l) {
        int64_t c = 0, m = -1;
        for (int t = 0; t < g_threads; ++t) { c += cnt[t][l]; m = std::max(m, mx[t][l]); }
        h->levels[l].nnz = c;
        h->levels[l].n_active = m + 1;
    }

    // Fused row program: row p of pi_0 holds the entries of vertex v = pi_0^{-1}(p) of
    // every level, in level order, inside a level in increasing level position of the
    // column (the CSR order of B_i).  Each entry reads X row pi_0(column vertex).
    // Rows with more than long_row entries (the head rows of hubs) are split: their
    // entries move to a separate stream cut into fixed-size segments, and their range
    // in the short-row stream is empty.  The program does not depend on the predicate: a
    // row of B_i holds, beside its head columns, the columns of one diagonal tile (block
    // predicate) or of the band |p - q| <= b, which spans three consecutive tiles (the
    // block-tridiagonal form of the band predicate); either way the row's entries are read
    // through the same index stream.
    {
        std::vector<int32_t> iperm0(n);
        const int32_t* perm0 = nl ? h->levels[0].perm.data() : nullptr;
        if (nl) for (int64_t v = 0; v < n; ++v) iperm0[perm0[v]] = int32_t(v);
        else std::iota(iperm0.begin(), iperm0.end(), 0);
        const int32_t long_row = std::min(o.long_row > 0 ? o.long_row : kDefaultLongRow, kMinTileNnz);
        const int32_t seg = o.segment > 0 ? o.segment : kDefaultSegment;
        h->long_row = long_row;
        std::vector<int32_t> len(n);
        for (int64_t p = 0; p < n; ++p) len[p] = int32_t(A->rowptr[iperm0[p] + 1] - A->rowptr[iperm0[p]]);
        h->f_rowptr.assign(n + 1, 0);
        h->long_rows.clear(); h->long_segptr.assign(1, 0); h->seg_begin.clear(); h->seg_end.clear();
        std::vector<int64_t> lptr;   // start of each split row in the long stream
        int64_t nl_ent = 0;
        for (int64_t p = 0; p < n; ++p) {
            const bool is_long = len[p] > long_row;
            h->f_rowptr[p + 1] = h->f_rowptr[p] + (is_long ? 0 : len[p]);
            if (is_long) {
                h->long_rows.push_back(int32_t(p));
                lptr.push_back(nl_ent);
                for (int32_t j = 0; j < len[p]; j += seg) {
                    h->seg_begin.push_back(int32_t(nl_ent + j));
                    h->seg_end.push_back(int32_t(nl_ent + std::min(len[p], j + seg)));
                }
                h->long_segptr.push_back(int32_t(h->seg_begin.size()));
                nl_ent += len[p];
            }
        }
        h->f_col.resize(h->f_rowptr[n]);
        h->f_src.resize(h->f_rowptr[n]);
        h->l_col.resize(nl_ent);
        h->l_src.resize(nl_ent);
        std::vector<int32_t> long_index(n, -1);
        for (size_t i = 0; i < h->long_rows.size(); ++i) long_index[h->long_rows[i]] = int32_t(i);
        std::vector<int64_t> lenp(n + 1, 0);   // entries of the pi_0 rows, as a prefix (chunking)
        for (int64_t p = 0; p < n; ++p) lenp[p + 1] = lenp[p] + len[p];
        pfor_rows(n, lenp.data(), [&](int64_t bb, int64_t e, int) {
            std::vector<std::pair<uint64_t, int32_t>> tmp;
            for (int64_t p = bb; p < e; ++p) {
                int32_t v = iperm0[p];
                tmp.clear();
                for (int64_t j = A->rowptr[v]; j < A->rowptr[v + 1]; ++j) {
                    uint8_t l = h->entry_level[j];
                    uint64_t key = (uint64_t(l) << 32) | uint32_t(h->levels[l].perm[A->colidx[j]]);
                    tmp.push_back({key, int32_t(j)});
                }
                std::sort(tmp.begin(), tmp.end());
                int32_t* dcol;
                int32_t* dsrc;
                if (long_index[p] >= 0) {
                    dcol = h->l_col.data() + lptr[long_index[p]];
                    dsrc = h->l_src.data() + lptr[long_index[p]];
                } else {
                    dcol = h->f_col.data() + h->f_rowptr[p];
                    dsrc = h->f_src.data() + h->f_rowptr[p];
                }
                for (size_t q = 0; q < tmp.size(); ++q) {
                    dcol[q] = perm0[A->colidx[tmp[q].second]];
                    dsrc[q] = tmp[q].second;
                }
            }
        });
        build_tiles(h, h->tune.tile_rows, h->tune.tile_nnz);
    }
    h->decompose_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return ARROW_OK;
}

// ---------------------------------------------------------------------------------------
// Structure report: where the entries of a level sit under the tiling of Section 3.1
// (head rows and columns, the band, the non-zero b x b tiles), and the non-zero tiles of
// an undecomposed matrix in its own order (the equally sized blocks a 1.5D distribution
// would deal out, which Section 6 compares against the decomposition's).
// ---------------------------------------------------------------------------------------
namespace {

// row_entries(p, emit) calls emit(q) for every entry (p, q) of position row p.  Tile rows
// are split over threads; a tile row's column tiles are sorted and counted once each.
template <class RowEntries>
ShapeCount shape_scan(int64_t n, int64_t b, int threads, RowEntries&& row_entries) {
    ShapeCount total;
    if (n <= 0) return total;
    const int64_t ntr = (n + b - 1) / b;
    const int T = int(std::max<int64_t>(1, std::min<int64_t>(threads, ntr)));
    std::vector<ShapeCount> part(T);
    auto work = [&](int t) {
        ShapeCount c;
        std::vector<int64_t> qs;
        for (int64_t P = ntr * t / T; P < ntr * (t + 1) / T; ++P) {
            qs.clear();
            const int64_t p1 = std::min(n, P * b + b);
            for (int64_t p = P * b; p < p1; ++p)
                row_entries(p, [&](int64_t q) {
                    if (p < b || q < b) ++c.head; else ++c.band;
                    qs.push_back(q / b);
                });
            std::sort(qs.begin(), qs.end());
            c.tiles += int64_t(std::unique(qs.begin(), qs.end()) - qs.begin());
        }
        part[t] = c;
    };
    std::vector<std::thread> th;
    for (int t = 1; t < T; ++t) th.emplace_back(work, t);
    work(0);
    for (auto& x : th) x.join();
    for (const ShapeCount& c : part) { total.head += c.head; total.band += c.band; total.tiles += c.tiles; }
    return total;
}

int report_threads() { return int(std::min(256u, std::max(1u, std::thread::hardware_concurrency()))); }

}  // namespace

ShapeCount level_shape_host(const arrow_handle_s* h, int level) {
    const int64_t n = h->n, b = h->b;
    const std::vector<int32_t>& perm = h->levels[level].perm;
    std::vector<int32_t> iperm(n);
    for (int64_t v = 0; v < n; ++v) iperm[perm[v]] = int32_t(v);
    return shape_scan(n, b, report_threads(), [&](int64_t p, auto&& emit) {
        const int64_t v = iperm[p];
        for (int64_t j = h->rowptr[v]; j < h->rowptr[v + 1]; ++j)
            if (h->entry_level[j] == level) emit(int64_t(perm[h->colidx[j]]));
    });
}

int count_tiles_host(const arrow_csr* A, int64_t b, int64_t* tiles) {
    if (b < 1) { set_error("arrow_count_tiles: b must be >= 1"); return ARROW_EINVAL; }
    int rc = validate(A);
    if (rc != ARROW_OK) return rc;
    *tiles = shape_scan(A->n, b, report_threads(), [&](int64_t r, auto&& emit) {
        for (int64_t j = A->rowptr[r]; j < A->rowptr[r + 1]; ++j) emit(int64_t(A->colidx[j]));
    }).tiles;
    return ARROW_OK;
}

}  // namespace arrow

// ---------------------------------------------------------------------------------------
// Serialisation of a decomposed handle (host state only; the device copy is rebuilt by
// arrow_upload).  Little-endian binary: magic, version, scalars, the levels' permutations,
// every host array with an int64 length prefix, and an FNV-1a 64 checksum of all of it.
// ---------------------------------------------------------------------------------------
#include <cstdio>

namespace arrow {
namespace {

constexpr char kMagic[8] = {'A', 'R', 'W', 'D', 'E', 'C', '1', '\0'};
constexpr int64_t kVersion = 3;

struct Writer {
    FILE* f;
    uint64_t h = 1469598103934665603ull;
    bool ok = true;
    void raw(const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
        if (n && std::fwrite(p, 1, n, f) != n) ok = false;
    }
    template <class T> void val(const T& v) { raw(&v, sizeof(T)); }
    template <class T, class Al> void vec(const std::vector<T, Al>& v) {
        val(int64_t(v.size()));
        raw(v.data(), v.size() * sizeof(T));
    }
};

struct Reader {
    FILE* f;
    uint64_t h = 1469598103934665603ull;
    bool ok = true;
    void raw(void* p, size_t n) {
        if (n && std::fread(p, 1, n, f) != n) { ok = false; return; }
        const unsigned char* c = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
    }
    template <class T> void val(T& v) { raw(&v, sizeof(T)); }
    template <class T, class Al> void vec(std::vector<T, Al>& v, int64_t max_len) {
        int64_t n = -1;
        val(n);
        if (!ok || n < 0 || n > max_len) { ok = false; return; }
        v.resize(size_t(n));
        raw(v.data(), size_t(n) * sizeof(T));
    }
};

}  // namespace

int save_host(const arrow_handle_s* h, const char* path) {
    FILE* f = std::fopen(path, "wb");
    if (!f) { set_error(std::string("arrow_save: cannot open ") + path); return ARROW_EINVAL; }
    Writer w{f};
    w.raw(kMagic, 8);
    w.val(kVersion);
    w.val(h->n); w.val(h->nnz); w.val(h->b);
    w.val(h->opts);
    w.val(h->long_row);
    w.val(h->tune);
    w.val(h->decompose_seconds);
    w.val(int64_t(h->levels.size()));
    for (const Level& l : h->levels) {
        w.val(l.n_active);
        w.val(l.nnz);
        w.vec(l.perm);
    }
    w.vec(h->rowptr); w.vec(h->colidx); w.vec(h->values); w.vec(h->entry_level);
    w.vec(h->f_rowptr); w.vec(h->f_col); w.vec(h->f_src); w.vec(h->l_col); w.vec(h->l_src);
    w.vec(h->long_rows); w.vec(h->long_segptr); w.vec(h->seg_begin); w.vec(h->seg_end);
    w.vec(h->tile_row); w.vec(h->tile_ent);
    const uint64_t sum = w.h;
    if (std::fwrite(&sum, sizeof(sum), 1, f) != 1) w.ok = false;
    if (std::fclose(f) != 0) w.ok = false;
    if (!w.ok) { set_error(std::string("arrow_save: write failed for ") + path); return ARROW_EINVAL; }
    return ARROW_OK;
}

int load_host(arrow_handle_s* h, const char* path) {
    FILE* f = std::fopen(path, "rb");
    if (!f) { set_error(std::string("arrow_load: cannot open ") + path); return ARROW_EINVAL; }
    Reader r{f};
    char magic[8];
    int64_t version = 0, nl = -1;
    r.raw(magic, 8);
    r.val(version);
    if (!r.ok || std::memcmp(magic, kMagic, 8) != 0 || version != kVersion) {
        std::fclose(f);
        set_error("arrow_load: not an arrow decomposition file (magic/version)");
        return ARROW_EINVAL;
    }
    r.val(h->n); r.val(h->nnz); r.val(h->b);
    r.val(h->opts);
    r.val(h->long_row);
    r.val(h->tune);
    r.val(h->decompose_seconds);
    r.val(nl);
    const int64_t n = h->n, nnz = h->nnz;
    if (!r.ok || n < 0 || n >= (int64_t(1) << 31) || nnz < 0 || nnz >= (int64_t(1) << 31) || nl < 0 || nl > 254) {
        std::fclose(f);
        set_error("arrow_load: corrupt header");
        return ARROW_EINVAL;
    }
    h->levels.resize(size_t(nl));
    for (Level& l : h->levels) {
        r.val(l.n_active);
        r.val(l.nnz);
        r.vec(l.perm, n);
    }
    r.vec(h->rowptr, n + 1); r.vec(h->colidx, nnz); r.vec(h->values, nnz); r.vec(h->entry_level, nnz);
    r.vec(h->f_rowptr, n + 1); r.vec(h->f_col, nnz); r.vec(h->f_src, nnz); r.vec(h->l_col, nnz); r.vec(h->l_src, nnz);
    r.vec(h->long_rows, n); r.vec(h->long_segptr, n + 1); r.vec(h->seg_begin, nnz + 1); r.vec(h->seg_end, nnz + 1);
    r.vec(h->tile_row, n + 2); r.vec(h->tile_ent, n + 2);
    const uint64_t want = r.h;
    uint64_t sum = 0;
    const bool got = std::fread(&sum, sizeof(sum), 1, f) == 1;
    std::fclose(f);
    if (!r.ok || !got || sum != want) {
        set_error("arrow_load: truncated or corrupt file (checksum)");
        return ARROW_EINVAL;
    }
    // structural consistency of what the device path will index
    bool bad = int64_t(h->rowptr.size()) != n + 1 ||
               int64_t(h->f_rowptr.size()) != (n ? n + 1 : int64_t(h->f_rowptr.size())) ||
               h->f_col.size() != h->f_src.size() || h->l_col.size() != h->l_src.size() ||
               h->seg_begin.size() != h->seg_end.size() || h->tile_row.size() != h->tile_ent.size();
    for (const Level& l : h->levels) bad = bad || int64_t(l.perm.size()) != n;
    for (int32_t c : h->f_col) bad = bad || c < 0 || c >= n;
    for (int32_t c : h->l_col) bad = bad || c < 0 || c >= n;
    for (int32_t s : h->f_src) bad = bad || s < 0 || s >= nnz;
    for (int32_t s : h->l_src) bad = bad || s < 0 || s >= nnz;
    if (!bad && !h->f_rowptr.empty()) bad = h->f_rowptr.back() != int32_t(h->f_col.size());
    if (bad) {
        set_error("arrow_load: inconsistent arrays");
        return ARROW_EINVAL;
    }
    return ARROW_OK;
}

}  // namespace arrow

// ---------------------------------------------------------------------------------------
// C-ABI of the structure report (host only)
// ---------------------------------------------------------------------------------------
extern "C" {

int arrow_get_level_shape(arrow_handle h, int32_t i, arrow_level_shape* out) {
    if (!h || !out || i < 0 || i >= int32_t(h->levels.size())) {
        arrow::set_error("arrow_get_level_shape: bad argument");
        return ARROW_EINVAL;
    }
    const arrow::ShapeCount c = arrow::level_shape_host(h, i);
    out->n_active = h->levels[i].n_active;
    out->nnz = h->levels[i].nnz;
    out->head_nnz = c.head;
    out->band_nnz = c.band;
    out->tiles = c.tiles;
    return ARROW_OK;
}

int arrow_get_program(arrow_handle h, arrow_program* out) {
    if (!h || !out) { arrow::set_error("arrow_get_program: NULL argument"); return ARROW_EINVAL; }
    if (h->f_rowptr.empty() && h->n > 0) {
        arrow::set_error("arrow_get_program: the handle has no device program");
        return ARROW_ESTATE;
    }
    out->n = h->n;
    out->n_short = int64_t(h->f_col.size());
    out->n_long_entries = int64_t(h->l_col.size());
    out->n_long_rows = int64_t(h->long_rows.size());
    out->n_segments = int64_t(h->seg_begin.size());
    out->n_tiles = h->tile_row.empty() ? 0 : int64_t(h->tile_row.size()) - 1;
    out->long_row = h->long_row;
    out->rowptr = h->f_rowptr.data();
    out->col = h->f_col.data();
    out->src = h->f_src.data();
    out->lcol = h->l_col.data();
    out->lsrc = h->l_src.data();
    out->long_rows = h->long_rows.data();
    out->long_segptr = h->long_segptr.data();
    out->seg_begin = h->seg_begin.data();
    out->seg_end = h->seg_end.data();
    out->tile_row = h->tile_row.data();
    out->tile_ent = h->tile_ent.data();
    return ARROW_OK;
}

int arrow_count_tiles(const arrow_csr* A, int64_t b, int64_t* tiles) {
    if (!tiles) { arrow::set_error("arrow_count_tiles: tiles is NULL"); return ARROW_EINVAL; }
    return arrow::count_tiles_host(A, b, tiles);
}

}  // extern "C"
