// Randomised check of the serving runtime's arena allocator (paper_2402_19364_gb300/csrc/arena.h)
// against a byte-occupancy model: first fit over maximal free intervals, exact coalescing,
// in-use and peak accounting.  Prints "ok" or the first mismatch; exit code 0 only on "ok".
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <utility>
#include <vector>

#include "arena.h"

static std::map<size_t, size_t> free_intervals(const std::vector<char>& used) {
    std::map<size_t, size_t> f;
    size_t i = 0;
    while (i < used.size()) {
        if (used[i]) { ++i; continue; }
        size_t j = i;
        while (j < used.size() && !used[j]) ++j;
        f[i] = j - i;
        i = j;
    }
    return f;
}

int main() {
    for (unsigned seed = 1; seed <= 20; ++seed) {
        std::mt19937 rng(seed);
        const size_t cap = 200 + rng() % 2000;
        arrow::Arena a;
        a.init(cap);
        std::vector<char> used(cap, 0);
        std::vector<std::pair<size_t, size_t>> live;
        size_t in_use = 0, peak = 0;
        for (int op = 0; op < 20000; ++op) {
            const bool do_alloc = live.empty() || rng() % 100 < 55;
            if (do_alloc) {
                const size_t bytes = 1 + rng() % (cap / 8);
                size_t want = size_t(-1);
                for (auto& iv : free_intervals(used))
                    if (iv.second >= bytes) { want = iv.first; break; }
                size_t off = 0;
                const bool ok = a.alloc(bytes, &off);
                if (ok != (want != size_t(-1)) || (ok && off != want)) {
                    std::printf("seed %u op %d: alloc(%zu) gave %d/%zu, first fit is %zu\n", seed, op, bytes, ok, off, want);
                    return 1;
                }
                if (ok) {
                    for (size_t i = off; i < off + bytes; ++i) used[i] = 1;
                    live.push_back({off, bytes});
                    in_use += bytes;
                    peak = std::max(peak, in_use);
                }
            } else {
                const size_t k = rng() % live.size();
                const auto blk = live[k];
                live[k] = live.back();
                live.pop_back();
                a.release(blk.first, blk.second);
                for (size_t i = blk.first; i < blk.first + blk.second; ++i) used[i] = 0;
                in_use -= blk.second;
            }
            if (a.free_ != free_intervals(used) || a.in_use != in_use || a.peak != peak) {
                std::printf("seed %u op %d: free list or accounting differs from the model\n", seed, op);
                return 1;
            }
        }
        for (auto& blk : live) a.release(blk.first, blk.second);
        if (a.free_.size() != 1 || a.free_.begin()->first != 0 || a.free_.begin()->second != cap || a.in_use != 0) {
            std::printf("seed %u: arena not whole again after releasing everything\n", seed);
            return 1;
        }
    }
    std::printf("ok\n");
    return 0;
}
