// First-fit allocator over one device arena (offsets only; the serving runtime owns the
// memory) with coalescing of neighbouring free blocks.  Host code, no CUDA.
#pragma once

#include <algorithm>
#include <cstddef>
#include <iterator>
#include <map>

namespace arrow {

struct Arena {
    size_t cap = 0, in_use = 0, peak = 0;
    std::map<size_t, size_t> free_;   // offset -> size
    void init(size_t c) { cap = c; free_.clear(); free_[0] = c; in_use = peak = 0; }
    // Lowest offset with `bytes` free after it; false if no free block is large enough.
    bool alloc(size_t bytes, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t at = it->first + bytes;
            free_.erase(it);
            if (rest) free_[at] = rest;
            in_use += bytes;
            peak = std::max(peak, in_use);
            return true;
        }
        return false;
    }
    // Return [off, off + bytes) (a block alloc handed out) and merge it with free neighbours.
    void release(size_t off, size_t bytes) {
        in_use -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

}  // namespace arrow
