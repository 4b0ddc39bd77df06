// First-fit placement of variable-size blocks in one fixed range [0, size) of bytes: the
// serving arena's bookkeeping (the device memory itself is one allocation of the budget).
// Plain C++ with no CUDA, so that the host tests compile it on its own.
#pragma once

#include <cstdint>
#include <iterator>
#include <map>

namespace snect {

struct ArenaBlocks {
    std::map<int64_t, int64_t> free_blocks;  // offset -> bytes; adjacent free blocks are merged

    // the whole range free
    void reset(int64_t size) {
        free_blocks.clear();
        if (size > 0) free_blocks[0] = size;
    }

    // the lowest-offset free block of at least `bytes` gives its front; -1 if none is large enough
    int64_t alloc(int64_t bytes) {
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
            if (it->second < bytes) continue;
            const int64_t off = it->first, rest = it->second - bytes;
            free_blocks.erase(it);
            if (rest > 0) free_blocks[off + bytes] = rest;
            return off;
        }
        return -1;
    }

    // returns [off, off + bytes), which alloc handed out, merging it with free neighbours
    void release(int64_t off, int64_t bytes) {
        auto it = free_blocks.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_blocks.end() && it->first + it->second == nx->first) {  // merge with the next
            it->second += nx->second;
            free_blocks.erase(nx);
        }
        if (it != free_blocks.begin()) {  // and with the previous
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_blocks.erase(it);
            }
        }
    }
};

}  // namespace snect
