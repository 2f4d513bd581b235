// First-fit sub-allocator over one caller-provided device arena (the serving
// loop's HBM budget).  Host-side bookkeeping only: offsets into the arena,
// never a CUDA call, so it can run inside a stream callback.  Blocks are
// multiples of 256 bytes; freed blocks coalesce with free neighbours.
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>

namespace ossort {

class ArenaAlloc {
public:
    static constexpr size_t ALIGN = 256;

    explicit ArenaAlloc(size_t bytes = 0) { reset(bytes); }

    void reset(size_t bytes) {
        cap_ = bytes & ~(ALIGN - 1);
        free_.clear();
        used_.clear();
        if (cap_) free_[0] = cap_;
        in_use_ = 0;
        peak_ = 0;
    }

    static size_t round(size_t b) { return (b + ALIGN - 1) & ~(ALIGN - 1); }

    // Offset of a block of at least `bytes` (rounded up), or SIZE_MAX when no free
    // block is large enough.
    size_t alloc(size_t bytes) {
        const size_t need = round(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            const size_t off = it->first, rest = it->second - need;
            free_.erase(it);
            if (rest) free_[off + need] = rest;
            used_[off] = need;
            in_use_ += need;
            if (in_use_ > peak_) peak_ = in_use_;
            return off;
        }
        return SIZE_MAX;
    }

    // Returns false for an offset that is not an allocated block.
    bool release(size_t off) {
        auto u = used_.find(off);
        if (u == used_.end()) return false;
        size_t beg = off, len = u->second;
        used_.erase(u);
        in_use_ -= len;
        auto nx = free_.lower_bound(beg);
        if (nx != free_.end() && nx->first == beg + len) {      // merge with the next free block
            len += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {                              // and with the previous one
            auto pv = std::prev(nx);
            if (pv->first + pv->second == beg) {
                beg = pv->first;
                len += pv->second;
                free_.erase(pv);
            }
        }
        free_[beg] = len;
        return true;
    }

    // Keep the first `keep` bytes (rounded up, at least one unit) of an allocated
    // block and free the rest.  Returns false for an unknown offset.
    bool shrink(size_t off, size_t keep) {
        auto u = used_.find(off);
        if (u == used_.end()) return false;
        const size_t k = round(keep ? keep : 1);
        if (k >= u->second) return true;
        const size_t tail = off + k, tail_len = u->second - k;
        u->second = k;
        used_[tail] = tail_len;
        return release(tail);
    }

    size_t capacity() const { return cap_; }
    size_t in_use() const { return in_use_; }
    size_t peak() const { return peak_; }
    size_t largest_free() const {
        size_t m = 0;
        for (const auto& f : free_) m = f.second > m ? f.second : m;
        return m;
    }
    size_t free_blocks() const { return free_.size(); }
    size_t used_blocks() const { return used_.size(); }

private:
    size_t cap_ = 0, in_use_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;   // offset -> length, disjoint, never adjacent
    std::map<size_t, size_t> used_;   // offset -> length
};

}  // namespace ossort
