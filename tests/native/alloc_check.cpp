// The serving loop's arena allocator against a brute-force model: random
// sequences of alloc / release / shrink, checking after every step that blocks
// are disjoint, inside the arena and 256-byte aligned, that the byte count in
// use matches, that free space is fully coalesced (an allocation of the largest
// free extent succeeds) and that first fit is honoured.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <vector>

#include "../../paper_1608_08648_gb300/csrc/arena_alloc.h"

using ossort::ArenaAlloc;

static unsigned long long rng_state = 88172645463325252ull;
static unsigned long long rnd() {   // xorshift64
    rng_state ^= rng_state << 13;
    rng_state ^= rng_state >> 7;
    rng_state ^= rng_state << 17;
    return rng_state;
}

int main() {
    const size_t cap = 1 << 20;
    const size_t units = cap / ArenaAlloc::ALIGN;
    int bad = 0;
    for (int trial = 0; trial < 200 && !bad; ++trial) {
        ArenaAlloc a(cap);
        std::vector<int> owner(units, -1);           // model: which live block owns each unit
        std::map<size_t, size_t> live;               // offset -> bytes
        int id = 0;
        for (int step = 0; step < 400 && !bad; ++step) {
            const int op = (int)(rnd() % 10);
            if (op < 5 || live.empty()) {
                const size_t want = 1 + rnd() % (cap / 8);
                const size_t need = ArenaAlloc::round(want) / ArenaAlloc::ALIGN;
                // model first fit
                size_t model = SIZE_MAX, run = 0;
                for (size_t u = 0; u < units; ++u) {
                    run = owner[u] < 0 ? run + 1 : 0;
                    if (run == need) { model = (u + 1 - need) * ArenaAlloc::ALIGN; break; }
                }
                const size_t off = a.alloc(want);
                if (off != model) { std::printf("first fit: got %zu expected %zu\n", off, model); bad = 1; break; }
                if (off == SIZE_MAX) continue;
                for (size_t u = off / ArenaAlloc::ALIGN; u < off / ArenaAlloc::ALIGN + need; ++u) owner[u] = id;
                live[off] = need * ArenaAlloc::ALIGN;
                ++id;
            } else if (op < 8) {
                auto it = live.begin();
                std::advance(it, rnd() % live.size());
                if (!a.release(it->first)) { std::printf("release refused\n"); bad = 1; break; }
                for (size_t u = it->first / ArenaAlloc::ALIGN; u < (it->first + it->second) / ArenaAlloc::ALIGN; ++u)
                    owner[u] = -1;
                live.erase(it);
            } else {
                auto it = live.begin();
                std::advance(it, rnd() % live.size());
                const size_t keep = rnd() % (it->second + 1);
                const size_t k = ArenaAlloc::round(keep ? keep : 1);
                if (!a.shrink(it->first, keep)) { std::printf("shrink refused\n"); bad = 1; break; }
                if (k < it->second) {
                    for (size_t u = (it->first + k) / ArenaAlloc::ALIGN; u < (it->first + it->second) / ArenaAlloc::ALIGN; ++u)
                        owner[u] = -1;
                    it->second = k;
                }
            }
            size_t in_use = 0, largest = 0, run = 0;
            for (size_t u = 0; u < units; ++u) {
                if (owner[u] >= 0) { in_use += ArenaAlloc::ALIGN; run = 0; }
                else { run += ArenaAlloc::ALIGN; largest = run > largest ? run : largest; }
            }
            if (a.in_use() != in_use || a.largest_free() != largest || a.used_blocks() != live.size()) {
                std::printf("state: in_use %zu/%zu largest %zu/%zu blocks %zu/%zu\n", a.in_use(), in_use,
                            a.largest_free(), largest, a.used_blocks(), live.size());
                bad = 1;
            }
        }
        if (!a.release(12345)) {} else { std::printf("release of an unknown offset accepted\n"); bad = 1; }
    }
    std::printf(bad ? "FAILED\n" : "allocator consistent\n");
    return bad;
}
