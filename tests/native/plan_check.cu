// Workspace-plan consistency check (host only, never touches a GPU).
// For every configuration it runs the planner twice -- once in measure mode,
// once as a real sort would (with a placeholder workspace and every launch
// compiled out by OSSORT_NO_LAUNCH) -- and requires the two to use exactly the
// same bytes, so os_workspace_size always covers what os_sort takes.
#include <cstdio>

#include "../../paper_1608_08648_gb300/csrc/segmented.cuh"

using namespace ossort;

template <class KT>
int check(const char* kname, uint64_t n, bool hv, int split, uint32_t p, uint32_t s) {
    os_params prm{split, p, s, OS_STABLE, 7};
    RunArgs m{};
    m.n = n;
    m.has_vals = hv;
    m.prm = prm;
    run_sort<KT>(m);
    RunArgs l{};
    l.n = n;
    l.has_vals = hv;
    l.prm = prm;
    l.ws = reinterpret_cast<void*>(static_cast<uintptr_t>(1) << 40);
    l.ws_bytes = m.used;
    l.num_sms = 152;
    const int rc = run_sort<KT>(l);
    if (rc != OS_OK || l.used != m.used) {
        std::printf("MISMATCH %s n=%llu hv=%d split=%d p=%u s=%u measure=%zu live=%zu rc=%d\n", kname,
                    (unsigned long long)n, (int)hv, split, p, s, m.used, l.used, rc);
        return 1;
    }
    return 0;
}

template <class KT>
int check_seg(const char* kname, uint64_t n, uint32_t nseg, bool hv, const SegClasses& cls) {
    SegArgs m{};
    m.n = n;
    m.nseg = nseg;
    m.has_vals = hv;
    m.cls = cls;
    run_segmented<KT>(m);
    SegArgs l = m;
    l.used = 0;
    l.ws = reinterpret_cast<void*>(static_cast<uintptr_t>(1) << 40);
    l.ws_bytes = m.used;
    l.num_sms = 152;
    l.off = reinterpret_cast<const uint64_t*>(static_cast<uintptr_t>(1) << 41);
    const int rc = run_segmented<KT>(l);
    if (rc != OS_OK || l.used != m.used) {
        std::printf("MISMATCH segmented %s n=%llu nseg=%u hv=%d classes=%u measure=%zu live=%zu rc=%d\n", kname,
                    (unsigned long long)n, nseg, (int)hv, cls.n, m.used, l.used, rc);
        return 1;
    }
    return 0;
}

int main() {
    const uint64_t ns[] = {0, 1, 100, 4097, 8193, 100003, 1u << 20, (1u << 22) + 7, 1u << 27};
    const uint32_t ps[] = {1, 2, 3, 64, 1000, 4096};
    const uint32_t ss[] = {1, 2, 16};
    int bad = 0, total = 0;
    for (uint64_t n : ns)
        for (uint32_t p : ps)
            for (uint32_t s : ss)
                for (int split = 0; split < 2; ++split)
                    for (int hv = 0; hv < 2; ++hv) {
                        bad += check<KeyI32>("i32", n, hv, split, p, s);
                        bad += check<KeyU64>("u64", n, hv, split, p, s);
                        bad += check<KeyF64>("f64", n, hv, split, p, s);
                        total += 3;
                    }
    // Batched segmented sort: class tables with and without partitioned classes.
    SegClasses tables[3] = {};
    tables[0].n = 1;
    tables[0].c[0] = SegClass{~0ull, 1, 1, 2048, 0};
    tables[1].n = 3;
    tables[1].c[0] = SegClass{4096, 1, 1, 4096, 0};
    tables[1].c[1] = SegClass{65536, 8, 16, 2048, 0};
    tables[1].c[2] = SegClass{1ull << 20, 64, 64, 8192, 0};
    tables[2].n = 1;
    tables[2].c[0] = SegClass{~0ull, 1024, 4, 2048, 0};
    const uint64_t sn[] = {0, 1, 5000, 1u << 20, 1u << 28};
    const uint32_t sseg[] = {1, 7, 10000};
    for (const SegClasses& t : tables)
        for (uint64_t n : sn)
            for (uint32_t nseg : sseg)
                for (int hv = 0; hv < 2; ++hv) {
                    bad += check_seg<KeyI32>("i32", n, nseg, hv, t);
                    bad += check_seg<KeyU64>("u64", n, nseg, hv, t);
                    bad += check_seg<KeyF64>("f64", n, nseg, hv, t);
                    total += 3;
                }
    std::printf("%d of %d configurations consistent\n", total - bad, total);
    return bad ? 1 : 0;
}
