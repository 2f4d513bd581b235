// Workspace-plan consistency check (host only, never touches a GPU).
// For every configuration it runs the planner twice -- once in measure mode,
// once as a real sort would (with a placeholder workspace and every launch
// compiled out by OSSORT_NO_LAUNCH) -- and requires the two to use exactly the
// same bytes, so os_workspace_size always covers what os_sort takes.
#include <cstdio>

#include "../../paper_1608_08648_gb300/csrc/driver.cuh"

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
    std::printf("%d of %d configurations consistent\n", total - bad, total);
    return bad ? 1 : 0;
}
