// Instantiation of the sort for one key type (one translation unit per type
// so the build compiles them in parallel).
#include "driver.cuh"

namespace ossort {
int run_f64(RunArgs& a) { return run_sort<KeyF64>(a); }
}  // namespace ossort
