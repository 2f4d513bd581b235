// Instantiation of the batched segmented sort for one key type (one
// translation unit per type so the build compiles them in parallel).
#include "segmented.cuh"

namespace ossort {
int run_seg_i32(SegArgs& a) { return run_segmented<KeyI32>(a); }
}  // namespace ossort
