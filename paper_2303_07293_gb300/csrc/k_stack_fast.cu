// k_stack_fast.cu — register-window shift-and-stack kernel (placeholder until
// the tiled kernel lands; the planner falls back to the generic kernel).
#include "st_internal.h"

namespace st {

struct FastPlan {
  int unused;
};

int fast_plan_size_bytes() { return (int)sizeof(FastPlan); }

bool fast_plan_build(const FieldDev&, const int32_t*, const int32_t*, FastPlan** out,
                     cudaStream_t) {
  *out = nullptr;
  return false;
}

void fast_plan_free(FastPlan* fp) { delete fp; }

int launch_stack_fast(const FieldDev&, const FastPlan*, int, int, const int32_t*, float*,
                      int32_t*, Pending*, int64_t, Counters*, cudaStream_t) {
  return -1;
}

}  // namespace st
