// st_pending.cuh — warp-aggregated append of above-threshold points.
#pragma once

#include "st_internal.h"

namespace st {

// Every lane of the warp must call this (pass may be false).  One atomicAdd
// per warp reserves the slots; points past `cap` are counted, not written,
// and raise ERR_PENDING_OVERFLOW.
__device__ __forceinline__ void push_pending(bool pass, const Pending& rec, Pending* pend,
                                             int64_t cap, Counters* ctr) {
  unsigned m = __ballot_sync(0xffffffffu, pass);
  if (m == 0u) return;
  int lane = threadIdx.x & 31;
  int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(&ctr->n_pending, (unsigned long long)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pass) {
    unsigned long long pos = base + (unsigned long long)__popc(m & ((1u << lane) - 1u));
    if (pos < (unsigned long long)cap)
      pend[pos] = rec;
    else
      atomicOr(&ctr->error, ERR_PENDING_OVERFLOW);
  }
}

}  // namespace st
