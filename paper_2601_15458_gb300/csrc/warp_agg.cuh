// Warp-aggregated counter increments for the pair-grouping kernels.
#pragma once
#include <cstdint>

namespace msa {

// counter[key] += 1 for every active lane, with one atomic per distinct key
// in the warp (the pairs of one query usually sit together, so a warp
// mostly holds one key and a batch of few queries does not serialise on a
// few counters).  Returns the counter's value before this lane's increment:
// the old value plus the lane's rank among the active lanes of its key.
// Every lane of the warp must call it.
__device__ __forceinline__ int warp_agg_inc(int32_t *counter, int key, bool active) {
    const int lane = threadIdx.x & 31;
    const unsigned act = __ballot_sync(0xffffffffu, active);
    int r = 0;
    if (active) {
        const unsigned peers = __match_any_sync(act, key);
        const int leader = __ffs(peers) - 1;
        int old = 0;
        if (lane == leader) old = atomicAdd(counter + key, __popc(peers));
        old = __shfl_sync(peers, old, leader);
        r = old + __popc(peers & ((1u << lane) - 1u));
    }
    return r;
}

}  // namespace msa
