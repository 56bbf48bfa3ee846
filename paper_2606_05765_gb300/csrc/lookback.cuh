// Decoupled look-back (single-pass prefix over CTAs in ticket order).
// Each tile publishes its aggregate, then walks back over its predecessors
// until it meets an inclusive prefix, and publishes its own inclusive prefix.
// Every wait is bounded by a 1 s device-clock limit; on expiry the caller's
// timeout flag is set and the partial prefix is used (the status reports it).
#pragma once
#include "pivco_dev.cuh"

namespace pv {

constexpr uint64_t kLbFlagAgg = 1ull << 62;
constexpr uint64_t kLbFlagInc = 2ull << 62;
constexpr uint64_t kLbValMask = (1ull << 62) - 1;

__device__ inline void lb_store(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ inline uint64_t lb_load(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Called by ONE thread.  Returns the exclusive prefix of `agg` over tiles
// 0 .. tile-1.  states[] must be zero before the launch.
__device__ inline uint64_t lookback_exclusive(uint64_t *states, int tile, uint64_t agg, int *timed_out) {
    if (tile == 0) {
        lb_store(&states[0], kLbFlagInc | (agg & kLbValMask));
        return 0;
    }
    lb_store(&states[tile], kLbFlagAgg | (agg & kLbValMask));
    uint64_t excl = 0;
    int j = tile - 1;
    const uint64_t t0 = globaltimer_ns();
    unsigned ns = 32;
    while (j >= 0) {
        const uint64_t v = lb_load(&states[j]);
        const uint64_t f = v & ~kLbValMask;
        if (f == 0) {
            if (globaltimer_ns() - t0 > kWaitLimitNs) { *timed_out = 1; break; }
            __nanosleep(ns);
            if (ns < 1024) ns <<= 1;
            continue;
        }
        excl += v & kLbValMask;
        if (f == kLbFlagInc) break;
        j--;
    }
    lb_store(&states[tile], kLbFlagInc | ((excl + agg) & kLbValMask));
    return excl;
}

// The same prefix with a whole warp walking back: each step reads the states
// of the 32 predecessors below j at once and sums the values up to the
// nearest inclusive prefix, so a walk over many published aggregates takes
// one load latency per 32 predecessors.  Called by all 32 lanes with the
// same arguments; returns the exclusive prefix in every lane.
__device__ inline uint64_t lookback_exclusive_warp(uint64_t *states, int tile, uint64_t agg, int *timed_out) {
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) lb_store(&states[0], kLbFlagInc | (agg & kLbValMask));
        return 0;
    }
    if (lane == 0) lb_store(&states[tile], kLbFlagAgg | (agg & kLbValMask));
    uint64_t excl = 0;
    int j = tile - 1;
    const uint64_t t0 = globaltimer_ns();
    unsigned ns = 32;
    for (;;) {
        const int k = j - lane;
        const uint64_t v = k >= 0 ? lb_load(&states[k]) : kLbFlagInc;   // before tile 0: an inclusive zero
        const uint64_t f = v & ~kLbValMask;
        const uint32_t inc = __ballot_sync(0xffffffffu, f == kLbFlagInc);
        const uint32_t unset = __ballot_sync(0xffffffffu, f == 0);
        const uint32_t upto = inc ? ((inc & (0u - inc)) << 1) - 1u : 0xFFFFFFFFu;   // lanes up to the nearest one
        if (unset & upto) {
            if (__any_sync(0xffffffffu, globaltimer_ns() - t0 > kWaitLimitNs)) {
                *timed_out = 1;
                break;
            }
            __nanosleep(ns);
            if (ns < 1024) ns <<= 1;
            continue;
        }
        uint64_t x = ((upto >> lane) & 1u) ? (v & kLbValMask) : 0ull;
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        excl += x;
        if (inc) break;
        j -= 32;
    }
    if (lane == 0) lb_store(&states[tile], kLbFlagInc | ((excl + agg) & kLbValMask));
    return excl;
}

}  // namespace pv
