// Decoupled look-back (single-pass prefix over CTAs in ticket order).
// Each tile publishes its aggregate, then walks back over its predecessors
// until it meets an inclusive prefix, and publishes its own inclusive prefix.
// Every wait is bounded by a device-clock limit (limit_ns); on expiry the
// caller's timeout flag is set and the tile publishes its partial prefix
// marked as poisoned.  A tile that meets a poisoned prefix sets its own
// timeout flag and passes the poison on, so every tile after an expired wait
// reports it and no tile takes a partial prefix for a final one.
#pragma once
#include "pivco_dev.cuh"

namespace pv {

constexpr uint64_t kLbFlagAgg = 1ull << 62;
constexpr uint64_t kLbFlagInc = 2ull << 62;
constexpr uint64_t kLbPoison = 1ull << 61;
constexpr uint64_t kLbValMask = (1ull << 61) - 1;

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
__device__ inline uint64_t lookback_exclusive(uint64_t *states, int tile, uint64_t agg, int *timed_out,
                                              uint64_t limit_ns) {
    if (tile == 0) {
        lb_store(&states[0], kLbFlagInc | (agg & kLbValMask));
        return 0;
    }
    lb_store(&states[tile], kLbFlagAgg | (agg & kLbValMask));
    uint64_t excl = 0;
    int j = tile - 1;
    bool bad = false;
    const uint64_t t0 = globaltimer_ns();
    unsigned ns = 32;
    while (j >= 0) {
        const uint64_t v = lb_load(&states[j]);
        const uint64_t f = v & (kLbFlagAgg | kLbFlagInc);
        if (f == 0) {
            if (globaltimer_ns() - t0 > limit_ns) { bad = true; break; }
            __nanosleep(ns);
            if (ns < 1024) ns <<= 1;
            continue;
        }
        excl += v & kLbValMask;
        if (f == kLbFlagInc) {
            bad = (v & kLbPoison) != 0;
            break;
        }
        j--;
    }
    if (bad) *timed_out = 1;
    lb_store(&states[tile], kLbFlagInc | (bad ? kLbPoison : 0ull) | ((excl + agg) & kLbValMask));
    return excl;
}

// The same prefix with a whole warp walking back: each step reads the states
// of the 32 predecessors below j at once and sums the values up to the
// nearest inclusive prefix, so a walk over many published aggregates takes
// one load latency per 32 predecessors.  Called by all 32 lanes with the
// same arguments; returns the exclusive prefix in every lane.
__device__ inline uint64_t lookback_exclusive_warp(uint64_t *states, int tile, uint64_t agg, int *timed_out,
                                                   uint64_t limit_ns) {
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) lb_store(&states[0], kLbFlagInc | (agg & kLbValMask));
        return 0;
    }
    if (lane == 0) lb_store(&states[tile], kLbFlagAgg | (agg & kLbValMask));
    uint64_t excl = 0;
    int j = tile - 1;
    bool bad = false;
    const uint64_t t0 = globaltimer_ns();
    unsigned ns = 32;
    for (;;) {
        const int k = j - lane;
        const uint64_t v = k >= 0 ? lb_load(&states[k]) : kLbFlagInc;   // before tile 0: an inclusive zero
        const uint64_t f = v & (kLbFlagAgg | kLbFlagInc);
        const uint32_t inc = __ballot_sync(0xffffffffu, f == kLbFlagInc);
        const uint32_t unset = __ballot_sync(0xffffffffu, f == 0);
        const uint32_t upto = inc ? ((inc & (0u - inc)) << 1) - 1u : 0xFFFFFFFFu;   // lanes up to the nearest one
        if (unset & upto) {
            if (__any_sync(0xffffffffu, globaltimer_ns() - t0 > limit_ns)) {
                bad = true;
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
        if (inc) {
            bad = (__ballot_sync(0xffffffffu, (v & kLbPoison) != 0) & inc & (0u - inc)) != 0;
            break;
        }
        j -= 32;
    }
    if (bad) *timed_out = 1;
    if (lane == 0) lb_store(&states[tile], kLbFlagInc | (bad ? kLbPoison : 0ull) | ((excl + agg) & kLbValMask));
    return excl;
}

// Two chains at once (the same tile in both): lanes 0-15 walk chain A and
// lanes 16-31 chain B, 16 predecessors per step each; a half that has met
// its inclusive prefix stops reading while the other goes on.  Called by all
// 32 lanes; returns both exclusive prefixes in every lane.
__device__ inline void lookback2_exclusive_warp(uint64_t *states_a, uint64_t *states_b, int tile, uint64_t agg_a,
                                                uint64_t agg_b, uint64_t &excl_a, uint64_t &excl_b,
                                                int *timed_out, uint64_t limit_ns) {
    const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    uint64_t *states = half ? states_b : states_a;
    const uint64_t agg = half ? agg_b : agg_a;
    if (tile == 0) {
        if (hl == 0) lb_store(&states[0], kLbFlagInc | (agg & kLbValMask));
        excl_a = excl_b = 0;
        return;
    }
    if (hl == 0) lb_store(&states[tile], kLbFlagAgg | (agg & kLbValMask));
    uint64_t excl = 0;
    int j = tile - 1;
    bool done = false;   // (the same in all lanes of a half)
    bool bad = false;    // an expired wait, or a poisoned prefix met (the same in all lanes)
    const uint64_t t0 = globaltimer_ns();
    unsigned ns = 32;
    for (;;) {
        const int k = j - hl;
        uint64_t v = kLbFlagInc;   // before tile 0: an inclusive zero
        if (!done && k >= 0) v = lb_load(&states[k]);
        const uint64_t f = v & (kLbFlagAgg | kLbFlagInc);
        const uint32_t inc = (__ballot_sync(0xffffffffu, f == kLbFlagInc) >> (16 * half)) & 0xFFFFu;
        const uint32_t unset = (__ballot_sync(0xffffffffu, f == 0) >> (16 * half)) & 0xFFFFu;
        const uint32_t pois = (__ballot_sync(0xffffffffu, (v & kLbPoison) != 0) >> (16 * half)) & 0xFFFFu;
        const uint32_t upto = inc ? ((inc & (0u - inc)) << 1) - 1u : 0xFFFFu;   // lanes up to the nearest one
        if (__any_sync(0xffffffffu, !done && (unset & upto))) {
            if (__any_sync(0xffffffffu, globaltimer_ns() - t0 > limit_ns)) {
                bad = true;
                break;
            }
            __nanosleep(ns);
            if (ns < 1024) ns <<= 1;
            continue;
        }
        uint64_t x = (!done && ((upto >> hl) & 1u)) ? (v & kLbValMask) : 0ull;
#pragma unroll
        for (int o = 8; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);   // within the half
        if (__any_sync(0xffffffffu, !done && (pois & inc & (0u - inc)) != 0)) bad = true;
        if (!done) {
            excl += x;
            if (inc) done = true;
            else j -= 16;
        }
        if (__all_sync(0xffffffffu, done)) break;
    }
    // a poisoned or partial prefix in either chain makes both chains' prefixes
    // unusable downstream (the block's offsets come from both)
    if (bad) *timed_out = 1;
    if (hl == 0) lb_store(&states[tile], kLbFlagInc | (bad ? kLbPoison : 0ull) | ((excl + agg) & kLbValMask));
    excl_a = __shfl_sync(0xffffffffu, excl, 0);
    excl_b = __shfl_sync(0xffffffffu, excl, 16);
}

}  // namespace pv
