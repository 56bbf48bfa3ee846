// Interleaved static-table rANS over node-bitmap bytes (Sec. 5.2): device
// routines shared by the encode-side and decode-side kernels.
//
// Coder (per segment of sb bytes, W states, byte j -> state j mod W):
//   decode round r: lanes i < W take byte j = rW + i; slot = x mod 2^15 picks
//   the byte b (classes by popcount, bytes ordered by (class, value));
//   x = f_b (x >> 15) + slot - c_b; a state below 2^16 reads the next 16-bit
//   word; within a round words are read in lane order.
//   encode runs the rounds backwards and pushes words so that the decoder's
//   read order results.
#pragma once
#include "pivco_dev.cuh"

namespace pv {

// tables of one ANS table id in shared memory
struct AnsSm {
    uint64_t m48[9];     // ceil(2^48 / q): x / q = (x 2^16 * m48) >> 64 exactly for x < 2^32
    uint32_t q[9];
    uint32_t start[10];
    uint32_t magic[9];
    uint8_t member[256];
    uint8_t base[10];
    uint8_t rank[256];
};

// (enc: also the multipliers the encoder divides with)
__device__ inline void load_ans_table(AnsSm &T, const AnsTables &A, int tid, int lane_id, int nthreads,
                                      bool enc = false) {
    for (int i = lane_id; i < 256; i += nthreads) { T.member[i] = A.class_member[i]; T.rank[i] = A.rank_in_class[i]; }
    if (lane_id < 9) {
        const uint32_t q = A.q[tid][lane_id];
        T.q[lane_id] = q;
        T.magic[lane_id] = A.magic[tid][lane_id];
        if (enc) T.m48[lane_id] = ((1ull << 48) + q - 1) / q;
    }
    if (lane_id < 10) { T.start[lane_id] = A.start[tid][lane_id]; T.base[lane_id] = A.class_base[lane_id]; }
}

// x / q for x < 2^32, q <= 2^15 by a multiply with m48 = ceil(2^48 / q)
// (division by an invariant integer through a multiply, Granlund and
// Montgomery 1994): with m48 = (2^48 + e) / q, 0 <= e < q, the error term
// x e / 2^48 stays below 1 and the quotient is exact.
__device__ inline uint32_t div_q(uint32_t x, uint64_t m48) { return (uint32_t)__umul64hi((uint64_t)x << 16, m48); }

// ---------------------------------------------------------------------------
// Decode one segment (one warp).  body points at the segment's states; words
// follow.  Writes sb bytes (XORed with xr) to dst.  Returns false on a
// malformed segment.  The words are read through `stage` (shared memory,
// kAnsWordWin words), refilled by the whole warp when a round could run past
// it.
// ---------------------------------------------------------------------------
constexpr uint32_t kAnsWordWin = 1024;
__device__ inline bool ans_decode_segment(const uint8_t *states, const uint8_t *words, uint32_t nw, uint32_t sb,
                                          const AnsSm &T, uint8_t xr, uint8_t *dst, uint8_t *stage) {
    const int lane = threadIdx.x & 31;
    const uint32_t W = ans_seg_lanes(sb);
    uint32_t x = lane < (int)W ? ld_le32(states + 4 * lane) : kAnsL;
    bool ok = (x >= kAnsL);
    uint32_t s1 = T.start[1], s2 = T.start[2], s3 = T.start[3], s4 = T.start[4], s5 = T.start[5], s6 = T.start[6],
             s7 = T.start[7], s8 = T.start[8];
    uint32_t rd = 0, wbase = 0, wlim = 0;   // words wbase .. wlim - 1 are staged
    const uint32_t rounds = (sb + W - 1) / W;
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t r = 0; r < rounds; r++) {
        const uint32_t j = r * W + lane;
        const bool active = lane < (int)W && j < sb;
        uint32_t b = 0;
        if (active) {
            const uint32_t slot = x & (kAnsM - 1);
            const uint32_t k = (slot >= s1) + (slot >= s2) + (slot >= s3) + (slot >= s4) + (slot >= s5) +
                               (slot >= s6) + (slot >= s7) + (slot >= s8);
            const uint32_t q = T.q[k], rel = slot - T.start[k];
            const uint32_t idx = T.magic[k] ? (uint32_t)(((uint64_t)rel * T.magic[k]) >> 32) : rel;
            b = T.member[T.base[k] + idx];
            x = q * (x >> kAnsScale) + (rel - idx * q);
        }
        const bool need = active && x < kAnsL;
        const uint32_t m = __ballot_sync(0xffffffffu, need);
        if (rd + __popc(m) > wlim && wlim < nw) {   // (warp-uniform) the next window of words
            __syncwarp();
            const uint32_t nb = 2u * min(kAnsWordWin, nw - rd);
            for (uint32_t i = lane; i < nb; i += 32) stage[i] = words[2ull * rd + i];
            __syncwarp();
            wbase = rd;
            wlim = rd + nb / 2;
        }
        if (need) {
            const uint32_t pos = rd + __popc(m & lt);
            if (pos < wlim) x = (x << 16) | ((uint32_t)stage[2 * (pos - wbase)] | ((uint32_t)stage[2 * (pos - wbase) + 1] << 8));
            else ok = false;
        }
        rd += __popc(m);
        if (active) dst[j] = (uint8_t)(b ^ xr);
    }
    if (lane < (int)W && x != kAnsL) ok = false;
    if (rd != nw) ok = false;
    return __all_sync(0xffffffffu, ok);
}

// ---------------------------------------------------------------------------
// Encode one segment (one warp).  src: sb raw bytes (XORed with xr before
// coding).  The first cap words emitted are staged backwards in stage[0 ..
// cap) (emission e at cap - 1 - e); later ones go to ovf (global) in
// emission order, word e - cap at ovf[2 (e - cap)], while they fit ovf_words.
// Returns the word count; final states in x (lane < W).
// ---------------------------------------------------------------------------
__device__ inline uint32_t ans_encode_segment(const uint8_t *src, uint32_t sb, const AnsSm &T, uint8_t xr,
                                              uint16_t *stage, uint32_t cap, uint8_t *ovf, uint32_t ovf_words,
                                              uint32_t &x_out) {
    const int lane = threadIdx.x & 31;
    const uint32_t W = ans_seg_lanes(sb);
    uint32_t x = kAnsL;
    uint32_t cnt = 0;
    const uint32_t rounds = (sb + W - 1) / W;
    const uint32_t gt = ~((2u << lane) - 1u);
    // the lane's bytes of 16 rounds at a time (rounds 16 w .. 16 w + 15 of
    // window w), loaded together, the next window's while this one is coded
    const uint32_t nwin = (rounds + 15) / 16;
    auto load_win = [&](int w, uint32_t (&p)[4]) {
#pragma unroll
        for (int i = 0; i < 4; i++) p[i] = 0;
        if (w < 0) return;
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const uint32_t j = (16u * (uint32_t)w + (uint32_t)i) * W + (uint32_t)lane;
            const uint32_t v = (lane < (int)W && j < sb) ? (uint32_t)src[j] : 0u;
            p[i >> 2] |= v << (8 * (i & 3));
        }
    };
    uint32_t cur[4], nxt[4];
    load_win((int)nwin - 1, cur);
    for (int w = (int)nwin - 1; w >= 0; w--) {
        load_win(w - 1, nxt);
#pragma unroll
        for (int i = 15; i >= 0; i--) {
            const uint32_t r = 16u * (uint32_t)w + (uint32_t)i;
            if (r >= rounds) continue;   // (warp-uniform)
            const uint32_t j = r * W + lane;
            const bool active = lane < (int)W && j < sb;
            uint32_t f = 1, c = 0, k = 0;
            bool emit = false;
            if (active) {
                const uint32_t b = ((cur[i >> 2] >> (8 * (i & 3))) & 0xFFu) ^ xr;
                k = __popc(b);
                f = T.q[k];
                c = T.start[k] + T.rank[b] * f;
                emit = (uint64_t)x >= ((uint64_t)f << 17);
            }
            const uint32_t m = __ballot_sync(0xffffffffu, emit);
            if (emit) {
                const uint32_t pos = cnt + __popc(m & gt);
                if (pos < cap) {
                    stage[cap - 1 - pos] = (uint16_t)(x & 0xFFFF);
                } else if (pos - cap < ovf_words) {
                    ovf[2 * (pos - cap)] = (uint8_t)x;
                    ovf[2 * (pos - cap) + 1] = (uint8_t)(x >> 8);
                }
                x >>= 16;
            }
            cnt += __popc(m);
            if (active) {
                const uint32_t qt = div_q(x, T.m48[k]);
                x = (qt << kAnsScale) + (x - qt * f) + c;
            }
        }
#pragma unroll
        for (int i = 0; i < 4; i++) cur[i] = nxt[i];
    }
    x_out = x;
    return cnt;
}

__device__ inline bool ans_segment_at(const uint8_t *body, uint64_t body_len, uint32_t nbytes, uint32_t s,
                                      uint64_t &st_pos, uint32_t &nw) {
    const int lane = threadIdx.x & 31;
    const uint32_t S = ans_seg_count(nbytes);
    if (4ull * S > body_len) return false;
    uint64_t acc = 0;
    for (uint32_t j = lane; j < s; j += 32) {
        const uint32_t sbj = min(kAnsSeg, nbytes - j * kAnsSeg);
        acc += 4ull * ans_seg_lanes(sbj) + 2ull * ld_le32(body + 4 * j);
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    st_pos = 4ull * S + acc;
    nw = ld_le32(body + 4 * s);
    const uint32_t sb = min(kAnsSeg, nbytes - s * kAnsSeg);
    return st_pos + 4ull * ans_seg_lanes(sb) + 2ull * nw <= body_len;
}


}  // namespace pv
