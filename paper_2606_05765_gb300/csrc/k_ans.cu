// Selective ANS of node bitmaps (Sec. 5.2): byte-wise static-table rANS,
// interleaved over W states per 16 KiB segment, one warp per segment.
//
// Coder (per segment of sb bytes, W states, byte j -> state j mod W):
//   decode round r: lanes i < W take byte j = rW + i; slot = x mod 2^15 picks
//   the byte b (classes by popcount, bytes ordered by (class, value));
//   x = f_b (x >> 15) + slot - c_b; a state below 2^16 reads the next 16-bit
//   word; within a round words are read in lane order.
//   encode runs the rounds backwards and pushes words so that the decoder's
//   read order results.
#include "lookback.cuh"

namespace pv {

// tables of one ANS table id in shared memory
struct AnsSm {
    uint32_t q[9];
    uint32_t start[10];
    uint32_t magic[9];
    uint8_t member[256];
    uint8_t base[10];
    uint8_t rank[256];
};

__device__ inline void load_ans_table(AnsSm &T, const AnsTables &A, int tid, int lane_id, int nthreads) {
    for (int i = lane_id; i < 256; i += nthreads) { T.member[i] = A.class_member[i]; T.rank[i] = A.rank_in_class[i]; }
    if (lane_id < 9) { T.q[lane_id] = A.q[tid][lane_id]; T.magic[lane_id] = A.magic[tid][lane_id]; }
    if (lane_id < 10) { T.start[lane_id] = A.start[tid][lane_id]; T.base[lane_id] = A.class_base[lane_id]; }
}

// ---------------------------------------------------------------------------
// Decode one segment (one warp).  body points at the segment's states; words
// follow.  Writes sb bytes (XORed with xr) to dst.  Returns false on a
// malformed segment.
// ---------------------------------------------------------------------------
__device__ inline bool ans_decode_segment(const uint8_t *states, const uint8_t *words, uint32_t nw, uint32_t sb,
                                          const AnsSm &T, uint8_t xr, uint8_t *dst) {
    const int lane = threadIdx.x & 31;
    const uint32_t W = ans_seg_lanes(sb);
    uint32_t x = lane < (int)W ? ld_le32(states + 4 * lane) : kAnsL;
    bool ok = (x >= kAnsL);
    uint32_t s1 = T.start[1], s2 = T.start[2], s3 = T.start[3], s4 = T.start[4], s5 = T.start[5], s6 = T.start[6],
             s7 = T.start[7], s8 = T.start[8];
    uint32_t rd = 0;
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
        if (need) {
            const uint32_t pos = rd + __popc(m & lt);
            if (pos < nw) x = (x << 16) | ((uint32_t)words[2 * pos] | ((uint32_t)words[2 * pos + 1] << 8));
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
// coding).  Words are staged backwards in stage[0 .. cap).  Returns the word
// count; final states in x (lane < W).
// ---------------------------------------------------------------------------
__device__ inline uint32_t ans_encode_segment(const uint8_t *src, uint32_t sb, const AnsSm &T, uint8_t xr,
                                              uint16_t *stage, uint32_t cap, uint32_t &x_out) {
    const int lane = threadIdx.x & 31;
    const uint32_t W = ans_seg_lanes(sb);
    uint32_t x = kAnsL;
    uint32_t cnt = 0;
    const uint32_t rounds = (sb + W - 1) / W;
    const uint32_t gt = ~((2u << lane) - 1u);
    for (int r = (int)rounds - 1; r >= 0; r--) {
        const uint32_t j = (uint32_t)r * W + lane;
        const bool active = lane < (int)W && j < sb;
        uint32_t f = 1, c = 0;
        bool emit = false;
        if (active) {
            const uint32_t b = (uint32_t)(src[j] ^ xr);
            const uint32_t k = __popc(b);
            f = T.q[k];
            c = T.start[k] + T.rank[b] * f;
            emit = (uint64_t)x >= ((uint64_t)f << 17);
        }
        const uint32_t m = __ballot_sync(0xffffffffu, emit);
        if (emit) {
            const uint32_t pos = cnt + __popc(m & gt);
            if (pos < cap) stage[cap - 1 - pos] = (uint16_t)(x & 0xFFFF);
            x >>= 16;
        }
        cnt += __popc(m);
        if (active) x = ((x / f) << kAnsScale) + (x % f) + c;
    }
    x_out = x;
    return cnt;
}

// ---------------------------------------------------------------------------
// Standalone bitmap ANS (one warp per bitmap; segments sequential).
// ---------------------------------------------------------------------------
constexpr int kAnsStageWords = kAnsSeg;   // at most one word per byte

__global__ void __launch_bounds__(32) ans_encode_kernel(const uint8_t *__restrict__ bm, const uint64_t *__restrict__ bm_off,
                                                        const uint8_t *__restrict__ table, uint8_t *__restrict__ bodies,
                                                        const uint64_t *__restrict__ body_off,
                                                        uint64_t *__restrict__ body_bytes, int32_t *__restrict__ status,
                                                        const __grid_constant__ AnsTables A) {
    extern __shared__ __align__(16) uint8_t sm[];
    AnsSm &T = *reinterpret_cast<AnsSm *>(sm);
    uint16_t *stage = reinterpret_cast<uint16_t *>(sm + ((sizeof(AnsSm) + 15) & ~15));
    const int i = blockIdx.x, lane = threadIdx.x;
    const uint32_t nbytes = (uint32_t)(bm_off[i + 1] - bm_off[i]);
    const uint8_t tb = table[i];
    const int tid = (tb & 0x7F) - 1;
    const uint64_t cap = body_off[i + 1] - body_off[i];
    if (tid < 0 || tid >= 50 || nbytes == 0) {
        if (lane == 0) { status[i] = PIVCO_ERR_INVALID_ARG; body_bytes[i] = 0; }
        return;
    }
    load_ans_table(T, A, tid, lane, 32);
    __syncwarp();
    const uint8_t xr = (tb & 0x80) ? 0xFF : 0;
    const uint8_t *src = bm + bm_off[i];
    uint8_t *dst = bodies + body_off[i];
    const uint32_t S = ans_seg_count(nbytes);
    uint64_t pos = 4ull * S;
    bool ok = pos <= cap;
    for (uint32_t s = 0; s < S && ok; s++) {
        const uint32_t sb = min(kAnsSeg, nbytes - s * kAnsSeg), W = ans_seg_lanes(sb);
        uint32_t x;
        const uint32_t nw = ans_encode_segment(src + (size_t)s * kAnsSeg, sb, T, xr, stage, kAnsStageWords, x);
        __syncwarp();
        if (pos + 4ull * W + 2ull * nw > cap) { ok = false; break; }
        if (lane == 0) st_le32(dst + 4 * s, nw);
        if (lane < (int)W) st_le32(dst + pos + 4 * lane, x);
        pos += 4ull * W;
        for (uint32_t k = lane; k < nw; k += 32) {
            const uint16_t w = stage[kAnsStageWords - nw + k];
            dst[pos + 2 * k] = (uint8_t)w;
            dst[pos + 2 * k + 1] = (uint8_t)(w >> 8);
        }
        pos += 2ull * nw;
        __syncwarp();
    }
    if (lane == 0) { status[i] = ok ? PIVCO_OK : PIVCO_ERR_CAPACITY; body_bytes[i] = ok ? pos : 0; }
}

// locate segment s of an ANS body: returns byte offset of its states, its word count
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

__global__ void __launch_bounds__(32) ans_decode_kernel(const uint8_t *__restrict__ bodies, const uint64_t *__restrict__ body_off,
                                                        const uint8_t *__restrict__ table, uint8_t *__restrict__ bm,
                                                        const uint64_t *__restrict__ bm_off, int32_t *__restrict__ status,
                                                        const __grid_constant__ AnsTables A) {
    __shared__ AnsSm T;
    const int i = blockIdx.x, lane = threadIdx.x;
    const uint32_t nbytes = (uint32_t)(bm_off[i + 1] - bm_off[i]);
    const uint8_t tb = table[i];
    const int tid = (tb & 0x7F) - 1;
    const uint64_t blen = body_off[i + 1] - body_off[i];
    if (tid < 0 || tid >= 50 || nbytes == 0) {
        if (lane == 0) status[i] = PIVCO_ERR_INVALID_ARG;
        return;
    }
    load_ans_table(T, A, tid, lane, 32);
    __syncwarp();
    const uint8_t *body = bodies + body_off[i];
    const uint32_t S = ans_seg_count(nbytes);
    bool ok = true;
    uint64_t total = 4ull * S;
    for (uint32_t s = 0; s < S && ok; s++) {
        uint64_t sp; uint32_t nw;
        if (!ans_segment_at(body, blen, nbytes, s, sp, nw)) { ok = false; break; }
        const uint32_t sb = min(kAnsSeg, nbytes - s * kAnsSeg), W = ans_seg_lanes(sb);
        ok = ans_decode_segment(body + sp, body + sp + 4 * W, nw, sb, T, (tb & 0x80) ? 0xFF : 0,
                                bm + bm_off[i] + (size_t)s * kAnsSeg);
        total += 4ull * W + 2ull * nw;
    }
    if (ok && total != blen) ok = false;
    if (lane == 0) status[i] = ok ? PIVCO_OK : PIVCO_ERR_CORRUPT;
}

cudaError_t launch_ans_encode(const uint8_t *bm, const uint64_t *bm_off, const uint8_t *table, int nbm, uint8_t *bodies,
                              const uint64_t *body_off, uint64_t *body_bytes, int32_t *status, cudaStream_t st) {
    if (nbm <= 0) return cudaSuccess;
    const int smem = (int)(((sizeof(AnsSm) + 15) & ~15) + 2 * kAnsStageWords);
    cudaError_t e = cudaFuncSetAttribute(ans_encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    ans_encode_kernel<<<nbm, 32, smem, st>>>(bm, bm_off, table, bodies, body_off, body_bytes, status, host_ans_tables());
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_ans_decode(const uint8_t *bodies, const uint64_t *body_off, const uint8_t *table, int nbm, uint8_t *bm,
                              const uint64_t *bm_off, int32_t *status, cudaStream_t st) {
    if (nbm <= 0) return cudaSuccess;
    ans_decode_kernel<<<nbm, 32, 0, st>>>(bodies, body_off, table, bm, bm_off, status, host_ans_tables());
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// In-record ANS pass (encode side): one warp per block.  Every node written
// with marker 0xFF (selected, raw) is coded into the workspace slot of its
// block; bodies not smaller than the raw bitmap are dropped (the node stays
// raw, marker 0xFF).  Then the selected region is rewritten in breadth-first
// order; each final body starts no later than its raw copy and ends before the
// next raw copy, so the in-place rewrite never overwrites unread bytes.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32) ans_encode_blocks_kernel(const BlockLayout *__restrict__ layout, uint8_t *__restrict__ out,
                                                               const uint64_t *__restrict__ out_off,
                                                               uint64_t *__restrict__ rec_bytes, uint8_t *__restrict__ ws,
                                                               uint64_t ws_bytes, int32_t *__restrict__ status,
                                                               const __grid_constant__ AnsTables A) {
    extern __shared__ __align__(16) uint8_t sm[];
    AnsSm &T = *reinterpret_cast<AnsSm *>(sm);
    uint16_t *stage = reinterpret_cast<uint16_t *>(sm + ((sizeof(AnsSm) + 15) & ~15));
    __shared__ uint32_t s_body[256];     // ANS body bytes per node (0 = keep raw)
    const int b = blockIdx.x, lane = threadIdx.x;
    const BlockLayout &L = *reinterpret_cast<const BlockLayout *>(reinterpret_cast<const uint8_t *>(layout) +
                                                                   (size_t)b * kLayoutBytes);
    if (status[b] != PIVCO_OK || L.kind != 2 || L.n_sel == 0) return;
    uint8_t *rec = out + out_off[b];
    uint8_t *wslot = ws + out_off[b];
    const uint64_t wcap = (out_off[b] < ws_bytes) ? umin64(ws_bytes - out_off[b], out_off[b + 1] - out_off[b]) : 0;
    const int V = L.n_int;
    uint64_t wpos = 0;
    for (int v = 0; v < V; v++) {
        if (!L.sel[v]) continue;
        if (lane == 0) s_body[v] = 0;
        const uint8_t tb = L.sel[v];
        const int tid = (tb & 0x7F) - 1;
        const uint32_t raw = (L.nv[v] + 7) / 8;
        __syncwarp();
        load_ans_table(T, A, tid, lane, 32);
        __syncwarp();
        const uint8_t xr = (tb & 0x80) ? 0xFF : 0;
        const uint8_t *src = rec + L.body_off[v];
        const uint32_t S = ans_seg_count(raw);
        uint64_t pos = 4ull * S;
        bool ok = wpos + pos <= wcap && pos < raw;
        for (uint32_t s = 0; s < S && ok; s++) {
            const uint32_t sb = min(kAnsSeg, raw - s * kAnsSeg), W = ans_seg_lanes(sb);
            uint32_t x;
            const uint32_t nw = ans_encode_segment(src + (size_t)s * kAnsSeg, sb, T, xr, stage, kAnsStageWords, x);
            __syncwarp();
            const uint64_t np = pos + 4ull * W + 2ull * nw;
            if (np >= raw || wpos + np > wcap) { ok = false; break; }
            uint8_t *dst = wslot + wpos;
            if (lane == 0) st_le32(dst + 4 * s, nw);
            if (lane < (int)W) st_le32(dst + pos + 4 * lane, x);
            pos += 4ull * W;
            for (uint32_t k = lane; k < nw; k += 32) {
                const uint16_t w = stage[kAnsStageWords - nw + k];
                dst[pos + 2 * k] = (uint8_t)w;
                dst[pos + 2 * k + 1] = (uint8_t)(w >> 8);
            }
            pos += 2ull * nw;
            __syncwarp();
        }
        if (ok && lane == 0) s_body[v] = (uint32_t)pos;
        if (ok) wpos += pos;
        __syncwarp();
    }
    // rewrite the selected region in breadth-first order
    __threadfence_block();
    uint32_t q = 0xFFFFFFFFu;
    for (int v = 0; v < V; v++)
        if (L.sel[v]) { q = L.body_off[v]; break; }
    const uint32_t alen_off = (kNvOff + 5u * V + 3u) & ~3u;
    uint64_t wread = 0;
    int k = 0;
    for (int v = 0; v < V; v++) {
        if (!L.sel[v]) continue;
        const uint32_t raw = (L.nv[v] + 7) / 8;
        const uint32_t bl = s_body[v];
        uint32_t len;
        if (bl) {
            for (uint32_t i = lane; i < bl; i += 32) rec[q + i] = wslot[wread + i];
            wread += bl;
            len = bl;
            if (lane == 0) rec[kNvOff + 4 * V + v] = L.sel[v];
        } else {
            const uint8_t *src = rec + L.body_off[v];
            if (q != L.body_off[v])
                for (uint32_t base = 0; base < raw; base += 32) {
                    const uint32_t i = base + lane;
                    const uint8_t c = i < raw ? src[i] : 0;
                    __syncwarp();
                    if (i < raw) rec[q + i] = c;
                    __syncwarp();
                }
            len = raw;
        }
        if (lane == 0) st_le32(rec + alen_off + 4 * k, len);
        k++;
        q += len;
        __syncwarp();
    }
    const uint32_t total = (q + 15u) & ~15u;
    for (uint32_t i = q + lane; i < total; i += 32) rec[i] = 0;
    if (lane == 0) {
        st_le32(rec, total);
        rec_bytes[b] = total;
    }
}

cudaError_t launch_ans_encode_blocks(const BlockLayout *layout, int nblk, uint8_t *out, const uint64_t *out_off,
                                     uint64_t *rec_bytes, uint8_t *ws, size_t ws_bytes, int32_t *status, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    const int smem = (int)(((sizeof(AnsSm) + 15) & ~15) + 2 * kAnsStageWords);
    cudaError_t e = cudaFuncSetAttribute(ans_encode_blocks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    ans_encode_blocks_kernel<<<nblk, 32, smem, st>>>(layout, out, out_off, rec_bytes, ws, ws_bytes, status,
                                                     host_ans_tables());
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Decode plan.  Workspace layout:
//   [0, 64)            header: u64 total scratch, u32 total segments, u32 ticket
//   [64, ..)           u64 look-back states[nblk]
//                      u64 blk_scratch[nblk]   (byte offset in the scratch area)
//                      u32 blk_seg[nblk]       (first descriptor of the block)
//   fixed part end F   descriptors (16 B): u32 block, u16 node, u16 seg,
//                                          u32 body offset, u32 node scratch offset
//   align256(F + 16 * total_segs): scratch (ANS-decoded bitmaps)
// Per ANS node the scratch holds ceil(n_v/8) bytes rounded up to 16 plus 16
// bytes of slack for aligned word reads.
// ---------------------------------------------------------------------------
struct DecDesc {
    uint32_t block;
    uint16_t node;
    uint16_t seg;
    uint32_t body_off;
    uint32_t scratch_off;
};

__device__ inline uint32_t scratch_stride(uint32_t raw) { return ((raw + 15u) & ~15u) + 16u; }

// parse the parts of a record the plan needs; returns false if malformed.
// Fills body offsets for every node (raw region, then the selected region).
__device__ inline bool parse_bodies(const uint8_t *rec, uint64_t avail, uint32_t &V, uint32_t *nv, uint8_t *marker,
                                    uint32_t *body_off, uint32_t *body_len) {
    if (avail < kHdr) return false;
    const uint32_t rb = ld_le32(rec), kind = rec[10];
    V = (uint32_t)rec[8] | ((uint32_t)rec[9] << 8);
    if (rec[12] != 'P' || rec[13] != 'V' || rec[14] != 'C' || rec[15] != '1') return false;
    if (rb < kHdr || (rb & 15u) || rb > avail) return false;
    if (kind != 2) { V = 0; return kind <= 1; }
    if (V < 1 || V > 255 || rb < kNvOff + 5 * V) return false;
    uint32_t nsel = 0;
    for (uint32_t v = 0; v < V; v++) {
        nv[v] = ld_le32(rec + kNvOff + 4 * v);
        marker[v] = rec[kNvOff + 4 * V + v];
        if (marker[v]) {
            nsel++;
            if (marker[v] != kMarkRawSel && ((marker[v] & 0x7F) < 1 || (marker[v] & 0x7F) > 50)) return false;
        }
    }
    uint64_t off = (kNvOff + 5ull * V + 3) & ~3ull;
    const uint64_t alen_off = off;
    off += 4ull * nsel;
    if (off > rb) return false;
    for (uint32_t v = 0; v < V; v++)
        if (!marker[v]) { body_off[v] = (uint32_t)off; body_len[v] = (nv[v] + 7) / 8; off += body_len[v]; }
    uint32_t k = 0;
    for (uint32_t v = 0; v < V; v++)
        if (marker[v]) {
            body_off[v] = (uint32_t)off;
            body_len[v] = ld_le32(rec + alen_off + 4 * k++);
            off += body_len[v];
            if (off > rb) return false;
        }
    if (off > rb || ((off + 15) & ~15ull) != rb) return false;
    return true;
}

constexpr int kPlanThreads = 32;

__global__ void __launch_bounds__(kPlanThreads) decode_plan_kernel(const uint8_t *__restrict__ comp,
                                                                   const uint64_t *__restrict__ comp_off, int nblk,
                                                                   uint8_t *__restrict__ ws, uint64_t ws_bytes,
                                                                   int32_t *__restrict__ status) {
    __shared__ uint32_t nv[256], body_off[256], body_len[256];
    __shared__ uint8_t marker[256];
    __shared__ int s_tile;
    __shared__ uint64_t s_excl;
    uint64_t *hdr64 = reinterpret_cast<uint64_t *>(ws);
    uint32_t *hdr32 = reinterpret_cast<uint32_t *>(ws);
    uint64_t *states = reinterpret_cast<uint64_t *>(ws + 64);
    uint64_t *blk_scratch = states + nblk;
    uint32_t *blk_seg = reinterpret_cast<uint32_t *>(blk_scratch + nblk);
    DecDesc *desc = reinterpret_cast<DecDesc *>(ws + decode_ws_fixed_bytes(nblk));
    const int lane = threadIdx.x;
    if (lane == 0) s_tile = (int)atomicAdd(&hdr32[3], 1u);
    __syncwarp();
    const int b = s_tile;
    uint32_t V = 0;
    bool ok = false;
    if (lane == 0) ok = parse_bodies(comp + comp_off[b], comp_off[b + 1] - comp_off[b], V, nv, marker, body_off, body_len);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    V = __shfl_sync(0xffffffffu, V, 0);
    __syncwarp();
    uint64_t bytes = 0;
    uint32_t segs = 0;
    if (ok) {
        for (uint32_t v = lane; v < V; v += 32)
            if (marker[v] && marker[v] != kMarkRawSel) {
                const uint32_t raw = (nv[v] + 7) / 8;
                bytes += scratch_stride(raw);
                segs += ans_seg_count(raw);
            }
        for (int o = 16; o; o >>= 1) {
            bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
            segs += __shfl_xor_sync(0xffffffffu, segs, o);
        }
    }
    // packed (bytes: 40 bits, segments: 22 bits)
    if (lane == 0) {
        int to = 0;
        s_excl = lookback_exclusive(states, b, (bytes << 22) | segs, &to);
        const uint64_t ex_bytes = s_excl >> 22, ex_segs = s_excl & ((1u << 22) - 1);
        blk_scratch[b] = ex_bytes;
        blk_seg[b] = (uint32_t)ex_segs;
        status[b] = !ok ? PIVCO_ERR_CORRUPT : (to ? PIVCO_ERR_TIMEOUT : PIVCO_OK);
        if (b == nblk - 1) {
            hdr64[0] = ex_bytes + bytes;
            hdr32[2] = (uint32_t)(ex_segs + segs);
        }
    }
    __syncwarp();
    if (ok && V) {
        // descriptors in node order (one lane walks the nodes)
        if (lane == 0) {
            uint32_t k = (uint32_t)(s_excl & ((1u << 22) - 1)), soff = 0;
            const uint64_t fixed = decode_ws_fixed_bytes(nblk);
            for (uint32_t v = 0; v < V; v++)
                if (marker[v] && marker[v] != kMarkRawSel) {
                    const uint32_t raw = (nv[v] + 7) / 8, S = ans_seg_count(raw);
                    for (uint32_t s = 0; s < S; s++, k++) {
                        if (fixed + 16ull * (k + 1) <= ws_bytes) {
                            DecDesc d;
                            d.block = (uint32_t)b; d.node = (uint16_t)v; d.seg = (uint16_t)s;
                            d.body_off = body_off[v]; d.scratch_off = soff;
                            desc[k] = d;
                        }
                    }
                    soff += scratch_stride(raw);
                }
        }
    }
}

cudaError_t launch_decode_plan(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *ws, size_t ws_bytes,
                               int32_t *status, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    cudaError_t e = launch_zero_bytes(ws, 64 + 8ull * nblk, st);
    if (e != cudaSuccess) return e;
    decode_plan_kernel<<<nblk, kPlanThreads, 0, st>>>(comp, comp_off, nblk, ws, ws_bytes, status);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t read_decode_ws_need(const uint8_t *ws, int nblk, size_t *need, cudaStream_t st) {
    uint64_t h[2];
    cudaError_t e = cudaMemcpyAsync(h, ws, 16, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    const uint64_t total_scratch = h[0];
    const uint32_t segs = (uint32_t)(h[1] & 0xFFFFFFFFu);
    const size_t dstart = (decode_ws_fixed_bytes(nblk) + 16ull * segs + 255) & ~(size_t)255;
    *need = dstart + total_scratch;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// ANS decode of every planned segment: persistent grid, one warp per segment.
// ---------------------------------------------------------------------------
constexpr int kAnsDecWarps = 4;

__global__ void __launch_bounds__(32 * kAnsDecWarps) ans_decode_planned_kernel(const uint8_t *__restrict__ comp,
                                                                               const uint64_t *__restrict__ comp_off,
                                                                               int nblk, uint8_t *__restrict__ ws,
                                                                               uint64_t ws_bytes,
                                                                               int32_t *__restrict__ status,
                                                                               const __grid_constant__ AnsTables A) {
    __shared__ AnsSm T[kAnsDecWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t total = reinterpret_cast<const uint32_t *>(ws)[2];
    const uint64_t *blk_scratch = reinterpret_cast<const uint64_t *>(ws + 64) + nblk;
    const DecDesc *desc = reinterpret_cast<const DecDesc *>(ws + decode_ws_fixed_bytes(nblk));
    const uint64_t dstart = (decode_ws_fixed_bytes(nblk) + 16ull * total + 255) & ~255ull;
    const uint64_t scratch_cap = ws_bytes > dstart ? ws_bytes - dstart : 0;
    uint8_t *scratch = ws + dstart;
    const uint64_t fixed_need = decode_ws_fixed_bytes(nblk) + 16ull * total;
    for (uint32_t g = blockIdx.x * kAnsDecWarps + w; g < total; g += gridDim.x * kAnsDecWarps) {
        if (fixed_need > ws_bytes) break;
        const DecDesc d = desc[g];
        const int b = (int)d.block;
        if (status[b] != PIVCO_OK) continue;
        const uint8_t *rec = comp + comp_off[b];
        const uint32_t V = (uint32_t)rec[8] | ((uint32_t)rec[9] << 8);
        const uint8_t mk = rec[kNvOff + 4 * V + d.node];
        const uint32_t nvv = ld_le32(rec + kNvOff + 4 * d.node);
        const uint32_t raw = (nvv + 7) / 8;
        // body length from the alen table: index of this node among selected nodes
        uint32_t k = 0;
        for (uint32_t v = lane; v < d.node; v += 32) k += rec[kNvOff + 4 * V + v] != 0;
        for (int o = 16; o; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
        const uint32_t alen_off = (kNvOff + 5u * V + 3u) & ~3u;
        const uint32_t blen = ld_le32(rec + alen_off + 4 * k);
        const uint64_t sdst = blk_scratch[b] + d.scratch_off;
        bool ok = sdst + scratch_stride(raw) <= scratch_cap;
        uint64_t sp = 0;
        uint32_t nw = 0;
        if (ok) ok = ans_segment_at(rec + d.body_off, blen, raw, d.seg, sp, nw);
        if (ok) {
            load_ans_table(T[w], A, (mk & 0x7F) - 1, lane, 32);
            __syncwarp();
            const uint32_t sb = min(kAnsSeg, raw - d.seg * kAnsSeg), W = ans_seg_lanes(sb);
            const uint8_t *body = rec + d.body_off;
            ok = ans_decode_segment(body + sp, body + sp + 4 * W, nw, sb, T[w], (mk & 0x80) ? 0xFF : 0,
                                    scratch + sdst + (size_t)d.seg * kAnsSeg);
            // the last segment also checks that the body is fully consumed
            if (ok && d.seg + 1 == ans_seg_count(raw) && sp + 4ull * W + 2ull * nw != blen) ok = false;
            if (d.seg + 1 == ans_seg_count(raw) && lane < 16) {
                // zero the slack after the bitmap (aligned reads past its end)
                const uint64_t e = sdst + raw;
                scratch[e + lane] = 0;
            }
        }
        if (!ok && lane == 0) status[b] = PIVCO_ERR_CORRUPT;
        __syncwarp();
    }
}

cudaError_t launch_ans_decode_planned(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *ws,
                                      size_t ws_bytes, int32_t *status, cudaStream_t st) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    ans_decode_planned_kernel<<<sms * 8, 32 * kAnsDecWarps, 0, st>>>(comp, comp_off, nblk, ws, ws_bytes, status,
                                                                     host_ans_tables());
    return cudaGetLastError();
}

}  // namespace pv
