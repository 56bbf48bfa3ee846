// Selective ANS of node bitmaps (Sec. 5.2): the standalone bitmap coder /
// decoder and the in-record ANS pass of the encoder.
#include "ans_dev.cuh"

namespace pv {
// ---------------------------------------------------------------------------
// Standalone bitmap ANS (one warp per bitmap; segments sequential).
// ---------------------------------------------------------------------------
constexpr int kAnsStageWords = 4096;      // words staged in shared memory (the rest of a segment's go to global memory)

// The words of a coded segment in decoder order at dst (one warp): word k is
// emission nw - 1 - k.  Emissions cap .. nw - 1 were written at dst in
// emission order (ans_encode_segment's ovf): reversed in place, they become
// words 0 .. nw - cap - 1; the staged emissions 0 .. cap - 1 are the rest.
__device__ inline void ans_place_words(const uint16_t *stage, uint32_t cap, uint32_t nw, uint8_t *dst) {
    const int lane = threadIdx.x & 31;
    if (nw > cap) {
        const uint32_t L = nw - cap;
        for (uint32_t i0 = 0; i0 < L / 2; i0 += 32) {
            const uint32_t i = i0 + lane, j = L - 1 - i;
            uint8_t a0 = 0, a1 = 0, b0 = 0, b1 = 0;
            if (i < L / 2) { a0 = dst[2 * i]; a1 = dst[2 * i + 1]; b0 = dst[2 * j]; b1 = dst[2 * j + 1]; }
            __syncwarp();
            if (i < L / 2) { dst[2 * i] = b0; dst[2 * i + 1] = b1; dst[2 * j] = a0; dst[2 * j + 1] = a1; }
            __syncwarp();
        }
    }
    const uint32_t ns = nw < cap ? nw : cap;
    for (uint32_t k = nw - ns + lane; k < nw; k += 32) {
        const uint16_t w = stage[cap - nw + k];
        dst[2 * k] = (uint8_t)w;
        dst[2 * k + 1] = (uint8_t)(w >> 8);
    }
}

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
    load_ans_table(T, A, tid, lane, 32, true);
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
        const uint8_t *ss = src + (size_t)s * kAnsSeg;
        // words past the stage go where the segment's words will be (after its states)
        const uint64_t wo = pos + 4ull * W;
        const uint32_t room = wo < cap ? (uint32_t)min((cap - wo) / 2, (uint64_t)0xFFFFFFFFu) : 0u;
        const uint32_t nw = ans_encode_segment(ss, sb, T, xr, stage, kAnsStageWords, dst + wo, room, x);
        __syncwarp();
        if (pos + 4ull * W + 2ull * nw > cap) { ok = false; break; }
        if (lane == 0) st_le32(dst + 4 * s, nw);
        if (lane < (int)W) st_le32(dst + pos + 4 * lane, x);
        pos += 4ull * W;
        __syncwarp();
        ans_place_words(stage, kAnsStageWords, nw, dst + pos);
        pos += 2ull * nw;
        __syncwarp();
    }
    if (lane == 0) { status[i] = ok ? PIVCO_OK : PIVCO_ERR_CAPACITY; body_bytes[i] = ok ? pos : 0; }
}

// locate segment s of an ANS body: returns byte offset of its states, its word count
__global__ void __launch_bounds__(32) ans_decode_kernel(const uint8_t *__restrict__ bodies, const uint64_t *__restrict__ body_off,
                                                        const uint8_t *__restrict__ table, uint8_t *__restrict__ bm,
                                                        const uint64_t *__restrict__ bm_off, int32_t *__restrict__ status,
                                                        const __grid_constant__ AnsTables A) {
    __shared__ AnsSm T;
    __shared__ uint8_t wst[2 * kAnsWordWin];
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
                                bm + bm_off[i] + (size_t)s * kAnsSeg, wst);
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
        load_ans_table(T, A, tid, lane, 32, true);
        __syncwarp();
        const uint8_t xr = (tb & 0x80) ? 0xFF : 0;
        const uint8_t *src = rec + L.body_off[v];
        const uint32_t S = ans_seg_count(raw);
        uint64_t pos = 4ull * S;
        bool ok = wpos + pos <= wcap && pos < raw;
        for (uint32_t s = 0; s < S && ok; s++) {
            const uint32_t sb = min(kAnsSeg, raw - s * kAnsSeg), W = ans_seg_lanes(sb);
            uint32_t x;
            const uint8_t *ss = src + (size_t)s * kAnsSeg;
            uint8_t *dst = wslot + wpos;
            // words past the stage go where the segment's words will be
            const uint64_t wo = wpos + pos + 4ull * W;
            const uint32_t room = wo < wcap ? (uint32_t)min((wcap - wo) / 2, (uint64_t)0xFFFFFFFFu) : 0u;
            const uint32_t nw = ans_encode_segment(ss, sb, T, xr, stage, kAnsStageWords, dst + pos + 4ull * W, room, x);
            __syncwarp();
            const uint64_t np = pos + 4ull * W + 2ull * nw;
            if (np >= raw || wpos + np > wcap) { ok = false; break; }
            if (lane == 0) st_le32(dst + 4 * s, nw);
            if (lane < (int)W) st_le32(dst + pos + 4 * lane, x);
            pos += 4ull * W;
            __syncwarp();
            ans_place_words(stage, kAnsStageWords, nw, dst + pos);
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


}  // namespace pv

namespace pv {
cudaError_t prepare_ans_kernels() {
    const int smem = (int)(((sizeof(AnsSm) + 15) & ~15) + 2 * kAnsStageWords);
    cudaError_t e = cudaFuncSetAttribute(ans_encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(ans_encode_blocks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}
}  // namespace pv
