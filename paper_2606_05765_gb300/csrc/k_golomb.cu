// PivCo-Golomb (App. G): pivoted coding applied to Golomb coding with a list
// of bitmaps in place of a tree.  The Golomb parameter is 1 (the unary
// code): value v is v continue bits then one stop bit (1); bitmap j holds,
// in sequence order, the j-th code bit of every value v >= j (1: v == j,
// 0: v > j).  The record layout is in include/pivco.h.
//
//   plan    one CTA per block: the values' histogram gives m (largest value
//           + 1) and n_j (values >= j, a suffix sum), hence the exact record
//           size.
//   encode  one CTA per block, top-down over the list: level j holds the
//           values >= j in order (shared memory); a warp takes 32 of them at
//           a time, the stop bits are one ballot (the bitmap word) and the
//           continuing values are compacted into the next level by ballot
//           and popcount, at offsets that a count pass and a prefix over the
//           warps give each warp.
//   decode  one CTA per block, bottom-up (App. G's merge_vec_cst_plus1 with
//           cst 0xFF): out_j[i] = B_j[i] ? 0x00 : out_{j+1}[rank0(B_j, i)] + 1,
//           ranks from a popcount pass and a prefix over the warps.
#include "pivco_dev.cuh"

namespace pv {

constexpr int kGThreads = 256;
constexpr int kGWarps = kGThreads / 32;
constexpr uint32_t kGMaxBlock = PIVCO_GOLOMB_MAX_BLOCK;   // values per block
constexpr uint32_t kGKind = 4;

struct __align__(16) GolombSmem {
    uint8_t buf[2][kGMaxBlock + 64];   // the current level and the next
    uint32_t cnt[256];
    uint32_t wcnt[kGWarps];
    uint32_t start[257];               // byte offset of bitmap j in the record
    uint32_t nj[257];
    uint32_t bad, m;
};

__device__ inline uint32_t g_size(uint32_t m, const uint32_t *nj) {
    uint64_t bytes = 16 + 4ull * m;
    for (uint32_t j = 0; j < m; j++) bytes += (nj[j] + 7) / 8;
    return (uint32_t)((bytes + 15) & ~15ull);
}

// Histogram of the block's values (counts aggregated per warp step), the
// largest value, and n_j = values >= j (suffix sums).  Whole CTA.
__device__ inline void g_counts(const uint8_t *src, uint32_t n, GolombSmem &S) {
    const int t = threadIdx.x, lane = t & 31;
    S.cnt[t] = 0;
    __syncthreads();
    for (uint32_t base = 32u * (t >> 5); base < n; base += 32u * kGWarps) {   // warp-uniform trip count
        const uint32_t i = base + lane;
        const bool act = i < n;
        const uint32_t v = act ? src[i] : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, v);
        if (act && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&S.cnt[v], (uint32_t)__popc(peers));
    }
    __syncthreads();
    if (t < 32) {
        // suffix sums over 256 counts: lane l holds values 8l .. 8l + 7
        uint32_t c[8], s = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) { c[k] = S.cnt[8 * lane + k]; s += c[k]; }
        uint32_t inc = s;   // inclusive suffix over lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_down_sync(0xffffffffu, inc, o);
            if (lane + o < 32) inc += y;
        }
        uint32_t run = inc - s;
        for (int k = 7; k >= 0; k--) { run += c[k]; S.nj[8 * lane + k] = run; }
        // m = largest value + 1 (0 for an empty block)
        uint32_t mx = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) if (c[k]) mx = 8u * lane + k + 1;
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (lane == 0) { S.m = mx; S.nj[256] = 0; }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kGThreads) golomb_plan_kernel(const uint8_t *__restrict__ in,
                                                                const uint64_t *__restrict__ blk_off,
                                                                uint64_t *__restrict__ rec_size,
                                                                int32_t *__restrict__ status) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    GolombSmem &S = *reinterpret_cast<GolombSmem *>(smem_raw);
    const int b = blockIdx.x, t = threadIdx.x;
    const uint64_t n = blk_off[b + 1] - blk_off[b];
    if (n > kGMaxBlock) {
        if (t == 0) { rec_size[b] = 16; status[b] = PIVCO_ERR_INVALID_ARG; }
        return;
    }
    g_counts(in + blk_off[b], (uint32_t)n, S);
    if (t == 0) {
        rec_size[b] = g_size(S.m, S.nj);
        status[b] = PIVCO_OK;
    }
}

__global__ void __launch_bounds__(kGThreads) golomb_encode_kernel(const uint8_t *__restrict__ in,
                                                                  const uint64_t *__restrict__ blk_off,
                                                                  uint8_t *__restrict__ out,
                                                                  const uint64_t *__restrict__ out_off,
                                                                  uint64_t *__restrict__ rec_bytes,
                                                                  int32_t *__restrict__ status) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    GolombSmem &S = *reinterpret_cast<GolombSmem *>(smem_raw);
    const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint64_t n64 = blk_off[b + 1] - blk_off[b];
    const uint8_t *src = in + blk_off[b];
    uint8_t *rec = out + out_off[b];
    const uint64_t cap = out_off[b + 1] - out_off[b];
    if (n64 > kGMaxBlock) {
        if (t == 0) { rec_bytes[b] = 0; status[b] = PIVCO_ERR_INVALID_ARG; }
        return;
    }
    const uint32_t n = (uint32_t)n64;
    g_counts(src, n, S);
    const uint32_t m = S.m, size = g_size(m, S.nj);
    if (cap < size) {
        if (t == 0) { rec_bytes[b] = 0; status[b] = PIVCO_ERR_CAPACITY; }
        return;
    }
    // header, counts, bitmap starts; the record is zeroed first (bits are
    // written a byte at a time, pad bits stay 0)
    for (uint32_t i = t; i < size; i += kGThreads) rec[i] = 0;
    if (t == 0) {
        uint32_t off = 16 + 4 * m;
        for (uint32_t j = 0; j < m; j++) { S.start[j] = off; off += (S.nj[j] + 7) / 8; }
    }
    // the values: level 0
    for (uint32_t i = t; i < n; i += kGThreads) S.buf[0][i] = src[i];
    __syncthreads();
    if (t < 16) {
        uint8_t v = 0;
        if (t < 4) v = (uint8_t)(size >> (8 * t));
        else if (t < 8) v = (uint8_t)(n >> (8 * (t - 4)));
        else if (t == 8) v = (uint8_t)m;
        else if (t == 9) v = (uint8_t)(m >> 8);
        else if (t == 10) v = (uint8_t)kGKind;
        else if (t >= 12) v = (uint8_t)"PVG1"[t - 12];
        rec[t] = v;
    }
    for (uint32_t j = t; j < m; j += kGThreads)
        for (int q = 0; q < 4; q++) rec[16 + 4 * j + q] = (uint8_t)(S.nj[j] >> (8 * q));
    __syncthreads();
    uint32_t cur = 0;
    for (uint32_t j = 0; j < m; j++) {
        const uint32_t len = S.nj[j];
        const uint8_t *lv = S.buf[cur];
        uint8_t *nx = S.buf[cur ^ 1];
        // each warp a contiguous run of whole 32-value groups
        const uint32_t per = ((len + 32u * kGWarps - 1) / (32u * kGWarps)) * 32u;
        const uint32_t w0 = min(len, per * warp), w1 = min(len, w0 + per);
        uint32_t cont = 0;
        for (uint32_t k = w0; k < w1; k += 32) {
            const uint32_t i = k + lane;
            cont += __popc(__ballot_sync(0xffffffffu, i < w1 && lv[i] > j));
        }
        if (lane == 0) S.wcnt[warp] = cont;
        __syncthreads();
        uint32_t base = 0;
        for (int w = 0; w < warp; w++) base += S.wcnt[w];
        const uint32_t lt = (1u << lane) - 1u;
        uint8_t *bm = rec + S.start[j];
        for (uint32_t k = w0; k < w1; k += 32) {
            const uint32_t i = k + lane;
            const uint32_t v = i < w1 ? lv[i] : 0u;
            const uint32_t stop = __ballot_sync(0xffffffffu, i < w1 && v == j);
            const uint32_t go = __ballot_sync(0xffffffffu, i < w1 && v > j);
            // the word's bytes (k is a multiple of 32: whole bytes of bitmap j)
            if (lane < 4 && k + 8u * lane < len) bm[(k >> 3) + lane] = (uint8_t)(stop >> (8 * lane));
            if ((go >> lane) & 1u) nx[base + __popc(go & lt)] = (uint8_t)v;
            base += __popc(go);
        }
        __syncthreads();
        cur ^= 1u;
    }
    if (t == 0) { rec_bytes[b] = size; status[b] = PIVCO_OK; }
}

__global__ void __launch_bounds__(kGThreads) golomb_decode_kernel(const uint8_t *__restrict__ comp,
                                                                  const uint64_t *__restrict__ comp_off,
                                                                  uint8_t *__restrict__ out,
                                                                  const uint64_t *__restrict__ out_off,
                                                                  int32_t *__restrict__ status) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    GolombSmem &S = *reinterpret_cast<GolombSmem *>(smem_raw);
    const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint8_t *rec = comp + comp_off[b];
    const uint64_t avail = comp_off[b + 1] - comp_off[b];
    const uint64_t ocap = out_off[b + 1] - out_off[b];
    uint8_t *dst = out + out_off[b];
    // header checks (one decision for the whole CTA)
    if (t == 0) {
        uint32_t bad = avail < 16;
        uint32_t size = 0, n = 0, m = 0;
        if (!bad) {
            size = ld_le32(rec);
            n = ld_le32(rec + 4);
            m = (uint32_t)rec[8] | ((uint32_t)rec[9] << 8);
            bad = rec[12] != 'P' || rec[13] != 'V' || rec[14] != 'G' || rec[15] != '1' || rec[10] != kGKind ||
                  rec[11] != 0 || (size & 15) || size > avail || size < 16 || m > 256 || (n == 0) != (m == 0) ||
                  16ull + 4ull * m > size || n > kGMaxBlock;
        }
        if (!bad) {
            uint64_t off = 16 + 4ull * m;
            for (uint32_t j = 0; j < m && !bad; j++) {
                const uint32_t c = ld_le32(rec + 16 + 4 * j);
                if ((j == 0 && c != n) || (j && c > S.nj[j - 1]) || c == 0) bad = 1;
                S.nj[j] = c;
                S.start[j] = (uint32_t)off;
                off += (c + 7) / 8;
            }
            if (!bad && ((off + 15) & ~15ull) != size) bad = 1;
        }
        S.bad = bad ? PIVCO_ERR_CORRUPT : (n != ocap ? PIVCO_ERR_CAPACITY : PIVCO_OK);
        S.m = m;
        S.nj[m < 256 ? m : 256] = 0;
    }
    __syncthreads();
    if (S.bad) {
        if (t == 0) status[b] = (int32_t)S.bad;
        return;
    }
    const uint32_t m = S.m;
    uint32_t cur = 0;   // the child's values are in buf[cur]
    int bad = 0;
    for (int j = (int)m - 1; j >= 0; j--) {
        const uint32_t len = S.nj[j], clen = S.nj[j + 1];
        const uint8_t *bm = rec + S.start[j];
        const uint8_t *child = S.buf[cur];
        uint8_t *lv = S.buf[cur ^ 1];
        const uint32_t per = ((len + 32u * kGWarps - 1) / (32u * kGWarps)) * 32u;
        const uint32_t w0 = min(len, per * warp), w1 = min(len, w0 + per);
        // the stop bits of this warp's run, then the ones before it
        uint32_t ones = 0;
        for (uint32_t k = w0 + 32u * lane; k < w1; k += 1024) {
            uint32_t word = 0;
            for (int q = 0; q < 4; q++)
                if (k + 8u * q < len) word |= (uint32_t)bm[(k >> 3) + q] << (8 * q);
            if (w1 - k < 32) word &= (1u << (w1 - k)) - 1u;
            ones += __popc(word);
        }
        ones = __reduce_add_sync(0xffffffffu, ones);
        if (lane == 0) S.wcnt[warp] = ones;
        __syncthreads();
        uint32_t r1 = 0, tot = 0;
        for (int w = 0; w < kGWarps; w++) {
            const uint32_t c = S.wcnt[w];
            if (w < warp) r1 += c;
            tot += c;
        }
        if (tot != len - clen) bad = 1;   // the stops and the values that continue must match the counts
        const uint32_t lt = (1u << lane) - 1u;
        for (uint32_t k = w0; k < w1; k += 32) {
            uint32_t word = 0;
            for (int q = 0; q < 4; q++)
                if (k + 8u * q < len) word |= (uint32_t)bm[(k >> 3) + q] << (8 * q);
            if (w1 - k < 32) word &= (1u << (w1 - k)) - 1u;
            const uint32_t i = k + lane;
            if (i < w1) {
                const uint32_t bit = (word >> lane) & 1u;
                const uint32_t z = i - (r1 + __popc(word & lt));   // zeros before i: the child's index
                uint8_t v = 0;
                if (!bit) v = z < clen ? (uint8_t)(child[z] + 1u) : 0u;
                lv[i] = v;
            }
            r1 += __popc(word);
        }
        // pad bits of the last byte are zero
        if (t == 0 && (len & 7) && (bm[len >> 3] >> (len & 7))) bad = 1;
        __syncthreads();
        cur ^= 1u;
    }
    if (__syncthreads_or(bad)) {
        if (t == 0) status[b] = PIVCO_ERR_CORRUPT;
        return;
    }
    const uint32_t n = S.nj[0];
    for (uint32_t i = t; i < (m ? n : 0u); i += kGThreads) dst[i] = S.buf[cur][i];
    if (t == 0) status[b] = PIVCO_OK;
}

static cudaError_t g_attr(const void *fn) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GolombSmem));
}

cudaError_t launch_golomb_plan(const uint8_t *in, const uint64_t *blk_off, int nblk, uint64_t *rec_size,
                               int32_t *status, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    cudaError_t e = g_attr((const void *)golomb_plan_kernel);
    if (e != cudaSuccess) return e;
    golomb_plan_kernel<<<nblk, kGThreads, sizeof(GolombSmem), st>>>(in, blk_off, rec_size, status);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_golomb_encode(const uint8_t *in, const uint64_t *blk_off, int nblk, uint8_t *out,
                                 const uint64_t *out_off, uint64_t *rec_bytes, int32_t *status, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    cudaError_t e = g_attr((const void *)golomb_encode_kernel);
    if (e != cudaSuccess) return e;
    golomb_encode_kernel<<<nblk, kGThreads, sizeof(GolombSmem), st>>>(in, blk_off, out, out_off, rec_bytes, status);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_golomb_decode(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *out,
                                 const uint64_t *out_off, int32_t *status, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    cudaError_t e = g_attr((const void *)golomb_decode_kernel);
    if (e != cudaSuccess) return e;
    golomb_decode_kernel<<<nblk, kGThreads, sizeof(GolombSmem), st>>>(comp, comp_off, out, out_off, status);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t prepare_golomb_kernels() {
    cudaError_t e = g_attr((const void *)golomb_plan_kernel);
    if (e == cudaSuccess) e = g_attr((const void *)golomb_encode_kernel);
    if (e == cudaSuccess) e = g_attr((const void *)golomb_decode_kernel);
    return e;
}

}  // namespace pv
