// Decode kernel: bottom-up merge through per-node rank directories (Sec. 3).
//
// One CTA decodes one block, in chunks of up to kChunk output symbols.  For a
// chunk, every internal node v needs a contiguous range of its bitmap: it
// starts at the node's cursor c_v (bits consumed by earlier chunks) and its
// length d_v is the number of the chunk's symbols whose code passes through
// v.  Top-down (demand pass), each node's range is staged into shared memory
// (shifted so that element k is bit k) and popcounted per 128-bit unit; the
// exclusive per-unit popcounts are the node's rank directory for this chunk
// (rank1 of any element = unit base + popcount inside the unit) and the
// node's total popcount is its right child's demand.  Bottom-up (merge pass,
// deepest level first), every node rebuilds its symbol sequence:
//   out_v[k] = bit ? R[rank1(k)] : L[k - rank1(k)]
// where L/R are the children's sequences in the next level buffer, or leaf
// constants (the MVV / MCV / MVC / MCC operations of Table 8).  The root's
// sequence is the chunk's output.
#include "pivco_dev.cuh"

namespace pv {

constexpr int kDecThreads = 512;
constexpr int kDecWarps = kDecThreads / 32;
constexpr int kDChunk = 16384;
constexpr int kDUnit = 128;
constexpr int kDBufBytes = kDChunk + 4 * 256;
constexpr int kDStageWords = 6144;
constexpr int kDMaxUnits = kDChunk * 15 / kDUnit + 256;

struct DecSmem {
    uint8_t buf[2][kDBufBytes];
    uint32_t stage[kDStageWords];
    uint32_t unit_base[kDMaxUnits];
    uint32_t cur[256];      // bits of node v consumed by earlier chunks
    uint32_t dem[256];      // bits of node v used by this chunk
    uint32_t span[256];     // span start of node v in its level buffer
    uint32_t ustart[256];   // first unit of node v (chunk-global numbering)
    uint32_t st_off[256];   // first staging word of node v
    uint32_t nv[256];
    uint32_t src_off[256];  // bitmap byte offset (record or scratch)
    uint32_t lvl_units[17]; // first unit of each depth
    uint32_t lvl_words[17]; // first staging word of each depth
    int32_t first[17];      // first node id of each depth
    int16_t child[256][2];
    uint8_t in_scratch[256];
    uint8_t lens[256];
    uint8_t sorted[256];
    uint8_t marker[256];
    uint16_t codes[256];
    int32_t rank_scratch[256];
    TreeShape ts;
    int32_t flag;           // error flag (corrupt)
};

__device__ inline int find_node_d(const uint32_t *key, int lo, int hi, uint32_t g) {
    while (hi - lo > 1) {
        const int m = (lo + hi) >> 1;
        if (key[m] <= g) lo = m; else hi = m;
    }
    return lo;
}

template <typename F, typename G>
__device__ inline uint32_t warp_scan_loop_d(int n, F f, G out) {
    const int lane = threadIdx.x & 31;
    uint32_t carry = 0;
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        const uint32_t x = i < n ? f(i) : 0;
        uint32_t inc = x;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (i < n) out(i, carry + inc - x);
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    return carry;
}

// 32 bits of a bitmap starting at bit `bit` of the byte array `base` (16-byte
// aligned allocation of at least `limit` bytes; words at or past limit read 0)
__device__ inline uint32_t bits32(const uint8_t *base, uint64_t bit, uint64_t limit) {
    const uint64_t wi = bit >> 5;
    const uint32_t sh = (uint32_t)(bit & 31);
    const uint32_t *w = reinterpret_cast<const uint32_t *>(base);
    const uint32_t lo = (4 * wi + 4 <= limit) ? __ldg(w + wi) : 0u;
    if (!sh) return lo;
    const uint32_t hi = (4 * wi + 8 <= limit) ? __ldg(w + wi + 1) : 0u;
    return __funnelshift_r(lo, hi, sh);
}

__global__ void __launch_bounds__(kDecThreads, 1) decode_kernel(const uint8_t *__restrict__ comp,
                                                                const uint64_t *__restrict__ comp_off,
                                                                int nblk, uint8_t *__restrict__ out,
                                                                const uint64_t *__restrict__ out_off,
                                                                const uint8_t *__restrict__ ws, uint64_t ws_bytes,
                                                                int32_t *__restrict__ status) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    DecSmem &S = *reinterpret_cast<DecSmem *>(smem_raw);
    const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (status[b] != PIVCO_OK) return;     // the plan / ANS pass already failed this block
    const uint8_t *rec = comp + comp_off[b];
    const uint64_t avail = comp_off[b + 1] - comp_off[b];
    uint8_t *dst = out + out_off[b];
    const uint64_t ocap = out_off[b + 1] - out_off[b];
    // ---- header ----
    const uint32_t rb = ld_le32(rec), n = ld_le32(rec + 4);
    const uint32_t V = (uint32_t)rec[8] | ((uint32_t)rec[9] << 8), kind = rec[10], aux = rec[11];
    if ((comp_off[b] & 15) || n != ocap || rb > avail) {   // plan validated magic / size / layout
        if (t == 0) status[b] = n != ocap ? PIVCO_ERR_CAPACITY : PIVCO_ERR_CORRUPT;
        return;
    }
    if (kind == 0) {
        if (t == 0 && (n != 0 || V != 0 || aux != 0 || rb != kHdr)) status[b] = PIVCO_ERR_CORRUPT;
        return;
    }
    if (kind == 1) {
        if (n == 0 || V != 0 || rb != kHdr) { if (t == 0) status[b] = PIVCO_ERR_CORRUPT; return; }
        for (uint32_t i = t; i < n; i += kDecThreads) dst[i] = (uint8_t)aux;
        return;
    }
    if (aux != 0 || n == 0) { if (t == 0) status[b] = PIVCO_ERR_CORRUPT; return; }
    // ---- tree from the code lengths ----
    if (t < 128) {
        const uint8_t x = rec[kLensOff + t];
        S.lens[2 * t] = x & 15;
        S.lens[2 * t + 1] = x >> 4;
    }
    if (t == 0) S.flag = 0;
    __syncthreads();
    build_tree_shape(S.lens, S.ts, S.codes, S.sorted, S.rank_scratch);
    if (!S.ts.ok || (uint32_t)S.ts.n_int != V) { if (t == 0) status[b] = PIVCO_ERR_CORRUPT; return; }
    const int maxd = S.ts.max_len;
    if (t < 17) S.first[t] = S.ts.first[t];
    if (t < (int)V) {
        const int d = node_depth(S.ts, t);
        S.child[t][0] = (int16_t)node_child(S.ts, S.sorted, t, d, 0);
        S.child[t][1] = (int16_t)node_child(S.ts, S.sorted, t, d, 1);
        S.nv[t] = ld_le32(rec + kNvOff + 4 * t);
        S.marker[t] = rec[kNvOff + 4 * V + t];
        S.cur[t] = 0;
    }
    __syncthreads();
    // body offsets (raw region, then the selected region) and scratch offsets
    if (t == 0) {
        int bad = S.nv[0] != n;
        uint32_t nsel = 0;
        for (uint32_t v = 0; v < V; v++) nsel += S.marker[v] != 0;
        uint32_t off = ((kNvOff + 5 * V + 3) & ~3u) + 4 * nsel;
        const uint32_t alen_off = (kNvOff + 5 * V + 3) & ~3u;
        for (uint32_t v = 0; v < V; v++)
            if (!S.marker[v]) { S.src_off[v] = off; S.in_scratch[v] = 0; off += (S.nv[v] + 7) / 8; }
        uint32_t k = 0, soff = 0;
        for (uint32_t v = 0; v < V; v++)
            if (S.marker[v]) {
                const uint32_t al = ld_le32(rec + alen_off + 4 * k++);
                const uint32_t raw = (S.nv[v] + 7) / 8;
                if (S.marker[v] == kMarkRawSel) {
                    if (al != raw) bad = 1;
                    S.src_off[v] = off; S.in_scratch[v] = 0;
                } else {
                    S.src_off[v] = soff; S.in_scratch[v] = 1;
                    soff += ((raw + 15u) & ~15u) + 16u;
                }
                off += al;
            }
        if (((off + 15u) & ~15u) != rb) bad = 1;
        for (uint32_t v = 0; v < V; v++) {
            if (S.nv[v] < 2) bad = 1;
            for (int c = 0; c < 2; c++) if (S.child[v][c] >= 0 && S.nv[S.child[v][c]] > S.nv[v]) bad = 1;
        }
        S.flag = bad;
    }
    __syncthreads();
    if (S.flag) { if (t == 0) status[b] = PIVCO_ERR_CORRUPT; return; }
    // scratch area of this block (ANS-decoded bitmaps)
    const uint8_t *scratch = nullptr;
    uint64_t scratch_lim = 0;
    {
        const uint32_t total_segs = reinterpret_cast<const uint32_t *>(ws)[2];
        const uint64_t *blk_scratch = reinterpret_cast<const uint64_t *>(ws + 64) + nblk;
        const uint64_t dstart = (decode_ws_fixed_bytes(nblk) + 16ull * total_segs + 255) & ~255ull;
        scratch = ws + dstart + blk_scratch[b];
        scratch_lim = ws_bytes > dstart + blk_scratch[b] ? ws_bytes - dstart - blk_scratch[b] : 0;
    }
    // chunk size: the staging must hold every node's range (<= maxd bits per symbol)
    const int64_t ceff64 = ((int64_t)(kDStageWords - (int)V - 32) * 32 / maxd) & ~(int64_t)(kDUnit - 1);
    const uint32_t ceff = (uint32_t)(ceff64 < kDChunk ? ceff64 : kDChunk);

    for (uint32_t P = 0; P < n; P += ceff) {
        const uint32_t cc = min(ceff, n - P);
        // ---------------- demand pass (top-down) ----------------
        if (t == 0) { S.dem[0] = cc; S.span[0] = 0; S.lvl_units[0] = 0; S.lvl_words[0] = 0; }
        __syncthreads();
        for (int d = 0; d < maxd; d++) {
            const int f0 = S.first[d], f1 = S.first[d + 1];
            if (warp == 0) {
                const uint32_t u = warp_scan_loop_d(f1 - f0, [&](int i) { return (S.dem[f0 + i] + kDUnit - 1) / kDUnit; },
                                                    [&](int i, uint32_t p) { S.ustart[f0 + i] = S.lvl_units[d] + p; });
                const uint32_t w = warp_scan_loop_d(f1 - f0, [&](int i) { return (S.dem[f0 + i] + 31) / 32; },
                                                    [&](int i, uint32_t p) { S.st_off[f0 + i] = S.lvl_words[d] + p; });
                if (lane == 0) { S.lvl_units[d + 1] = S.lvl_units[d] + u; S.lvl_words[d + 1] = S.lvl_words[d] + w; }
            }
            __syncthreads();
            // stage the ranges of this depth's nodes, shifted to bit 0
            const uint32_t w0 = S.lvl_words[d], w1 = S.lvl_words[d + 1];
            for (uint32_t i = w0 + t; i < w1; i += kDecThreads) {
                const int v = find_node_d(S.st_off, f0, f1, i);
                const uint32_t j = i - S.st_off[v];
                const uint64_t bit = (uint64_t)S.cur[v] + 32ull * j;
                uint32_t word;
                if (S.in_scratch[v]) word = bits32(scratch + S.src_off[v], bit, scratch_lim > S.src_off[v] ? scratch_lim - S.src_off[v] : 0);
                else word = bits32(rec, bit + 8ull * S.src_off[v], rb);
                const uint32_t left = S.dem[v] - 32 * j;
                if (left < 32) word &= (1u << left) - 1u;
                S.stage[i] = word;
            }
            __syncthreads();
            // rank directory: per-unit exclusive popcounts; children's demands
            for (int v = f0 + warp; v < f1; v += kDecWarps) {
                const uint32_t dv = S.dem[v];
                if (!dv) {
                    if (lane < 2 && S.child[v][lane] >= 0) S.dem[S.child[v][lane]] = 0;
                    continue;
                }
                const uint32_t nu = (dv + kDUnit - 1) / kDUnit, u0 = S.ustart[v], so = S.st_off[v], nwd = (dv + 31) / 32;
                const uint32_t ones = warp_scan_loop_d((int)nu, [&](int i) {
                    uint32_t pc = 0;
                    for (uint32_t q = 0; q < 4; q++) { const uint32_t wj = 4 * i + q; if (wj < nwd) pc += __popc(S.stage[so + wj]); }
                    return pc;
                }, [&](int i, uint32_t p) { S.unit_base[u0 + i] = p; });
                if (lane < 2) {
                    const int c = S.child[v][lane];
                    if (c >= 0) {
                        const uint32_t dc = lane ? ones : dv - ones;
                        S.dem[c] = dc;
                        if ((uint64_t)S.cur[c] + dc > S.nv[c]) S.flag = 1;
                    }
                }
            }
            __syncthreads();
            // spans of the next depth
            if (d + 1 < maxd && warp == 0) {
                const int g0 = S.first[d + 1], g1 = S.first[d + 2 <= 16 ? d + 2 : 16];
                warp_scan_loop_d(g1 - g0, [&](int i) { return (S.dem[g0 + i] + 3u) & ~3u; },
                                 [&](int i, uint32_t p) { S.span[g0 + i] = p; });
            }
            __syncthreads();
            if (S.flag) break;
        }
        if (S.flag) break;
        // ---------------- merge pass (bottom-up) ----------------
        for (int d = maxd - 1; d >= 0; d--) {
            const int f0 = S.first[d], f1 = S.first[d + 1];
            const uint8_t *bin = S.buf[(d + 1) & 1];
            uint8_t *bout = S.buf[d & 1];
            const uint32_t g0 = S.lvl_units[d], g1 = S.lvl_units[d + 1];
            for (uint32_t g = g0 + warp; g < g1; g += kDecWarps) {
                const int v = find_node_d(S.ustart, f0, f1, g);
                const uint32_t k0 = (g - S.ustart[v]) * kDUnit, k = k0 + 4 * lane;
                const uint32_t dv = S.dem[v], q = lane >> 3;
                const uint32_t wq = (k0 / 32 + q < (dv + 31) / 32) ? S.stage[S.st_off[v] + k0 / 32 + q] : 0u;
                const uint32_t w0 = __shfl_sync(0xffffffffu, wq, 0), w1 = __shfl_sync(0xffffffffu, wq, 8),
                               w2 = __shfl_sync(0xffffffffu, wq, 16);
                uint32_t r = S.unit_base[g] + (q > 0 ? __popc(w0) : 0) + (q > 1 ? __popc(w1) : 0) +
                             (q > 2 ? __popc(w2) : 0) + __popc(wq & ((1u << (4 * (lane & 7))) - 1u));
                if (k < dv) {
                    const uint32_t nib = (wq >> (4 * (lane & 7))) & 15u;
                    const uint32_t nval = min(4u, dv - k);
                    const int c0 = S.child[v][0], c1 = S.child[v][1];
                    const uint32_t sp0 = c0 >= 0 ? S.span[c0] : 0, sp1 = c1 >= 0 ? S.span[c1] : 0;
                    uint32_t packed = 0;
                    for (uint32_t j = 0; j < nval; j++) {
                        const uint32_t bit = (nib >> j) & 1u;
                        uint32_t sym;
                        if (bit) sym = c1 >= 0 ? bin[sp1 + r] : (uint32_t)(-c1 - 1);
                        else sym = c0 >= 0 ? bin[sp0 + (k + j - r)] : (uint32_t)(-c0 - 1);
                        packed |= sym << (8 * j);
                        r += bit;
                    }
                    *reinterpret_cast<uint32_t *>(bout + S.span[v] + k) = packed;
                }
            }
            __syncthreads();
        }
        // ---------------- root output ----------------
        {
            uint8_t *o = dst + P;
            const uint8_t *src = S.buf[0];
            if ((reinterpret_cast<uintptr_t>(o) & 15) == 0) {
                const uint32_t nv16 = cc / 16;
                for (uint32_t i = t; i < nv16; i += kDecThreads)
                    reinterpret_cast<uint4 *>(o)[i] = reinterpret_cast<const uint4 *>(src)[i];
                for (uint32_t i = nv16 * 16 + t; i < cc; i += kDecThreads) o[i] = src[i];
            } else {
                for (uint32_t i = t; i < cc; i += kDecThreads) o[i] = src[i];
            }
        }
        // advance cursors
        for (uint32_t v = t; v < V; v += kDecThreads) S.cur[v] += S.dem[v];
        __syncthreads();
    }
    // every node's bitmap must be consumed exactly; pad bits must be zero
    int bad = S.flag;
    for (uint32_t v = t; v < V && !bad; v += kDecThreads) {
        if (S.cur[v] != S.nv[v]) bad = 1;
        else if (S.nv[v] & 7) {
            const uint32_t byte = S.nv[v] >> 3;
            const uint8_t last = S.in_scratch[v] ? scratch[S.src_off[v] + byte] : rec[S.src_off[v] + byte];
            if (last >> (S.nv[v] & 7)) bad = 1;
        }
    }
    bad = __syncthreads_or(bad);
    if (t == 0 && bad) status[b] = PIVCO_ERR_CORRUPT;
}

cudaError_t launch_decode(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *out,
                          const uint64_t *out_off, uint8_t *ws, size_t ws_bytes, int32_t *status, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    cudaError_t e = launch_decode_plan(comp, comp_off, nblk, ws, ws_bytes, status, st);
    if (e != cudaSuccess) return e;
    e = launch_ans_decode_planned(comp, comp_off, nblk, ws, ws_bytes, status, st);
    if (e != cudaSuccess) return e;
    const int smem = (int)sizeof(DecSmem);
    e = cudaFuncSetAttribute(decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    decode_kernel<<<nblk, kDecThreads, smem, st>>>(comp, comp_off, nblk, out, out_off, ws, ws_bytes, status);
    return cudaGetLastError();
}

}  // namespace pv
