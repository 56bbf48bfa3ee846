// Encode kernel: per-node bitmap emission by stable partition (Sec. 4, Table 11).
//
// One CTA encodes one block.  The block is processed in chunks of up to
// kChunk symbols.  Within a chunk the symbols sit in a "level buffer" ordered
// by (d-bit code prefix, block position): at depth 0 this is the chunk itself,
// and each node's symbols occupy one aligned span.  For every depth d the CTA
//   A) computes the code bit d of every symbol (the node's bitmap bits, in
//      block order) and ORs them into a shared-memory window of the node's
//      bitmap,
//   B) scans the per-unit popcounts of each node (rank directory),
//   C) stably partitions each node's span into its internal children's spans
//      of the next level buffer (bit 0 -> left child, 1 -> right child).
// Work is split in units of 128 symbols (4 per lane).  After the last depth the
// bitmap windows are written to the record; the partial last word of every
// window is carried to the next chunk.
#include "pivco_dev.cuh"

namespace pv {

constexpr int kEncThreads = 512;
constexpr int kEncWarps = kEncThreads / 32;
constexpr int kChunk = 16384;
constexpr int kUnit = 128;
constexpr int kBufBytes = kChunk + 4 * 256;
constexpr int kStageWords = 6144;
constexpr int kMaxUnits = kChunk / kUnit + 256;

struct EncSmem {
    uint8_t buf[2][kBufBytes];
    uint32_t stage[kStageWords];
    uint32_t hist[256];
    uint32_t cnt[256];      // symbols of node v in this chunk
    uint32_t cur[256];      // bit cursor of node v (bits already emitted)
    uint32_t pend[256];     // partial bitmap word holding bits below cur % 32
    uint32_t lvl_off[256];  // span start of node v in its level buffer
    uint32_t ustart[256];   // first unit of node v within its level
    uint32_t st_off[256];   // first staging word of node v's window
    uint32_t nwin[256];     // window words
    uint32_t body_off[256];
    uint32_t nv[256];
    uint32_t unit_pc[kMaxUnits];
    uint32_t unit_base[kMaxUnits];
    uint32_t nunits[17];
    uint32_t total_words;
    uint16_t rc[256];       // bit d = code bit at depth d
    uint16_t tree_a[17];
    int16_t child[256][2];
    uint8_t len[256];
    uint8_t depth_first[17];
    uint8_t sel[256];
};

// largest node v in [lo, hi) with key[v] <= g
__device__ inline int find_node(const uint32_t *key, int lo, int hi, uint32_t g) {
    while (hi - lo > 1) {
        const int m = (lo + hi) >> 1;
        if (key[m] <= g) lo = m; else hi = m;
    }
    return lo;
}

// Exclusive warp scan helper over n values produced by f(i); writes via out(i, prefix); returns total.
template <typename F, typename G>
__device__ inline uint32_t warp_scan_loop(int n, F f, G out) {
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

__global__ void __launch_bounds__(kEncThreads, 1) encode_kernel(const uint8_t *__restrict__ in,
                                                                const uint64_t *__restrict__ blk_off,
                                                                const BlockLayout *__restrict__ layout,
                                                                uint8_t *__restrict__ out,
                                                                const uint64_t *__restrict__ out_off,
                                                                uint64_t *__restrict__ rec_bytes,
                                                                int32_t *__restrict__ status) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    EncSmem &S = *reinterpret_cast<EncSmem *>(smem_raw);
    const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const BlockLayout &L = *reinterpret_cast<const BlockLayout *>(reinterpret_cast<const uint8_t *>(layout) +
                                                                   (size_t)b * kLayoutBytes);
    const uint64_t n = blk_off[b + 1] - blk_off[b];
    uint8_t *rec = out + out_off[b];
    const uint64_t cap = out_off[b + 1] - out_off[b];
    const uint32_t kind = L.kind;
    // ---- argument checks (uniform) ----
    int st = PIVCO_OK;
    if (L.status != 0) st = L.status;
    else if (L.n != n) st = PIVCO_ERR_INVALID_ARG;
    else if (cap < L.rec_bound) st = PIVCO_ERR_CAPACITY;
    if (st != PIVCO_OK) {
        if (t == 0) { status[b] = st; rec_bytes[b] = 0; }
        return;
    }
    const int V = L.n_int;
    // ---- header (App. D adapted): all threads ----
    if (t < 16) {
        uint8_t v = 0;
        const uint32_t rb = L.rec_bound;
        if (t < 4) v = (uint8_t)(rb >> (8 * t));
        else if (t < 8) v = (uint8_t)((uint32_t)n >> (8 * (t - 4)));
        else if (t == 8) v = (uint8_t)V;
        else if (t == 9) v = (uint8_t)(V >> 8);
        else if (t == 10) v = (uint8_t)kind;
        else if (t == 11) v = kind == 1 ? L.csym : 0;
        else v = (uint8_t)"PVC1"[t - 12];
        rec[t] = v;
    }
    if (kind != 2) {
        if (t == 0) { status[b] = PIVCO_OK; rec_bytes[b] = kHdr; }
        return;
    }
    for (int i = t; i < 128; i += kEncThreads) rec[kLensOff + i] = (uint8_t)(L.len[2 * i] | (L.len[2 * i + 1] << 4));
    for (int i = t; i < 4 * V; i += kEncThreads) rec[kNvOff + i] = (uint8_t)(L.nv[i >> 2] >> (8 * (i & 3)));
    for (int v = t; v < V; v += kEncThreads) rec[kNvOff + 4 * V + v] = L.sel[v] ? kMarkRawSel : 0;
    {
        const uint32_t pad_lo = kNvOff + 5 * V, alen_off = (pad_lo + 3) & ~3u;
        for (uint32_t i = pad_lo + t; i < alen_off; i += kEncThreads) rec[i] = 0;
        if (t == 0) {
            int k = 0;
            for (int v = 0; v < V; v++)
                if (L.sel[v]) {
                    const uint32_t raw = (L.nv[v] + 7) / 8;
                    for (int j = 0; j < 4; j++) rec[alen_off + 4 * k + j] = (uint8_t)(raw >> (8 * j));
                    k++;
                }
        }
        // tail padding after the last body
        uint32_t end = 0;
        for (int v = 0; v < V; v++) end = max(end, L.body_off[v] + (L.nv[v] + 7) / 8);
        for (uint32_t i = end + t; i < L.rec_bound; i += kEncThreads) rec[i] = 0;
    }
    // ---- per-block tables into shared memory ----
    for (int s = t; s < 256; s += kEncThreads) {
        const int l = L.len[s];
        uint32_t r = 0;
        for (int d = 0; d < l; d++) r |= ((uint32_t)(L.code[s] >> (l - 1 - d)) & 1u) << d;
        S.rc[s] = (uint16_t)r;
        S.len[s] = (uint8_t)l;
        S.cur[s] = 0;
        S.pend[s] = 0;
        S.body_off[s] = L.body_off[s];
        S.nv[s] = L.nv[s];
        S.child[s][0] = L.child[s][0];
        S.child[s][1] = L.child[s][1];
        S.sel[s] = L.sel[s];
    }
    if (t < 17) { S.tree_a[t] = L.tree_a[t]; S.depth_first[t] = L.depth_first[t]; }
    __syncthreads();
    const int maxd = L.max_depth;
    const int64_t ceff64 = ((int64_t)(kStageWords - 2 * V) * 32 / maxd) & ~(int64_t)(kUnit - 1);
    const uint32_t ceff = (uint32_t)(ceff64 < kChunk ? ceff64 : kChunk);
    const uint8_t *src = in + blk_off[b];

    for (uint64_t P = 0; P < n; P += ceff) {
        const uint32_t cc = (uint32_t)umin64(ceff, n - P);
        // ---- load chunk, histogram ----
        for (int s = t; s < 256; s += kEncThreads) { S.hist[s] = 0; S.cnt[s] = 0; }
        __syncthreads();
        for (uint32_t i = t; i < cc; i += kEncThreads) {
            const uint8_t v = src[P + i];
            S.buf[0][i] = v;
            atomicAdd(&S.hist[v], 1u);
        }
        __syncthreads();
        // ---- per-node chunk counts: every symbol adds to each node of its path ----
        for (int s = t; s < 256; s += kEncThreads) {
            const uint32_t h = S.hist[s];
            const int l = S.len[s];
            if (h && l) {
                const uint32_t code = L.code[s];
                for (int d = 0; d < l; d++) {
                    const int v = S.depth_first[d] + (int)(code >> (l - d)) - S.tree_a[d];
                    atomicAdd(&S.cnt[v], h);
                }
            }
        }
        __syncthreads();
        // ---- spans, units and staging windows (one warp per depth, one for windows) ----
        if (warp < maxd) {
            const int d = warp, f0 = S.depth_first[d], f1 = S.depth_first[d + 1];
            warp_scan_loop(f1 - f0, [&](int i) { return (S.cnt[f0 + i] + 3u) & ~3u; },
                           [&](int i, uint32_t p) { S.lvl_off[f0 + i] = p; });
            const uint32_t tot = warp_scan_loop(f1 - f0, [&](int i) { return (S.cnt[f0 + i] + kUnit - 1) / kUnit; },
                                                [&](int i, uint32_t p) { S.ustart[f0 + i] = p; });
            if (lane == 0) S.nunits[d] = tot;
        } else if (warp == kEncWarps - 1) {
            const uint32_t tot = warp_scan_loop(V, [&](int v) {
                const uint32_t w = S.cnt[v] ? ((S.cur[v] & 31u) + S.cnt[v] + 31u) >> 5 : 0u;
                S.nwin[v] = w;
                return w;
            }, [&](int v, uint32_t p) { S.st_off[v] = p; });
            if (lane == 0) S.total_words = tot;
        }
        __syncthreads();
        for (uint32_t i = t; i < S.total_words; i += kEncThreads) S.stage[i] = 0;
        __syncthreads();
        for (int v = t; v < V; v += kEncThreads)
            if (S.nwin[v]) S.stage[S.st_off[v]] = S.pend[v];
        __syncthreads();

        // ---- levels ----
        for (int d = 0; d < maxd; d++) {
            const uint8_t *bin = S.buf[d & 1];
            uint8_t *bout = S.buf[(d + 1) & 1];
            const int f0 = S.depth_first[d], f1 = S.depth_first[d + 1];
            const uint32_t nu = S.nunits[d];
            // A: bits of every unit into the node windows
            for (uint32_t g = warp; g < nu; g += kEncWarps) {
                const int v = find_node(S.ustart, f0, f1, g);
                const uint32_t k0 = (g - S.ustart[v]) * kUnit, k = k0 + 4 * lane;
                const uint32_t cntv = S.cnt[v];
                uint32_t nib = 0;
                if (k < cntv) {
                    const uint32_t w = *reinterpret_cast<const uint32_t *>(bin + S.lvl_off[v] + k);
                    const uint32_t nval = min(4u, cntv - k);
                    for (uint32_t j = 0; j < nval; j++) nib |= ((uint32_t)(S.rc[(w >> (8 * j)) & 0xFF] >> d) & 1u) << j;
                }
                uint32_t word = nib << (4 * (lane & 7));
                word |= __shfl_xor_sync(0xffffffffu, word, 1);
                word |= __shfl_xor_sync(0xffffffffu, word, 2);
                word |= __shfl_xor_sync(0xffffffffu, word, 4);
                const uint32_t pc = __popc(word);
                const uint32_t tot = __shfl_sync(0xffffffffu, pc, 0) + __shfl_sync(0xffffffffu, pc, 8) +
                                     __shfl_sync(0xffffffffu, pc, 16) + __shfl_sync(0xffffffffu, pc, 24);
                if (lane == 0) S.unit_pc[g] = tot;
                if ((lane & 7) == 0 && word) {
                    const uint32_t pos = (S.cur[v] & 31u) + k0 + 4 * lane;   // 4*lane = 32*q
                    const uint32_t wi = pos >> 5, sh = pos & 31u;
                    uint32_t *win = S.stage + S.st_off[v];
                    atomicOr(&win[wi], word << sh);
                    if (sh && (word >> (32 - sh))) atomicOr(&win[wi + 1], word >> (32 - sh));
                }
            }
            __syncthreads();
            // B: per-node exclusive scan of unit popcounts (the rank directory)
            for (int v = f0 + warp; v < f1; v += kEncWarps) {
                const uint32_t u0 = S.ustart[v], nuv = (S.cnt[v] + kUnit - 1) / kUnit;
                warp_scan_loop((int)nuv, [&](int i) { return S.unit_pc[u0 + i]; },
                               [&](int i, uint32_t p) { S.unit_base[u0 + i] = p; });
            }
            __syncthreads();
            // C: stable partition into the internal children's spans
            if (d + 1 < maxd) {
                for (uint32_t g = warp; g < nu; g += kEncWarps) {
                    const int v = find_node(S.ustart, f0, f1, g);
                    const uint32_t k0 = (g - S.ustart[v]) * kUnit, k = k0 + 4 * lane;
                    const uint32_t cntv = S.cnt[v];
                    uint32_t nib = 0, w = 0, nval = 0;
                    if (k < cntv) {
                        w = *reinterpret_cast<const uint32_t *>(bin + S.lvl_off[v] + k);
                        nval = min(4u, cntv - k);
                        for (uint32_t j = 0; j < nval; j++) nib |= ((uint32_t)(S.rc[(w >> (8 * j)) & 0xFF] >> d) & 1u) << j;
                    }
                    uint32_t word = nib << (4 * (lane & 7));
                    word |= __shfl_xor_sync(0xffffffffu, word, 1);
                    word |= __shfl_xor_sync(0xffffffffu, word, 2);
                    word |= __shfl_xor_sync(0xffffffffu, word, 4);
                    const uint32_t w0 = __shfl_sync(0xffffffffu, word, 0), w1 = __shfl_sync(0xffffffffu, word, 8),
                                   w2 = __shfl_sync(0xffffffffu, word, 16);
                    const uint32_t q = lane >> 3;
                    uint32_t r = S.unit_base[g] + (q > 0 ? __popc(w0) : 0) + (q > 1 ? __popc(w1) : 0) +
                                 (q > 2 ? __popc(w2) : 0) + __popc(word & ((1u << (4 * (lane & 7))) - 1u));
                    const int c0 = S.child[v][0], c1 = S.child[v][1];
                    for (uint32_t j = 0; j < nval; j++) {
                        const uint32_t bit = (nib >> j) & 1u;
                        const int c = bit ? c1 : c0;
                        if (c >= 0) {
                            const uint32_t idx = bit ? r : (k + j - r);
                            bout[S.lvl_off[c] + idx] = (uint8_t)(w >> (8 * j));
                        }
                        r += bit;
                    }
                }
                __syncthreads();
            }
        }
        // ---- flush windows to the record; carry partial words ----
        for (uint32_t i = t; i < S.total_words; i += kEncThreads) {
            const int v = find_node(S.st_off, 0, V, i);
            const uint32_t j = i - S.st_off[v];
            if (j >= S.nwin[v]) continue;     // (nodes with empty windows share st_off)
            const uint32_t word = S.stage[i];
            const uint32_t byte0 = 4 * ((S.cur[v] >> 5) + j), raw = (S.nv[v] + 7) / 8;
            uint8_t *dst = rec + S.body_off[v];
#pragma unroll
            for (int q = 0; q < 4; q++)
                if (byte0 + q < raw) dst[byte0 + q] = (uint8_t)(word >> (8 * q));
        }
        __syncthreads();
        for (int v = t; v < V; v += kEncThreads) {
            const uint32_t c = S.cur[v], nc = c + S.cnt[v];
            if (S.cnt[v]) S.pend[v] = (nc & 31u) ? S.stage[S.st_off[v] + ((nc >> 5) - (c >> 5))] : 0u;
            S.cur[v] = nc;
        }
        __syncthreads();
    }
    // every node must have emitted exactly n_v bits
    int bad = 0;
    for (int v = t; v < V; v += kEncThreads) bad |= S.cur[v] != S.nv[v];
    bad = __syncthreads_or(bad);
    if (t == 0) {
        status[b] = bad ? PIVCO_ERR_INVALID_ARG : PIVCO_OK;
        rec_bytes[b] = L.rec_bound;
    }
}

cudaError_t launch_encode(const uint8_t *in, const uint64_t *blk_off, int nblk, const BlockLayout *layout,
                          uint8_t *out, const uint64_t *out_off, uint64_t *rec_bytes, int32_t *status,
                          cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    const int smem = (int)sizeof(EncSmem);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    encode_kernel<<<nblk, kEncThreads, smem, st>>>(in, blk_off, layout, out, out_off, rec_bytes, status);
    return cudaGetLastError();
}

}  // namespace pv
