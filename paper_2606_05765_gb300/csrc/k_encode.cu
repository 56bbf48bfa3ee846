// Encode kernel: per-node bitmap emission by stable partition (Sec. 4, Table 11).
//
// One CTA encodes one block in root chunks.  The root reads the chunk straight
// from global memory; only depths >= 1 need level buffers, so a chunk can be
// as long as the busiest level below the root allows (for skewed data a
// whole block).  Within a chunk the symbols of depth d sit in a level buffer
// ordered by (d-bit code prefix, block position), each node owning one
// aligned span.  For every depth:
//   A) the code bit d of every symbol is computed (the node's bitmap bits in
//      block order) and ORed into a shared-memory window of the node's bitmap;
//      each 128-symbol unit's popcount is recorded,
//   B) per node, the unit popcounts are scanned (rank directory); the node's
//      ones are its right child's symbol count in this chunk, its zeros the
//      left child's,
//   C) each node's span is stably partitioned into its internal children's
//      spans (bit 0 -> left, 1 -> right): EPF / EPL / EPR / EPN of Table 11;
//      meanwhile the depth's windows are written to the record and the
//      partial last word of each window is kept for the next chunk.
// A chunk whose levels would overflow the buffers is shortened and redone
// (a redo rewrites the same leading bits, so the record stays exact).
#include "tma.cuh"

namespace pv {

constexpr int kEncThreads = 256;
constexpr int kEncWarps = kEncThreads / 32;
constexpr int kUnit = 128;
constexpr int kECap = 14336;                 // level buffer capacity (depths >= 1)
constexpr int kELvlBytes = kECap + 16;
constexpr int kEMaxRoot = 65536;             // longest chunk
constexpr int kERegion = kEMaxRoot / 32 + 32;  // staging words of one depth's windows
constexpr int kEUnits = kEMaxRoot / kUnit + 256;

struct EncSmem {
    uint8_t buf[2][kELvlBytes];  // level buffers (depth d >= 1 uses buf[d & 1])
    uint32_t stage[2][kERegion]; // bitmap windows of depth d in stage[d & 1]
    uint32_t unit_pc[kEUnits];
    uint32_t unit_base[kEUnits];
    uint32_t cnt[256];           // symbols of node v in this chunk
    uint32_t cur[256];           // bits of node v already emitted
    uint32_t pend[256];          // partial bitmap word holding bits below cur % 32
    uint32_t npend[256];         // pend after this chunk
    uint32_t span[256];
    uint32_t ustart[256];        // first unit of node v within its depth
    uint32_t st_off[256];        // first word of node v's window in its depth's region
    uint32_t nwin[256];
    uint32_t body_off[256];
    uint32_t nv[256];
    uint32_t lvl_tot[17];
    uint32_t nunits[17];
    uint32_t nwords[17];
    uint16_t rc[256];            // bit d = code bit at depth d
    int16_t child[256][2];
    uint8_t depth[256];
    uint8_t depth_first[17];
    int32_t overflow;
    uint32_t chunk;
};

__device__ inline int find_node(const uint32_t *key, int lo, int hi, uint32_t g) {
    while (hi - lo > 1) {
        const int m = (lo + hi) >> 1;
        if (key[m] <= g) lo = m; else hi = m;
    }
    return lo;
}

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

// 4 input bytes at p (any alignment, p < end) from global memory
__device__ inline uint32_t ldg4_any(const uint8_t *p, const uint8_t *end) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uint32_t *w = reinterpret_cast<const uint32_t *>(a & ~uintptr_t(3));
    const uint32_t sh = (uint32_t)(a & 3) * 8;
    const uint32_t lo = __ldg(w);
    if (!sh) return lo;
    const uint32_t hi = (reinterpret_cast<const uint8_t *>(w + 1) < end) ? __ldg(w + 1) : 0u;
    return __funnelshift_r(lo, hi, sh);
}

// one warp: spans / units / windows of the depth-d nodes for this chunk
__device__ inline void level_setup(EncSmem &S, int d) {
    const int lane = threadIdx.x & 31;
    const int f0 = S.depth_first[d], f1 = S.depth_first[d + 1];
    uint64_t carry = 0;
    uint32_t wcarry = 0;
    for (int base = f0; base < f1; base += 32) {
        const int v = base + lane;
        const uint32_t c = v < f1 ? S.cnt[v] : 0u;
        const uint32_t win = c ? ((S.cur[v] & 31u) + c + 31u) >> 5 : 0u;
        const uint64_t x = ((uint64_t)((c + kUnit - 1) / kUnit) << 32) | ((c + 3u) & ~3u);
        uint64_t inc = x;
        uint32_t winc = win;
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
            const uint32_t wy = __shfl_up_sync(0xffffffffu, winc, o);
            if (lane >= o) { inc += y; winc += wy; }
        }
        if (v < f1) {
            const uint64_t ex = carry + inc - x;
            S.span[v] = (uint32_t)ex;
            S.ustart[v] = (uint32_t)(ex >> 32);
            S.st_off[v] = wcarry + winc - win;
            S.nwin[v] = win;
        }
        carry += __shfl_sync(0xffffffffu, inc, 31);
        wcarry += __shfl_sync(0xffffffffu, winc, 31);
    }
    if (lane == 0) {
        S.nunits[d] = (uint32_t)(carry >> 32);
        S.nwords[d] = wcarry;
        if ((d > 0 && (uint32_t)carry > (uint32_t)kECap) || (carry >> 32) > (uint64_t)kEUnits || wcarry > (uint32_t)kERegion)
            S.overflow = 1;
    }
}

// zero the depth-d windows; each node's pending partial word goes first
__device__ inline void level_windows_init(EncSmem &S, int d) {
    const int f0 = S.depth_first[d], f1 = S.depth_first[d + 1];
    uint32_t *reg = S.stage[d & 1];
    for (uint32_t i = threadIdx.x; i < S.nwords[d]; i += kEncThreads) {
        const int v = find_node(S.st_off, f0, f1, i);
        reg[i] = (i == S.st_off[v]) ? S.pend[v] : 0u;
    }
}

__global__ void __launch_bounds__(kEncThreads, 3) encode_kernel(const uint8_t *__restrict__ in,
                                                                const uint64_t *__restrict__ blk_off,
                                                                const BlockLayout *__restrict__ layout,
                                                                uint8_t *__restrict__ out,
                                                                const uint64_t *__restrict__ out_off,
                                                                uint64_t *__restrict__ rec_bytes,
                                                                int32_t *__restrict__ status) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    EncSmem &S = *reinterpret_cast<EncSmem *>(smem_raw);
    const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const BlockLayout &L = *reinterpret_cast<const BlockLayout *>(reinterpret_cast<const uint8_t *>(layout) +
                                                                   (size_t)b * kLayoutBytes);
    const uint64_t n = blk_off[b + 1] - blk_off[b];
    uint8_t *rec = out + out_off[b];
    const uint64_t cap = out_off[b + 1] - out_off[b];
    const uint32_t kind = L.kind;
    int st = PIVCO_OK;
    if (L.status != 0) st = L.status;
    else if (L.n != n) st = PIVCO_ERR_INVALID_ARG;
    else if (cap < L.rec_bound) st = PIVCO_ERR_CAPACITY;
    if (st != PIVCO_OK) {
        if (t == 0) { status[b] = st; rec_bytes[b] = 0; }
        return;
    }
    const int V = L.n_int;
    // ---- record header (App. D, adapted) ----
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
    if (t < 128) rec[kLensOff + t] = (uint8_t)(L.len[2 * t] | (L.len[2 * t + 1] << 4));
    for (int i = t; i < 4 * V; i += kEncThreads) rec[kNvOff + i] = (uint8_t)(L.nv[i >> 2] >> (8 * (i & 3)));
    if (t < V) rec[kNvOff + 4 * V + t] = L.sel[t] ? kMarkRawSel : 0;
    {
        const uint32_t pad_lo = kNvOff + 5 * V, alen_off = (pad_lo + 3) & ~3u;
        if (pad_lo + t < alen_off) rec[pad_lo + t] = 0;
        if (warp == 0) {
            // the alen table: raw sizes of the selected nodes, in node order
            warp_scan_loop(V, [&](int v) { return (uint32_t)(L.sel[v] != 0); }, [&](int v, uint32_t p) {
                if (L.sel[v]) {
                    const uint32_t raw = (L.nv[v] + 7) / 8;
                    for (int j = 0; j < 4; j++) rec[alen_off + 4 * p + j] = (uint8_t)(raw >> (8 * j));
                }
            });
        }
        for (uint32_t i = L.body_end + t; i < L.rec_bound; i += kEncThreads) rec[i] = 0;
    }
    // ---- per-block tables ----
    {
        const int s = t;
        const int l = L.len[s];
        uint32_t r = 0;
        for (int d = 0; d < l; d++) r |= ((uint32_t)(L.code[s] >> (l - 1 - d)) & 1u) << d;
        S.rc[s] = (uint16_t)r;
        S.cur[s] = 0;
        S.pend[s] = 0;
        S.body_off[s] = L.body_off[s];
        S.nv[s] = L.nv[s];
        S.child[s][0] = L.child[s][0];
        S.child[s][1] = L.child[s][1];
        S.depth[s] = L.depth[s];
    }
    if (t < 17) { S.depth_first[t] = L.depth_first[t]; S.lvl_tot[t] = 0; }
    __syncthreads();
    if (t < V) {
        // per-depth symbol totals below the root (chunk sizing)
        for (int c = 0; c < 2; c++) {
            const int ch = S.child[t][c];
            if (ch >= 0) atomicAdd(&S.lvl_tot[S.depth[ch]], S.nv[ch]);
        }
    }
    __syncthreads();
    if (t == 0) {
        uint64_t mx = 1;
        for (int d = 1; d < 16; d++) mx = S.lvl_tot[d] > mx ? S.lvl_tot[d] : mx;
        uint64_t X = (uint64_t)(kECap - 4 * 256) * n / mx;
        X = X > (uint64_t)kEMaxRoot ? (uint64_t)kEMaxRoot : X;
        X = X < n ? (X & ~(uint64_t)(kUnit - 1)) : n;
        S.chunk = X < (uint64_t)kUnit ? (uint32_t)kUnit : (uint32_t)X;
    }
    __syncthreads();
    const int maxd = L.max_depth;
    const uint8_t *src = in + blk_off[b];
    const uint8_t *src_end = in + blk_off[b + 1];

    for (uint64_t P = 0; P < n;) {
        const uint32_t cc = (uint32_t)umin64(S.chunk, n - P);
        const uint8_t *in0 = src + P;
        if (t == 0) { S.cnt[0] = cc; S.overflow = 0; }
        __syncthreads();
        if (warp == 0) level_setup(S, 0);
        __syncthreads();
        level_windows_init(S, 0);
        __syncthreads();

        for (int d = 0; d < maxd; d++) {
            const uint8_t *bin = S.buf[d & 1];
            uint8_t *bout = S.buf[(d + 1) & 1];
            uint32_t *reg = S.stage[d & 1];
            const int f0 = S.depth_first[d], f1 = S.depth_first[d + 1];
            const uint32_t nu = S.nunits[d];
            // A: bits of every unit into the node windows, unit popcounts
            for (uint32_t g = warp; g < nu; g += kEncWarps) {
                const int v = find_node(S.ustart, f0, f1, g);
                const uint32_t k0 = (g - S.ustart[v]) * kUnit, k = k0 + 4 * lane;
                const uint32_t cntv = S.cnt[v];
                uint32_t nib = 0;
                if (k < cntv) {
                    const uint32_t w = d == 0 ? ldg4_any(in0 + k, src_end) : *reinterpret_cast<const uint32_t *>(bin + S.span[v] + k);
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
                    const uint32_t pos = (S.cur[v] & 31u) + k0 + 4 * lane;   // 4 * lane = 32 * word index
                    const uint32_t wi = pos >> 5, sh = pos & 31u;
                    uint32_t *win = reg + S.st_off[v];
                    atomicOr(&win[wi], word << sh);
                    if (sh && (word >> (32 - sh))) atomicOr(&win[wi + 1], word >> (32 - sh));
                }
            }
            __syncthreads();
            // B: rank directory of each node; children's counts for this chunk
            for (int v = f0 + warp; v < f1; v += kEncWarps) {
                const uint32_t cntv = S.cnt[v];
                uint32_t ones = 0;
                if (cntv) {
                    const uint32_t u0 = S.ustart[v], nuv = (cntv + kUnit - 1) / kUnit;
                    ones = warp_scan_loop((int)nuv, [&](int i) { return S.unit_pc[u0 + i]; },
                                          [&](int i, uint32_t p) { S.unit_base[u0 + i] = p; });
                }
                if (lane < 2 && S.child[v][lane] >= 0) S.cnt[S.child[v][lane]] = lane ? ones : cntv - ones;
            }
            __syncthreads();
            if (d + 1 < maxd && warp == 0) level_setup(S, d + 1);
            __syncthreads();
            if (S.overflow) break;
            // C: stable partition into the internal children's spans
            if (d + 1 < maxd) {
                for (uint32_t g = warp; g < nu; g += kEncWarps) {
                    const int v = find_node(S.ustart, f0, f1, g);
                    const int c0 = S.child[v][0], c1 = S.child[v][1];
                    if (c0 < 0 && c1 < 0) continue;   // both children are leaves: nothing moves
                    const uint32_t k0 = (g - S.ustart[v]) * kUnit, k = k0 + 4 * lane;
                    const uint32_t cntv = S.cnt[v];
                    uint32_t nib = 0, w = 0, nval = 0;
                    if (k < cntv) {
                        w = d == 0 ? ldg4_any(in0 + k, src_end) : *reinterpret_cast<const uint32_t *>(bin + S.span[v] + k);
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
                    const uint32_t sp0 = c0 >= 0 ? S.span[c0] : 0, sp1 = c1 >= 0 ? S.span[c1] : 0;
                    for (uint32_t j = 0; j < nval; j++) {
                        const uint32_t bit = (nib >> j) & 1u;
                        if (bit) { if (c1 >= 0) bout[sp1 + r] = (uint8_t)(w >> (8 * j)); }
                        else if (c0 >= 0) bout[sp0 + (k + j - r)] = (uint8_t)(w >> (8 * j));
                        r += bit;
                    }
                }
                level_windows_init(S, d + 1);
            }
            // write the depth-d windows to the record; keep the partial last words
            for (uint32_t i = t; i < S.nwords[d]; i += kEncThreads) {
                const int v = find_node(S.st_off, f0, f1, i);
                const uint32_t j = i - S.st_off[v];
                if (j >= S.nwin[v]) continue;
                const uint32_t word = reg[i];
                const uint32_t c = S.cur[v], nc = c + S.cnt[v];
                if (j == ((nc >> 5) - (c >> 5))) S.npend[v] = (nc & 31u) ? word : 0u;
                const uint32_t byte0 = 4 * ((c >> 5) + j), raw = (S.nv[v] + 7) / 8;
                uint8_t *dstp = rec + S.body_off[v] + byte0;
                if (byte0 + 4 <= raw && ((reinterpret_cast<uintptr_t>(dstp) & 3) == 0)) {
                    *reinterpret_cast<uint32_t *>(dstp) = word;
                } else {
#pragma unroll
                    for (int qb = 0; qb < 4; qb++)
                        if (byte0 + qb < raw) dstp[qb] = (uint8_t)(word >> (8 * qb));
                }
            }
            __syncthreads();
        }
        if (S.overflow) {
            // a level did not fit: shorten the chunk and redo it
            if (t == 0) S.chunk = max((uint32_t)kUnit, (S.chunk / 4 * 3) & ~(uint32_t)(kUnit - 1));
            __syncthreads();
            continue;
        }
        for (int v = t; v < V; v += kEncThreads) {
            if (S.cnt[v]) {
                const uint32_t nc = S.cur[v] + S.cnt[v];
                S.pend[v] = (nc & 31u) ? S.npend[v] : 0u;
                S.cur[v] = nc;
            }
        }
        P += cc;
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
    cudaError_t e = cudaFuncSetAttribute(encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    encode_kernel<<<nblk, kEncThreads, smem, st>>>(in, blk_off, layout, out, out_off, rec_bytes, status);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pv

namespace pv {
cudaError_t prepare_encode_kernels() {
    return cudaFuncSetAttribute(encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(EncSmem));
}
}  // namespace pv
