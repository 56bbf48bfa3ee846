// Encode kernel: per-node bitmap emission by stable partition (Sec. 4, Sec. 2.4.1).
//
// One CTA encodes one block; its warps split the block into contiguous
// chunks and work independently.  A node's bitmap holds, in block order, the
// code bit of every symbol passing through it, so a warp's first bit of node
// v is the number of the block's earlier symbols under v: the chunk
// histograms, prefix-summed over the warps and summed over each node's
// subtree, give every warp its start cursors.  A warp encodes its chunk in
// sub-chunks whose levels fit its buffers:
//   - the sub-chunk's histogram gives every node's symbol count (demand),
//     hence the spans of each level buffer;
//   - top-down, a lane takes 32 consecutive symbols of one node: their code
//     bits at the node's depth form one 32-bit bitmap word (written to the
//     record at the node's cursor, assembled across lanes; words shared with
//     a neighbour are ORed in), and the symbols are stably partitioned into
//     the internal children's spans (EPF / EPL / EPR / EPN of Sec. 2.4.1).
// Below the root a symbol travels as its remaining code bits, most
// significant first in 16 bits, so a node's bit is bit 15 and the child
// receives the value shifted left by one.

#include "pivco_dev.cuh"

namespace pv {

constexpr int kEncThreads = 256;
constexpr int kEncWarps = kEncThreads / 32;
constexpr int kEncCtasPerSm = 2;
constexpr int kEBufE = kEncCtasPerSm == 1 ? 5376 : 2304;   // symbols per level buffer of a warp
constexpr int kESlack = 48;                                  // over-read room (symbols)

struct __align__(16) EncWarp {
    uint16_t buf[2][kEBufE + kESlack];   // depth d >= 1 reads buf[d & 1], writes its children to the other
    uint32_t pos[256];                   // bit address of node v's next bitmap bit in the record
    uint32_t dem[256];                   // symbols of node v in the current sub-chunk
    uint32_t start[256];                 // symbols before this warp's chunk, per symbol
    uint16_t sp[256];                    // first symbol of node v's span in its level buffer
    uint16_t gs[256];                    // first 32-symbol group of node v within its level
    uint16_t lg[16];                     // groups of each level
    uint32_t bad;                        // a level held more symbols than its counts
    uint32_t pad[3];
};
static_assert(sizeof(EncWarp) % 16 == 0 && ((kEBufE + kESlack) * 2) % 16 == 0, "16-byte aligned level buffers");

struct EncSmem {
    uint16_t code16[256];    // code of symbol s, most significant bit at bit 15 (0: absent)
    uint32_t ch[256];        // children: 0x8000 | symbol for a leaf, else the node index
    uint32_t bitsrc[256];    // bit address of node v's bitmap in the record
    uint32_t htot[256];      // the block's histogram
    uint32_t pmask[8];       // symbols that have a code
    __align__(16) uint8_t ci[256];   // canonical index of symbol s (its place in (length, symbol) order)
    uint8_t nlo[256];        // node v's leaves are canonical indices nlo[v] .. nhi1[v]
    uint8_t nhi1[256];
    uint32_t nocode;         // a symbol without a code has a count
    int32_t a[17];           // d-bit prefixes under leaves of length <= d
    uint8_t first[17];       // first node of each depth
    uint8_t maxd;
    uint8_t pad[2];
    uint32_t hot;            // the symbol with the shortest code (the most frequent one)
    EncWarp w[kEncWarps];
};
static_assert(offsetof(EncSmem, w) % 16 == 0, "16-byte aligned warp areas");
static_assert(offsetof(BlockLayout, ci) <= sizeof(EncWarp::buf[1]) && offsetof(BlockLayout, ci) % 16 == 0,
              "the staged part of the layout fits a level buffer");

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

// 32 input bytes at p (any alignment; bytes at or past `end` read as 0)
__device__ inline void ldg32(const uint8_t *p, const uint8_t *end, uint32_t (&x)[8]) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    if (!(a & 15) && p + 32 <= end) {
        const uint4 u0 = __ldg(reinterpret_cast<const uint4 *>(p)), u1 = __ldg(reinterpret_cast<const uint4 *>(p) + 1);
        x[0] = u0.x; x[1] = u0.y; x[2] = u0.z; x[3] = u0.w;
        x[4] = u1.x; x[5] = u1.y; x[6] = u1.z; x[7] = u1.w;
        return;
    }
    const uint32_t *w = reinterpret_cast<const uint32_t *>(a & ~uintptr_t(3));
    const uint32_t sh = (uint32_t)(a & 3) * 8;
    const uint8_t *wend = reinterpret_cast<const uint8_t *>(w);
    uint32_t prev = wend < end ? __ldg(w) : 0u;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const uint32_t nx = (wend + 4 * (j + 1) < end) ? __ldg(w + j + 1) : 0u;
        x[j] = sh ? __funnelshift_r(prev, nx, sh) : prev;
        prev = nx;
    }
}

// adds the 32 bytes x (first vl valid) to a shared histogram.  The block's
// most frequent symbol h is counted with a 4-byte compare and added once per
// warp; only the other bytes use atomics (skewed data would otherwise
// serialize on one counter).
__device__ inline void hist_add32(uint32_t *hist, const uint32_t (&x)[8], uint32_t vl, uint32_t h) {
    const int lane = threadIdx.x & 31;
    const uint32_t h4 = h * 0x01010101u;
    uint32_t hot = 0;
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const uint32_t nb = vl > 4u * q ? min(4u, vl - 4u * q) : 0u;   // valid bytes of word q
        const uint32_t bm = nb >= 4 ? 0xFFFFFFFFu : ((1u << (8 * nb)) - 1u);
        const uint32_t m = __vcmpeq4(x[q], h4) & bm;
        hot += __popc(m) >> 3;
#pragma unroll
        for (int i = 0; i < 4; i++)
            if ((uint32_t)i < nb && !((m >> (8 * i)) & 1u)) atomicAdd(&hist[(x[q] >> (8 * i)) & 0xFFu], 1u);
    }
    hot = __reduce_add_sync(0xffffffffu, hot);
    if (lane == 0 && hot) atomicAdd(&hist[h], hot);
}

// Node symbol counts of a histogram h by prefix sums in canonical order: the
// leaves under a node are the contiguous canonical range nlo .. nhi1, so its
// count is a difference of two prefix sums.  One warp; hc (256) and ps (257)
// are scratch.
__device__ inline void enc_counts(const EncSmem &S, const uint32_t *h, uint32_t *cnt, uint32_t *hc, uint32_t *ps) {
    const int lane = threadIdx.x & 31;
    const int V = S.first[S.maxd];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int s = lane + 32 * i;
        if ((S.pmask[i] >> lane) & 1u) hc[S.ci[s]] = h[s];
    }
    __syncwarp();
    uint32_t x[8], sum = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) { x[j] = hc[8 * lane + j]; sum += x[j]; }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    uint32_t run = inc - sum;
    if (lane == 0) ps[0] = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) { run += x[j]; ps[8 * lane + j + 1] = run; }
    __syncwarp();
    for (int v = lane; v < V; v += 32) cnt[v] = ps[S.nhi1[v] + 1] - ps[S.nlo[v]];
    __syncwarp();
}

// Spans and groups of every level for the current demands; false when a
// level (depth >= 1) does not fit a buffer.
__device__ inline bool enc_layout(const EncSmem &S, EncWarp &E, uint64_t &maxlvl) {
    const int lane = threadIdx.x & 31;
    bool fits = true;
    maxlvl = 0;
    for (int d = 0; d < (int)S.maxd; d++) {
        const int f0 = S.first[d], f1 = S.first[d + 1];
        uint64_t carry = 0;
        for (int base = f0; base < f1; base += 32) {
            const int v = base + lane;
            uint64_t x = 0;
            if (v < f1) {
                const uint32_t dv = E.dem[v];
                if (d && dv > (uint32_t)kEBufE) fits = false;
                const uint32_t el = d ? ((min(dv, (uint32_t)kEBufE) + 1u) & ~1u) : 0u;
                x = ((uint64_t)el << 32) | max(1u, (dv + 31u) >> 5);
            }
            uint64_t inc = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            const uint64_t ex = carry + inc - x;
            if (v < f1) {
                E.sp[v] = (uint16_t)min((uint64_t)kEBufE, ex >> 32);
                E.gs[v] = (uint16_t)ex;
            }
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (d && (carry >> 32) > (uint64_t)kEBufE) fits = false;
        if ((uint32_t)carry > 0xFFFFu) fits = false;
        if (d && (carry >> 32) > maxlvl) maxlvl = carry >> 32;
        if (lane == 0) E.lg[d] = (uint16_t)carry;
    }
    __syncwarp();
    return __all_sync(0xffffffffu, fits);
}

// Writes bits bw (vl of them valid) of one node at bit address a of the
// record.  Lanes of the same node hold consecutive 32-bit runs; a lane
// stores the aligned word its run starts in, completed with the previous
// lane's spill; words shared with another run (or another node) are ORed.
__device__ inline void enc_put_bits(uint32_t *rec32, bool act, uint32_t v, uint32_t a, uint32_t bw, uint32_t vl) {
    const int lane = threadIdx.x & 31;
    const uint32_t sh = a & 31u, wi = a >> 5;
    const uint32_t lo = bw << sh;
    const uint32_t hi = sh ? bw >> (32 - sh) : 0u;
    const uint32_t key = act ? v : 0xFFFFFFFFu;
    const uint32_t pkey = __shfl_up_sync(0xffffffffu, key, 1), nkey = __shfl_down_sync(0xffffffffu, key, 1);
    const uint32_t phi = __shfl_up_sync(0xffffffffu, hi, 1);
    const bool prev_same = lane > 0 && act && pkey == v;
    const bool next_same = lane < 31 && act && nkey == v;
    if (!act) return;
    const uint32_t word = lo | (prev_same ? phi : 0u);
    const bool full = (sh == 0 || prev_same) && vl >= 32 - sh;
    if (full) rec32[wi] = word;
    else if (word) atomicOr(&rec32[wi], word);
    if (hi && !next_same) atomicOr(&rec32[wi + 1], hi);
}

// The top bit of each of the 8 16-bit values in x0..x3 (value j at bits j)
__device__ inline uint32_t top_bits8(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3) {
    const uint32_t h0 = __byte_perm(x0, x1, 0x7531), h1 = __byte_perm(x2, x3, 0x7531);
    const uint32_t b0 = ((h0 & 0x80808080u) * 0x00204081u) >> 28;
    const uint32_t b1 = ((h1 & 0x80808080u) * 0x00204081u) >> 28;
    return b0 | (b1 << 4);
}

__device__ inline uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ inline void sts16(uint32_t a, uint32_t v) {
    asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"((unsigned short)v) : "memory");
}

// Stable partition of up to 32 symbols (values y[j], bits in bw, vl valid)
// into the left (bit 0) and right (bit 1) spans of the next level, given as
// shared-memory byte addresses.  Only internal children keep symbols: with
// both internal every symbol is stored (one address select each); with one,
// only that side's symbols are.
__device__ inline void enc_split(uint32_t la, uint32_t ra, bool i0, bool i1, const uint32_t (&y)[16], uint32_t bw,
                                 uint32_t vl) {
    const uint32_t vm = vl >= 32 ? 0xFFFFFFFFu : ((1u << vl) - 1u);
    if (i0 && i1) {
        // the j-th symbol goes to ra + 2 ones_before(j) or la + 2 (j - ones_before(j))
        uint32_t ob = 0;
        if (vl >= 32) {
#pragma unroll
            for (int j = 0; j < 32; j++) {
                const uint32_t bit = (bw >> j) & 1u;
                const uint32_t val = (y[j >> 1] >> (16 * (j & 1))) << 1;
                sts16(bit ? ra + ob : la + (2u * j - ob), val);
                ob += 2u * bit;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 32; j++) {
                const uint32_t bit = (bw >> j) & 1u;
                const uint32_t val = (y[j >> 1] >> (16 * (j & 1))) << 1;
                if ((uint32_t)j < vl) sts16(bit ? ra + ob : la + (2u * j - ob), val);
                ob += 2u * bit;
            }
        }
    } else if (i0 || i1) {
        // one side: its symbols are the set bits of m, stored in order
        const uint32_t m = (i1 ? bw : ~bw) & vm;
        uint32_t a = i1 ? ra : la;
#pragma unroll
        for (int j = 0; j < 32; j++) {
            const uint32_t val = (y[j >> 1] >> (16 * (j & 1))) << 1;
            if ((m >> j) & 1u) sts16(a, val);
            a += 2u * ((m >> j) & 1u);
        }
    }
}

__global__ void __launch_bounds__(kEncThreads, kEncCtasPerSm) encode_kernel(const uint8_t *__restrict__ in,
                                                                            const uint64_t *__restrict__ blk_off,
                                                                            const BlockLayout *__restrict__ layout,
                                                                            const uint32_t *__restrict__ chunk_hist,
                                                                            uint8_t *__restrict__ out,
                                                                            const uint64_t *__restrict__ out_off,
                                                                            uint64_t *__restrict__ rec_bytes,
                                                                            int32_t *__restrict__ status) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    EncSmem &S = *reinterpret_cast<EncSmem *>(smem_raw);
    const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // global reads the setup needs, issued first so their latencies overlap
    const uint64_t i0 = blk_off[b], i1 = blk_off[b + 1], o0 = out_off[b], o1 = out_off[b + 1];
    uint32_t chv[8];   // this warp's chunk histogram (symbol lane + 32 i)
    if (chunk_hist) {
        const uint32_t *ch = chunk_hist + ((size_t)b * kEncChunks + warp) * 256;
#pragma unroll
        for (int i = 0; i < 8; i++) chv[i] = __ldg(ch + lane + 32 * i);
    }
    // the block's input is read by the root pass: ask L2 for it now, so
    // those reads find it there
    {
        const uint8_t *p0 = in + i0;
        const uint64_t nb = i1 - i0;
        for (uint64_t i = 128ull * t; i < nb; i += 128ull * kEncThreads)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(p0 + i));
    }
    // the block's layout, staged into shared memory once (coalesced): every
    // later read of it is a shared-memory read.  It borrows the last warp's
    // second level buffer, unused until that warp's levels start.
    {
        const uint4 *g = reinterpret_cast<const uint4 *>(reinterpret_cast<const uint8_t *>(layout) +
                                                          (size_t)b * kLayoutBytes);
        uint4 *d = reinterpret_cast<uint4 *>(S.w[kEncWarps - 1].buf[1]);
        constexpr int kStaged = (int)(offsetof(BlockLayout, ci) / 16), kTab = 768 / 16;
        for (int i = t; i < kStaged; i += kEncThreads) d[i] = __ldg(g + i);
        // the canonical order and the nodes' leaf ranges, straight into their tables
        if (t < kTab) reinterpret_cast<uint4 *>(S.ci)[t] = __ldg(g + kStaged + t);
    }
    __syncthreads();
    const BlockLayout &L = *reinterpret_cast<const BlockLayout *>(S.w[kEncWarps - 1].buf[1]);
    const uint64_t n = i1 - i0;
    uint8_t *rec = out + o0;
    const uint64_t cap = o1 - o0;
    const uint32_t kind = L.kind;
    int st = PIVCO_OK;
    if (L.status != 0) st = L.status;
    else if (L.n != n || (reinterpret_cast<uintptr_t>(rec) & 15)) st = PIVCO_ERR_INVALID_ARG;
    else if (cap < L.rec_bound) st = PIVCO_ERR_CAPACITY;
    if (st != PIVCO_OK) {
        if (t == 0) { status[b] = st; rec_bytes[b] = 0; }
        return;
    }
    const int V = L.n_int;
    const uint32_t rec_bound = L.rec_bound;   // the staged layout is overwritten once the levels start
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
    // the record start is 16-byte aligned: the length nibbles and n_v as words
    if (t < 32) {
        uint32_t x = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) x |= (uint32_t)(L.len[8 * t + j] & 15u) << (4 * j);
        reinterpret_cast<uint32_t *>(rec + kLensOff)[t] = x;
    }
    if (t < V) reinterpret_cast<uint32_t *>(rec + kNvOff)[t] = L.nv[t];
    if (t < V) rec[kNvOff + 4 * V + t] = L.sel[t] ? kMarkRawSel : 0;
    {
        const uint32_t pad_lo = kNvOff + 5 * V, alen_off = (pad_lo + 3) & ~3u;
        if (pad_lo + t < alen_off) rec[pad_lo + t] = 0;
        if (warp == 0 && L.n_sel) {
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
    // ---- the bitmaps are ORed into a zeroed body ----
    {
        const uint32_t b0 = L.body0, b1 = L.body_end;
        const uint32_t h0 = min(b1, (b0 + 15u) & ~15u), h1 = max(h0, b1 & ~15u);
        for (uint32_t i = b0 + t; i < h0; i += kEncThreads) rec[i] = 0;
        for (uint32_t i = h0 + 16 * t; i < h1; i += 16 * kEncThreads)
            *reinterpret_cast<uint4 *>(rec + i) = make_uint4(0u, 0u, 0u, 0u);
        for (uint32_t i = h1 + t; i < b1; i += kEncThreads) rec[i] = 0;
    }
    // ---- per-block tables ----
    {
        const uint32_t l = L.len[t];
        S.code16[t] = l ? (uint16_t)((uint32_t)L.code[t] << (16 - l)) : 0;
        if (t < V) {
            uint32_t code2 = 0;
            for (int c = 0; c < 2; c++) {
                const int ch = L.child[t][c];
                code2 |= (ch >= 0 ? (uint32_t)ch : (0x8000u | (uint32_t)(-ch - 1))) << (16 * c);
            }
            S.ch[t] = code2;
            S.bitsrc[t] = 8u * L.body_off[t];
        }
        if (t < 17) { S.a[t] = L.tree_a[t]; S.first[t] = L.depth_first[t]; }
        if (t == 0) { S.maxd = L.max_depth; S.hot = 0xFFFFu; S.nocode = 0; }
    }
    __syncthreads();
    {
        const uint32_t my_len = L.len[t];
        const uint32_t key = __reduce_min_sync(0xffffffffu, my_len ? (my_len << 8) | (uint32_t)t : 0xFFFFu);
        if (lane == 0) atomicMin(&S.hot, key);
        const uint32_t pm = __ballot_sync(0xffffffffu, my_len != 0);
        if (lane == 0) S.pmask[warp] = pm;
    }
    __syncthreads();
    const uint32_t hot = S.hot & 0xFFu;
    // ---- warp chunks and their histograms ----
    static_assert(kEncChunks == kEncWarps, "one warp per chunk");
    const uint32_t nw = enc_nchunks(n);
    const uint32_t Q0 = enc_chunk_start(n, warp, nw), Q1 = enc_chunk_start(n, warp + 1, nw);
    const uint8_t *src = in + i0;
    const uint8_t *src_end = in + i1;
    EncWarp &E = S.w[warp];
    if (lane == 0) E.bad = 0;
    // histograms live in the first level buffer until the levels need it
    uint32_t *hist = reinterpret_cast<uint32_t *>(E.buf[0]);
    for (int s = lane; s < 256; s += 32) hist[s] = 0;
    __syncwarp();
    if (chunk_hist) {
        // counted by the chunked histogram pass (loaded at the start)
#pragma unroll
        for (int i = 0; i < 8; i++) hist[lane + 32 * i] = chv[i];
    } else if ((uint32_t)warp < nw) {
        // two input loads in flight per lane
        for (uint32_t kb = Q0; kb < Q1; kb += 2048) {
            const uint32_t k0 = kb + 32 * lane, k1 = k0 + 1024;
            uint32_t x0[8] = {0, 0, 0, 0, 0, 0, 0, 0}, x1[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (k0 < Q1) ldg32(src + k0, src_end, x0);
            if (k1 < Q1) ldg32(src + k1, src_end, x1);
            hist_add32(hist, x0, k0 < Q1 ? min(32u, Q1 - k0) : 0u, hot);
            hist_add32(hist, x1, k1 < Q1 ? min(32u, Q1 - k1) : 0u, hot);
        }
    }
    __syncthreads();
    // exclusive prefix over the warps (each warp's start counts), block totals
    {
        uint32_t run = 0;
        for (uint32_t w = 0; w < nw; w++) {
            const uint32_t h = reinterpret_cast<const uint32_t *>(S.w[w].buf[0])[t];
            S.w[w].start[t] = run;
            run += h;
        }
        S.htot[t] = run;
        if (run && !L.len[t]) S.nocode = 1;   // a symbol the code does not have: mismatch below
    }
    __syncthreads();
    // node counts of the symbols before each chunk's end (the histograms are
    // dead: their buffers take the counts), all warps at once; the last
    // chunk's are the block's totals, checked against the layout.  A chunk's
    // start counts are the previous chunk's end counts, its demands the
    // difference.
    auto endc = [&](uint32_t w) { return reinterpret_cast<uint32_t *>(S.w[w].buf[0]); };
    if ((uint32_t)warp < nw)
        enc_counts(S, (uint32_t)warp + 1 < nw ? S.w[warp + 1].start : S.htot, endc(warp), endc(warp) + 256,
                   endc(warp) + 512);
    __syncthreads();
    {
        int bad = t < V && endc(nw - 1)[t] != L.nv[t];
        if (t == 0 && S.nocode) bad = 1;
        if (__syncthreads_or(bad)) {
            if (t == 0) { status[b] = PIVCO_ERR_INVALID_ARG; rec_bytes[b] = 0; }
            return;
        }
    }
    if ((uint32_t)warp < nw) {
        for (int v = lane; v < V; v += 32) {
            const uint32_t s0 = warp ? endc(warp - 1)[v] : 0u;
            E.pos[v] = s0 + S.bitsrc[v];
            E.dem[v] = endc(warp)[v] - s0;
        }
    }
    __syncthreads();   // the count buffers are level buffers again
    uint32_t *rec32 = reinterpret_cast<uint32_t *>(rec);
    if ((uint32_t)warp < nw) {
        // the symbols before this chunk are exactly its start: every chunk's
        // counts then total its length, so the root's bits stay in its span
        const bool start_ok = E.pos[0] == S.bitsrc[0] + Q0;
        if (!start_ok && lane == 0) E.bad = 1;
        // the whole chunk at once when its levels fit; else equal sub-chunks
        // sized from the chunk's busiest level (each with its own histogram)
        const uint32_t Q = Q1 - Q0;
        uint32_t C = Q;
        bool whole = true;
        for (uint32_t P = start_ok ? Q0 : Q1; P < Q1;) {
            C = min(C, Q1 - P);
            if (!whole) {   // (the whole chunk's demands were set above)
                for (int s = lane; s < 256; s += 32) hist[s] = 0;
                __syncwarp();
                for (uint32_t kb = P; kb < P + C; kb += 1024) {
                    const uint32_t k = kb + 32 * lane;
                    uint32_t x[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                    if (k < P + C) ldg32(src + k, src_end, x);
                    hist_add32(hist, x, k < P + C ? min(32u, P + C - k) : 0u, hot);
                }
                __syncwarp();
                enc_counts(S, hist, E.dem, hist + 256, hist + 512);
            }
            uint64_t maxlvl = 0;
            if (!enc_layout(S, E, maxlvl)) {
                if (whole && chunk_hist) {
                    // sub-chunks advance the cursors by their own counts: the
                    // given chunk counts must be this chunk's bytes' counts
                    for (int s = lane; s < 256; s += 32) hist[s] = 0;
                    __syncwarp();
                    for (uint32_t kb = Q0; kb < Q1; kb += 1024) {
                        const uint32_t k = kb + 32 * lane;
                        uint32_t x[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                        if (k < Q1) ldg32(src + k, src_end, x);
                        hist_add32(hist, x, k < Q1 ? min(32u, Q1 - k) : 0u, hot);
                    }
                    __syncwarp();
                    uint32_t diff = 0;
                    for (int s = lane; s < 256; s += 32)
                        diff |= hist[s] ^ (((uint32_t)warp + 1 < nw ? S.w[warp + 1].start[s] : S.htot[s]) - E.start[s]);
                    if (__any_sync(0xffffffffu, diff != 0)) {
                        if (lane == 0) E.bad = 1;
                        break;
                    }
                }
                uint32_t nc = C / 2;
                if (whole) {
                    const uint64_t room = kEBufE - 2 * 128;
                    const uint32_t ns = (uint32_t)min((uint64_t)Q, (maxlvl * 9 / 8 + room - 1) / room);
                    nc = (Q + ns - 1) / max(ns, 1u);
                }
                whole = false;
                C = max(32u, (min(nc, C / 2 + 32)) & ~31u);
                continue;
            }
            // ---- the root: input bytes -> codes; bits; children ----
            {
                const uint32_t chv = S.ch[0], c0 = chv & 0xFFFFu, c1 = chv >> 16;
                const bool i0 = !(c0 & 0x8000u), i1 = !(c1 & 0x8000u);
                const uint32_t nb = smem_addr(E.buf[1]);
                const uint32_t lp0 = nb + 2u * (i0 ? E.sp[c0 & 0xFFu] : 0u), rp0 = nb + 2u * (i1 ? E.sp[c1 & 0xFFu] : 0u);
                uint32_t carry = 0;
                // the next window's 32 bytes are loaded while this one is coded
                uint32_t xn[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                if (32u * lane < C) ldg32(src + P + 32u * lane, src_end, xn);
                for (uint32_t kb = 0; kb < C; kb += 1024) {
                    const uint32_t kk = kb + 32u * lane;
                    const bool act = kk < C;
                    const uint32_t vl = act ? min(32u, C - kk) : 0u;
                    uint32_t x[8];
#pragma unroll
                    for (int q = 0; q < 8; q++) { x[q] = xn[q]; xn[q] = 0u; }
                    if (kk + 1024 < C) ldg32(src + P + kk + 1024, src_end, xn);
                    uint32_t y[16];
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        const uint32_t s0 = (x[j >> 1] >> (16 * (j & 1))) & 0xFFu, s1 = (x[j >> 1] >> (16 * (j & 1) + 8)) & 0xFFu;
                        y[j] = (uint32_t)S.code16[s0] | ((uint32_t)S.code16[s1] << 16);
                    }
                    uint32_t bw = top_bits8(y[0], y[1], y[2], y[3]) | (top_bits8(y[4], y[5], y[6], y[7]) << 8) |
                                  (top_bits8(y[8], y[9], y[10], y[11]) << 16) |
                                  (top_bits8(y[12], y[13], y[14], y[15]) << 24);
                    if (vl < 32) bw &= (1u << vl) - 1u;
                    const uint32_t pc = __popc(bw);
                    uint32_t inc = pc;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t yy = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += yy;
                    }
                    const uint32_t r1 = carry + inc - pc;
                    carry += __shfl_sync(0xffffffffu, inc, 31);
                    enc_put_bits(rec32, act, 0u, E.pos[0] + kk, bw, vl);
                    // a chunk whose symbols do not match its counts must not write past the spans
                    if (act && ((i1 && r1 + pc > E.dem[c1 & 0xFFu]) || (i0 && kk + vl - r1 - pc > E.dem[c0 & 0xFFu])))
                        E.bad = 1;
                    else if (act) enc_split(lp0 + 2u * (kk - r1), rp0 + 2u * r1, i0, i1, y, bw, vl);
                }
            }
            __syncwarp();
            // ---- depths 1.. : node spans of buf[d & 1] into the children's spans ----
            for (int d = 1; d < (int)S.maxd; d++) {
                const uint16_t *bin = E.buf[d & 1];
                uint16_t *bout = E.buf[(d + 1) & 1];
                const uint32_t f0 = S.first[d], f1 = S.first[d + 1], G = E.lg[d];
                const uint32_t le = 0xFFFFFFFFu >> (31 - lane);
                uint32_t vcur = f0, carry = 0;
                for (uint32_t base = 0; base < G; base += 32) {
                    const uint32_t cand = vcur + 1 + lane;
                    uint32_t bit = 0;
                    if (cand < f1) {
                        const uint32_t s = (uint32_t)E.gs[cand] - base;
                        if (s < 32) bit = 1u << s;
                    }
                    const uint32_t starts = __reduce_or_sync(0xffffffffu, bit);
                    const uint32_t v = vcur + __popc(starts & le);
                    const uint32_t g = base + lane;
                    const uint32_t kk = (g - E.gs[v]) * 32u;
                    const uint32_t dv = E.dem[v];
                    const bool act = g < G && kk < dv;
                    const uint32_t vl = act ? min(32u, dv - kk) : 0u;
                    uint32_t y[16];
                    if (act) {
                        const uint32_t *p = reinterpret_cast<const uint32_t *>(bin + E.sp[v] + kk);
#pragma unroll
                        for (int q = 0; q < 16; q++) y[q] = p[q];
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; j++) y[j] = 0;
                    }
                    uint32_t bw = top_bits8(y[0], y[1], y[2], y[3]) | (top_bits8(y[4], y[5], y[6], y[7]) << 8) |
                                  (top_bits8(y[8], y[9], y[10], y[11]) << 16) |
                                  (top_bits8(y[12], y[13], y[14], y[15]) << 24);
                    if (vl < 32) bw &= (1u << vl) - 1u;
                    const uint32_t pc = __popc(bw);
                    uint32_t inc = pc;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t yy = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += yy;
                    }
                    const uint32_t sl = starts & le;
                    const int s0 = sl ? 31 - __clz(sl) : -1;
                    const uint32_t before = __shfl_sync(0xffffffffu, inc, s0 > 0 ? s0 - 1 : 0);
                    const uint32_t r1 = inc - pc - (s0 > 0 ? before : 0u) + (s0 < 0 ? carry : 0u);
                    carry = __shfl_sync(0xffffffffu, r1 + pc, 31);
                    vcur = __shfl_sync(0xffffffffu, v, 31);
                    enc_put_bits(rec32, act, v, E.pos[v] + kk, bw, vl);
                    if (act) {
                        const uint32_t chv = S.ch[v], c0 = chv & 0xFFFFu, c1 = chv >> 16;
                        const bool i0 = !(c0 & 0x8000u), i1 = !(c1 & 0x8000u);
                        const uint32_t ob = smem_addr(bout);
                        const uint32_t lp = ob + 2u * ((i0 ? E.sp[c0 & 0xFFu] : 0u) + (kk - r1));
                        const uint32_t rp = ob + 2u * ((i1 ? E.sp[c1 & 0xFFu] : 0u) + r1);
                        if ((i1 && r1 + pc > E.dem[c1 & 0xFFu]) || (i0 && kk + vl - r1 - pc > E.dem[c0 & 0xFFu]))
                            E.bad = 1;
                        else
                            enc_split(lp, rp, i0, i1, y, bw, vl);
                    }
                }
                __syncwarp();
            }
            for (int v = lane; v < V; v += 32) E.pos[v] += E.dem[v];
            __syncwarp();
            P += C;
        }
    }
    __syncthreads();
    if (t == 0) {
        uint32_t bad = 0;
        for (int w = 0; w < kEncWarps; w++) bad |= S.w[w].bad;
        status[b] = bad ? PIVCO_ERR_INVALID_ARG : PIVCO_OK;
        rec_bytes[b] = bad ? 0 : rec_bound;
    }
}

cudaError_t launch_encode(const uint8_t *in, const uint64_t *blk_off, int nblk, const BlockLayout *layout,
                          const uint32_t *chunk_hist, uint8_t *out, const uint64_t *out_off, uint64_t *rec_bytes,
                          int32_t *status, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    const int smem = (int)sizeof(EncSmem);
    cudaError_t e = cudaFuncSetAttribute(encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    encode_kernel<<<nblk, kEncThreads, smem, st>>>(in, blk_off, layout, chunk_hist, out, out_off, rec_bytes, status);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pv

namespace pv {
cudaError_t prepare_encode_kernels() {
    return cudaFuncSetAttribute(encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(EncSmem));
}
}  // namespace pv
