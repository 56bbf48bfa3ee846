// Encode kernel: per-node bitmap emission by stable partition (Sec. 4, Sec. 2.4.1).
//
// One CTA encodes one block, top-down, level by level; its warps share two
// level buffers.  The block is coded in chunks whose levels fit those
// buffers (usually a few of the planning pass's chunks, whose histograms
// give every node's symbol count in the chunk; a chunk too large for the
// buffers is cut and counted again).  A node's bitmap holds, in block order,
// the code bit of every symbol passing through it, so the chunk's bits of
// node v start at the symbols under v in the chunks before it: the cursors
// advance by each chunk's counts.  Per level, the symbols of every node are
// cut into groups of 32 (one lane each) and windows of 32 groups, which the
// warps take in rounds of eight.  A lane's 32 code bits at the node's depth
// form one bitmap word (written to the record at the node's cursor; words
// shared with a neighbour are ORed into the zeroed body), and its symbols
// are stably partitioned into the internal children's spans (EPF / EPL /
// EPR / EPN of Sec. 2.4.1) at the zeros / ones of the node before the group:
// a segmented warp scan within the window, the windows' summaries across a
// round (one barrier), a carry across rounds.  Below the root a symbol
// travels as its remaining code bits, most significant first in 16 bits, so
// a node's bit is bit 15 and the child receives the value shifted left by
// one.  A flat node (Sec. 2.2.3) takes the top D bits of each value, its
// symbol's index in the flat group, and packs them D bits per symbol.

#include "pivco_dev.cuh"

namespace pv {

constexpr int kEncThreads = 256;
constexpr int kEncWarps = kEncThreads / 32;
constexpr int kEncCtasPerSm = 3;
constexpr int kESlack = 48;                 // over-read room (symbols)
constexpr int kEWinPerLvl = 32;             // windows of a level below the root (<= kEBuf/32 + 128 groups)

struct EncWin {                             // one window of a round
    uint32_t sum;                           // ones of its last node from that node's start in the window
    uint32_t flags;                         // 1 its first node starts at its first group, 2 a node starts in it, 4 active
};

template <int kBufT, int kWinT>
struct __align__(16) EncSmemT {
    static constexpr int kBuf = kBufT;      // symbols per level buffer
    static constexpr int kWin = kWinT;      // windows of a level below the root (>= (kBuf / 32 + 256) / 32)
    uint16_t buf[2][kBufT + kESlack];       // depth d >= 1 reads buf[d & 1], writes its children to the other
                                            // (spans start on 16-byte boundaries)
    uint32_t pos[256];                      // bit address of node v's first bit of the current chunk
    uint32_t dem[256];                      // symbols of node v in the current chunk
    uint32_t ch[256];                       // children word (node-table format; ch_flat for a flat node)
    uint32_t bitsrc[256];                   // bit address of node v's bitmap in the record
    uint32_t nv[256];                       // bits of node v's body (n_v, n_v D for a flat node)
    uint16_t code16[256];                   // code of symbol s, most significant bit at bit 15 (0: absent)
    uint16_t sp[256];                       // first symbol of node v's span in its level buffer
    uint16_t gs[256];                       // first 32-symbol group of node v within its level
    uint16_t lg[16];                        // groups of each level
    uint8_t wnode[16][kWinT];               // node holding the first group of each window of a level
    EncWin win[2][kEncWarps];               // window summaries, two rounds deep
    uint8_t ci[256];                        // canonical index of symbol s (its place in (length, symbol) order)
    uint8_t nlo[256];                       // node v's leaves are canonical indices nlo[v] .. nhi1[v]
    uint8_t nhi1[256];
    uint32_t pmask[8];                      // symbols that have a code
    uint32_t hot;                           // the symbol with the shortest code (the most frequent one)
    uint32_t bad, fits;
    uint32_t lvl_max;                       // symbols of the largest level below the root (a try's layout)
    uint8_t first[17];
    uint8_t maxd;
    uint8_t pad[14];
};
// the whole-block encoder's buffers (3 CTAs per SM), and the chunk
// encoder's (2 CTAs per SM, parts of big blocks almost twice as long)
using EncSmem = EncSmemT<kEBuf, kEWinPerLvl>;
constexpr int kEBufBig = 25600;
constexpr int kEncChunkCtasPerSm = 2;
using EncSmemBig = EncSmemT<kEBufBig, 36>;
static_assert(offsetof(BlockLayout, ci) <= sizeof(EncSmem::buf[1]) && offsetof(BlockLayout, ci) % 16 == 0,
              "the staged part of the layout fits a level buffer");
static_assert(sizeof(EncSmem::buf[0]) >= 4 * (288 + 256 + 257), "a level buffer holds the counting scratch");
static_assert(kEncChunkCtasPerSm * (sizeof(EncSmemBig) + 1024) <= 228 * 1024, "chunk encoder CTAs per SM");
static_assert((kEBufBig / 32 + 256) / 32 <= 36, "window table of the chunk encoder");

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

// adds the 32 bytes x (first vl valid) to a shared histogram of 256 bins
// and 32 per-lane bins (256 + lane, one bank each) that take the block's most
// frequent symbol h (skewed data would otherwise serialize on one counter):
// one shared add per byte, no branch for a full lane; hist_fold_hot adds the
// lane bins into bin h
__device__ inline void hist_add32(uint32_t *hist, const uint32_t (&x)[8], uint32_t vl, uint32_t h) {
    const uint32_t hb = 256u + (threadIdx.x & 31);
    if (vl >= 32) {
#pragma unroll
        for (int q = 0; q < 8; q++)
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const uint32_t v = __byte_perm(x[q], 0u, 0x4440u + i);
                atomicAdd(&hist[v == h ? hb : v], 1u);
            }
    } else {
#pragma unroll
        for (int q = 0; q < 8; q++)
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const uint32_t v = __byte_perm(x[q], 0u, 0x4440u + i);
                if ((uint32_t)(4 * q + i) < vl) atomicAdd(&hist[v == h ? hb : v], 1u);
            }
    }
}
// the lane bins of hist_add32 into bin h (one warp, after the CTA's counting)
__device__ inline void hist_fold_hot(uint32_t *hist, uint32_t h) {
    const int lane = threadIdx.x & 31;
    const uint32_t c = __reduce_add_sync(0xffffffffu, hist[256 + lane]);
    if (lane == 0) hist[h] += c;
}

// Node symbol counts of a histogram h by prefix sums in canonical order: the
// leaves under a node are the contiguous canonical range nlo .. nhi1, so its
// count is a difference of two prefix sums.  One warp; hc (256) and ps (257)
// are scratch.
template <typename SM>
__device__ inline void enc_counts(const SM &S, const uint32_t *h, uint32_t *cnt, uint32_t *hc, uint32_t *ps) {
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

// Spans, groups and window nodes of level d for the current demands (one
// warp; the levels are independent).  False when the level (depth >= 1)
// does not fit a buffer or has more windows than its window-node table.
template <typename SM>
__device__ inline bool enc_layout_level(SM &S, int d) {
    constexpr int kBuf = SM::kBuf;
    const int lane = threadIdx.x & 31;
    bool fits = true;
    const int f0 = S.first[d], f1 = S.first[d + 1];
    uint64_t carry = 0;
    uint32_t raw = 0;   // this lane's nodes' symbols, rounded as spans are (capped: only sizes near a buffer matter)
    for (int base = f0; base < f1; base += 32) {
        const int v = base + lane;
        uint64_t x = 0;
        if (v < f1) {
            const uint32_t dv = S.dem[v];
            raw = min(raw + ((min(dv, 1u << 24) + 7u) & ~7u), 1u << 25);
            if (d && dv > (uint32_t)kBuf) fits = false;
            const uint32_t el = d ? ((min(dv, (uint32_t)kBuf) + 7u) & ~7u) : 0u;   // spans of whole 16-byte units
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
            S.sp[v] = (uint16_t)min((uint64_t)kBuf, ex >> 32);
            S.gs[v] = (uint16_t)ex;
        }
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (d && (carry >> 32) > (uint64_t)kBuf) fits = false;
    if ((uint32_t)carry > 0xFFFFu) fits = false;
    const uint32_t G = (uint32_t)carry & 0xFFFFu;
    const uint32_t lraw = __reduce_add_sync(0xffffffffu, raw);
    if (lane == 0) {
        S.lg[d] = (uint16_t)G;
        if (d) atomicMax(&S.lvl_max, lraw);
    }
    __syncwarp();
    if (d) {
        const uint32_t nwin = (G + 31) >> 5;
        if (nwin > (uint32_t)SM::kWin) fits = false;
        for (uint32_t i = lane; i < nwin && i < (uint32_t)SM::kWin; i += 32) {
            int lo = f0, hi = f1;
            while (hi - lo > 1) {
                const int m = (lo + hi) >> 1;
                if ((uint32_t)S.gs[m] <= 32u * i) lo = m; else hi = m;
            }
            S.wnode[d][i] = (uint8_t)lo;
        }
    }
    __syncwarp();
    return __all_sync(0xffffffffu, fits);
}

// The carry into this warp's window of the round (the ones, before the
// window, of the node that runs into it) and the carry into the next round;
// every warp calls it after the round's summaries are written.
template <typename SM>
__device__ inline uint32_t enc_round_carry(const SM &S, uint32_t par, uint32_t &rc_sum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const EncWin x = lane < kEncWarps ? S.win[par][lane] : EncWin{0u, 0u};
    uint32_t val = x.sum, seg = (x.flags >> 1) & 1u;
#pragma unroll
    for (int o = 1; o < kEncWarps; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, val, o), f = __shfl_up_sync(0xffffffffu, seg, o);
        if (lane >= o && !seg) { val += y; seg |= f; }
    }
    if (!seg) val += rc_sum;
    const uint32_t prev = __shfl_up_sync(0xffffffffu, val, 1);
    const uint32_t c = (x.flags & 1u) ? 0u : (lane ? prev : rc_sum);
    const uint32_t cin = __shfl_sync(0xffffffffu, c, warp);
    const uint32_t act = __ballot_sync(0xffffffffu, (x.flags & 4u) != 0);   // window 0 always is
    rc_sum = __shfl_sync(0xffffffffu, val, 31 - __clz(act));
    return cin;
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

// Packs the top D bits of the 16-bit values y (value j in half j & 1 of
// y[j >> 1]; the first vl valid) D bits per value, value j at bits [jD,
// jD + D) (Sec. 2.2.3 packed indices, App. D), and writes the vl D bits at
// bit address a of the record: words inside the run are stored, the two it
// shares with its neighbours are ORed into the zeroed body.
template <int D>
__device__ inline void flat_emit(uint32_t *rec32, uint32_t a, const uint32_t (&y)[16], uint32_t vl) {
    uint32_t w[D];
#pragma unroll
    for (int k = 0; k < D; k++) w[k] = 0;
#pragma unroll
    for (int j = 0; j < 32; j++) {
        const uint32_t x = (uint32_t)j < vl ? ((y[j >> 1] >> (16 * (j & 1))) & 0xFFFFu) >> (16 - D) : 0u;
        const int b = j * D, wi = b >> 5, sh = b & 31;
        w[wi] |= x << sh;
        if (sh + D > 32) w[wi + 1] |= x >> (32 - sh);
    }
    const uint32_t sh = a & 31u, wi = a >> 5, end = sh + vl * (uint32_t)D;
    uint32_t prev = 0;
#pragma unroll
    for (int k = 0; k <= D; k++) {
        const uint32_t cur = k < D ? w[k] : 0u;
        const uint32_t o = sh ? (cur << sh) | (prev >> (32 - sh)) : cur;
        prev = cur;
        const uint32_t lo = 32u * (uint32_t)k;
        if (lo < end) {
            if (lo >= sh && lo + 32u <= end) rec32[wi + k] = o;
            else if (o) atomicOr(&rec32[wi + k], o);
        }
    }
}

__device__ inline void flat_emit_d(uint32_t D, uint32_t *rec32, uint32_t a, const uint32_t (&y)[16], uint32_t vl) {
    switch (D) {
        case 2: flat_emit<2>(rec32, a, y, vl); break;
        case 3: flat_emit<3>(rec32, a, y, vl); break;
        case 4: flat_emit<4>(rec32, a, y, vl); break;
        case 5: flat_emit<5>(rec32, a, y, vl); break;
        case 6: flat_emit<6>(rec32, a, y, vl); break;
        case 7: flat_emit<7>(rec32, a, y, vl); break;
        default: flat_emit<8>(rec32, a, y, vl); break;
    }
}

// Codes plan chunks cA .. cB - 1 of block b with the whole CTA (every
// thread calls it with the same arguments).  whole: the block entire, its
// header written, its body zeroed here and its status written; else one
// chunk of a big block: the reset pass has checked the block, zeroed its
// body and set its status, the chunk starts at the node cursors the counts
// of the chunks before it give, chunk 0 writes the header and tables, and
// the status only ever turns to an error.
template <bool whole, typename SM>
__device__ inline void encode_item(int b, uint32_t cA, uint32_t cB, const uint8_t *__restrict__ in,
                                   const uint64_t *__restrict__ blk_off, const BlockLayout *__restrict__ layout,
                                   const uint32_t *__restrict__ chunk_hist, uint8_t *__restrict__ out,
                                   const uint64_t *__restrict__ out_off, uint64_t *__restrict__ rec_bytes,
                                   int32_t *__restrict__ status, SM &S) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint64_t i0 = blk_off[b], i1 = blk_off[b + 1], o0 = out_off[b], o1 = out_off[b + 1];
    const uint32_t nw = enc_nchunks(i1 - i0), cEnd = cB < nw ? cB : nw;
    // the item's input is read by the root pass: ask L2 for it now, so
    // those reads find it there
    {
        const uint64_t lo = enc_chunk_start(i1 - i0, cA, nw), hi = enc_chunk_start(i1 - i0, cEnd, nw);
        const uint8_t *p0 = in + i0 + lo;
        for (uint64_t i = 128ull * t; i < hi - lo; i += 128ull * kEncThreads)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(p0 + i));
    }
    // the block's layout, staged into shared memory once (coalesced); it
    // borrows the second level buffer, unused until the levels start
    {
        const uint4 *g = reinterpret_cast<const uint4 *>(reinterpret_cast<const uint8_t *>(layout) +
                                                          (size_t)b * kLayoutBytes);
        uint4 *d = reinterpret_cast<uint4 *>(S.buf[1]);
        constexpr int kStaged = (int)(offsetof(BlockLayout, ci) / 16), kTab = 768 / 16;
        for (int i = t; i < kStaged; i += kEncThreads) d[i] = __ldg(g + i);
        // the canonical order and the nodes' leaf ranges, straight into their tables
        if (t < kTab) reinterpret_cast<uint4 *>(S.ci)[t] = __ldg(g + kStaged + t);
    }
    __syncthreads();
    const BlockLayout &L = *reinterpret_cast<const BlockLayout *>(S.buf[1]);
    const uint64_t n = i1 - i0;
    uint8_t *rec = out + o0;
    const uint64_t cap = o1 - o0;
    const uint32_t kind = L.kind;
    int st = PIVCO_OK;
    if (L.status != 0) st = L.status;
    else if (L.n != n || (reinterpret_cast<uintptr_t>(rec) & 15)) st = PIVCO_ERR_INVALID_ARG;
    else if (cap < L.rec_bound) st = PIVCO_ERR_CAPACITY;
    if (st != PIVCO_OK || (!whole && kind != 2)) {   // (the reset pass has reported a big block's)
        if (t == 0 && whole) { status[b] = st; rec_bytes[b] = 0; }
        return;
    }
    const int V = L.n_int;
    const uint32_t rec_bound = L.rec_bound;   // the staged layout is overwritten once the levels start
    const bool head = whole || cA == 0;   // this item writes the header and tables
    // ---- record header (App. D, adapted) ----
    if (t < 16 && head) {
        uint8_t v = 0;
        const uint32_t rb = L.rec_bound;
        if (t < 4) v = (uint8_t)(rb >> (8 * t));
        else if (t < 8) v = (uint8_t)((uint32_t)n >> (8 * (t - 4)));
        else if (t == 8) v = (uint8_t)V;
        else if (t == 9) v = (uint8_t)(V >> 8);
        else if (t == 10) v = (uint8_t)kind;
        else if (t == 11) v = kind == 1 ? L.csym : 0;
        else v = t == 15 ? (L.flat ? '2' : '1') : (uint8_t)"PVC"[t - 12];
        rec[t] = v;
    }
    if (kind != 2) {
        if (t == 0) { status[b] = PIVCO_OK; rec_bytes[b] = kHdr; }
        return;
    }
    // the record start is 16-byte aligned: the length nibbles and n_v as words
    if (t < 32 && head) {
        uint32_t x = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) x |= (uint32_t)(L.len[8 * t + j] & 15u) << (4 * j);
        reinterpret_cast<uint32_t *>(rec + kLensOff)[t] = x;
    }
    if (t < V && head) reinterpret_cast<uint32_t *>(rec + kNvOff)[t] = L.nv[t];
    if (t < V && head) rec[kNvOff + 4 * V + t] = L.fd[t] ? (uint8_t)(kMarkFlat + L.fd[t]) : (L.sel[t] ? kMarkRawSel : 0);
    if (head) {
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
        if (whole)
            for (uint32_t i = L.body_end + t; i < L.rec_bound; i += kEncThreads) rec[i] = 0;
    }
    // ---- the bitmaps are ORed into a zeroed body ----
    if (whole) {
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
            S.ch[t] = L.fd[t] ? ch_flat(L.fd[t], L.fbase[t]) : code2;
            S.bitsrc[t] = 8u * L.body_off[t];
            S.pos[t] = 8u * L.body_off[t];
            S.nv[t] = L.nv[t] * max(1u, (uint32_t)L.fd[t]);
        }
        if (t < 17) S.first[t] = L.depth_first[t];
        if (t == 0) { S.maxd = L.max_depth; S.hot = 0xFFFFu; S.bad = 0; }
    }
    __syncthreads();
    {
        const uint32_t l = L.len[t];
        const uint32_t key = __reduce_min_sync(0xffffffffu, l ? (l << 8) | (uint32_t)t : 0xFFFFu);
        if (lane == 0) atomicMin(&S.hot, key);
        const uint32_t pm = __ballot_sync(0xffffffffu, l != 0);
        if (lane == 0) S.pmask[warp] = pm;
    }
    __syncthreads();   // (the staged layout is dead from here on)
    const uint32_t hot = S.hot & 0xFFu;
    const uint8_t *src = in + i0;
    const uint8_t *src_end = in + i1;
    uint32_t *rec32 = reinterpret_cast<uint32_t *>(rec);
    // counting scratch in the second level buffer (free between chunks)
    uint32_t *hist = reinterpret_cast<uint32_t *>(S.buf[1]);
    uint32_t *hc = hist + 288, *ps = hist + 544;   // (after the 32 lane bins of the counting)
    // a chunk of a big block starts every node's cursor after the symbols
    // the chunks before it put there
    if (cA > 0) {
        uint32_t h = 0;
        for (uint32_t c = 0; c < cA; c++) h += __ldg(chunk_hist + ((size_t)b * kEncChunks + c) * 256 + t);
        hist[t] = h;
        __syncthreads();
        if (warp == 0) enc_counts(S, hist, S.dem, hc, ps);
        __syncthreads();
        if (t < V) S.pos[t] += S.dem[t] * max(1u, ch_flat_d(S.ch[t]));
        __syncthreads();
    }
    // ---- chunks: runs of the planning pass's chunks, or parts of one ----
    uint32_t c0 = cA, k = cEnd - cA;    // the run of plan chunks tried: c0 .. c0 + k - 1
    uint32_t P = enc_chunk_start(n, cA, nw), sub = 0;   // sub > 0: cutting plan chunk c0 into parts of `sub` symbols
    const uint32_t Pend = enc_chunk_start(n, cEnd, nw);
    uint32_t acc = 0;              // count of symbol t in the coded parts of plan chunk c0
    while (P < Pend) {
        const uint32_t Q1 = enc_chunk_start(n, c0 + (sub ? 1u : k), nw);   // end of the run / plan chunk
        const uint32_t C = sub ? min(sub, Q1 - P) : Q1 - P;
        // the chunk's histogram: the planning pass's chunk counts, or counted here
        for (int s2 = t; s2 < 256 + 32; s2 += kEncThreads) hist[s2] = 0;
        __syncthreads();
        if (chunk_hist && !sub) {
            uint32_t h = 0;
            for (uint32_t c = c0; c < c0 + k; c++) h += __ldg(chunk_hist + ((size_t)b * kEncChunks + c) * 256 + t);
            hist[t] = h;
        } else {
            for (uint32_t kb = P + 32u * t; kb < P + C; kb += 32u * kEncThreads) {
                uint32_t x[8];
                ldg32(src + kb, src_end, x);
                hist_add32(hist, x, min(32u, P + C - kb), hot);
            }
            __syncthreads();
            if (warp == 0) hist_fold_hot(hist, hot);
        }
        __syncthreads();
        const uint32_t hcount = hist[t];
        if (warp == 0) {
            // the counts must total the chunk, with no symbol the code lacks
            uint32_t tot = 0, nocode = 0;
            for (int s2 = lane; s2 < 256; s2 += 32) {
                tot += hist[s2];
                if (hist[s2] && !((S.pmask[s2 >> 5] >> (s2 & 31)) & 1u)) nocode = 1;
            }
            tot = __reduce_add_sync(0xffffffffu, tot);
            if (__any_sync(0xffffffffu, nocode) || tot != C) { if (lane == 0) S.bad = 1; }
            else enc_counts(S, hist, S.dem, hc, ps);
            if (lane == 0) { S.fits = 1; S.lvl_max = 0; }
        }
        __syncthreads();
        if (S.bad) break;
        // no node's bits of this chunk may run past its body (counts that do
        // not describe the input could otherwise carry a cursor beyond it)
        if (t < V && (uint64_t)S.pos[t] + (uint64_t)S.dem[t] * max(1u, ch_flat_d(S.ch[t])) >
                         (uint64_t)S.bitsrc[t] + S.nv[t])
            S.bad = 1;
        __syncthreads();
        if (S.bad) break;
        for (int d = warp; d < (int)S.maxd; d += kEncWarps)
            if (!enc_layout_level(S, d) && lane == 0) S.fits = 0;
        __syncthreads();
        const bool fits = S.fits != 0;
        __syncthreads();
        if (!fits) {
            // a shorter run of plan chunks, or parts of one chunk (32 symbols
            // always fit: a level then holds at most 32 symbols in 160 groups)
            if (sub == 32u) {
                if (t == 0) S.bad = 1;
                break;
            }
            if (!sub && k > 1) {
                k = (k + 1) / 2;
            } else {
                // parts whose largest level fills at most 7/8 of a buffer,
                // scaled from this try's largest level, and at least halved
                const uint32_t cur = sub ? sub : C, lm = S.lvl_max;
                const uint32_t est = lm ? (uint32_t)((uint64_t)cur * (SM::kBuf - SM::kBuf / 8) / lm) : cur / 2;
                sub = max(32u, min(cur / 2, est) & ~31u);
            }
            continue;
        }
        // ---- the root: input bytes -> codes; bits; children ----
        uint32_t par = 0;
        if (const uint32_t rD = ch_flat_d(S.ch[0])) {
            // a flat root (the whole alphabet one group): the packed indices
            for (uint32_t kk = 32u * t; kk < C; kk += 32u * kEncThreads) {
                uint32_t x[8];
                ldg32(src + P + kk, src_end, x);
                uint32_t y[16];
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const uint32_t s0 = (x[j >> 1] >> (16 * (j & 1))) & 0xFFu, s1 = (x[j >> 1] >> (16 * (j & 1) + 8)) & 0xFFu;
                    y[j] = (uint32_t)S.code16[s0] | ((uint32_t)S.code16[s1] << 16);
                }
                flat_emit_d(rD, rec32, S.pos[0] + kk * rD, y, min(32u, C - kk));
            }
        } else {
            const uint32_t chv = S.ch[0], c0n = chv & 0xFFFFu, c1n = chv >> 16;
            const bool i0c = !(c0n & 0x8000u), i1c = !(c1n & 0x8000u);
            const uint32_t nb = smem_addr(S.buf[1]);
            const uint32_t lp0 = nb + 2u * (i0c ? S.sp[c0n & 0xFFu] : 0u), rp0 = nb + 2u * (i1c ? S.sp[c1n & 0xFFu] : 0u);
            const uint32_t G = (C + 31) >> 5;
            uint32_t rc = 0;
            // the next round's 32 bytes of each lane are loaded while this one is coded
            uint32_t xn[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (32u * (32u * warp + lane) < C) ldg32(src + P + 32u * (32u * warp + lane), src_end, xn);
            for (uint32_t r0 = 0; r0 < G; r0 += 32 * kEncWarps) {
                const uint32_t kk = 32u * (r0 + 32u * warp + lane);
                const bool act = kk < C;
                const uint32_t vl = act ? min(32u, C - kk) : 0u;
                uint32_t x[8];
#pragma unroll
                for (int q = 0; q < 8; q++) { x[q] = xn[q]; xn[q] = 0u; }
                if (kk + 32u * 32u * kEncWarps < C) ldg32(src + P + kk + 32u * 32u * kEncWarps, src_end, xn);
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
                if (lane == 31) S.win[par][warp] = EncWin{inc, 0u};
                __syncthreads();
                uint32_t cin;
                {
                    const uint32_t ws = lane < kEncWarps ? S.win[par][lane].sum : 0u;
                    uint32_t wi = ws;
#pragma unroll
                    for (int o = 1; o < kEncWarps; o <<= 1) {
                        const uint32_t yy = __shfl_up_sync(0xffffffffu, wi, o);
                        if (lane >= o) wi += yy;
                    }
                    cin = rc + __shfl_sync(0xffffffffu, wi - ws, warp);
                    rc += __shfl_sync(0xffffffffu, wi, kEncWarps - 1);
                }
                par ^= 1u;
                const uint32_t r1 = cin + inc - pc;
                enc_put_bits(rec32, act, 0u, S.pos[0] + kk, bw, vl);
                // a chunk whose symbols do not match its counts must not write past the spans
                if (act && ((i1c && r1 + pc > S.dem[c1n & 0xFFu]) || (i0c && kk + vl - r1 - pc > S.dem[c0n & 0xFFu])))
                    S.bad = 1;
                else if (act) enc_split(lp0 + 2u * (kk - r1), rp0 + 2u * r1, i0c, i1c, y, bw, vl);
            }
        }
        __syncthreads();
        // ---- depths 1.. : node spans of buf[d & 1] into the children's spans ----
        for (int d = 1; d < (int)S.maxd; d++) {
            const uint16_t *bin = S.buf[d & 1];
            uint16_t *bout = S.buf[(d + 1) & 1];
            const uint32_t f1 = S.first[d + 1], G = S.lg[d];
            const uint32_t le = 0xFFFFFFFFu >> (31 - lane);
            uint32_t rc_sum = 0;
            for (uint32_t r0 = 0; r0 < G; r0 += 32 * kEncWarps) {
                const uint32_t base = r0 + 32u * warp;
                if (base >= G) {
                    // past the level's end (its last round only): an empty
                    // summary and nothing to code
                    if (lane == 0) S.win[par][warp] = EncWin{0u, 0u};
                    __syncthreads();
                    par ^= 1u;
                    continue;
                }
                // this warp's window: the node of each group
                uint32_t v = 0, kk = 0, dv = 0, starts = 0;
                bool act = false;
                if (base < G) {
                    const uint32_t u = S.wnode[d][base >> 5];
                    const uint32_t vcur = (uint32_t)S.gs[u] == base ? u - 1 : u;
                    const uint32_t cand = vcur + 1 + lane;
                    uint32_t bit = 0;
                    if (cand < f1) {
                        const uint32_t sd = (uint32_t)S.gs[cand] - base;
                        if (sd < 32) bit = 1u << sd;
                    }
                    starts = __reduce_or_sync(0xffffffffu, bit);
                    v = vcur + __popc(starts & le);
                    const uint32_t g = base + lane;
                    kk = (g - S.gs[v]) * 32u;
                    dv = S.dem[v];
                    act = g < G && kk < dv;
                }
                const uint32_t vl = act ? min(32u, dv - kk) : 0u;
                uint32_t y[16];
                if (act) {
                    // 16-byte loads: four per lane instead of sixteen, and four
                    // times fewer shared-memory wavefronts for the same bytes
                    const uint4 *p = reinterpret_cast<const uint4 *>(bin + S.sp[v] + kk);
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const uint4 u = p[q];
                        y[4 * q] = u.x; y[4 * q + 1] = u.y; y[4 * q + 2] = u.z; y[4 * q + 3] = u.w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; j++) y[j] = 0;
                }
                const uint32_t fD = act ? ch_flat_d(S.ch[v]) : 0u;   // a flat node's lanes have no ranks
                uint32_t bw = top_bits8(y[0], y[1], y[2], y[3]) | (top_bits8(y[4], y[5], y[6], y[7]) << 8) |
                              (top_bits8(y[8], y[9], y[10], y[11]) << 16) |
                              (top_bits8(y[12], y[13], y[14], y[15]) << 24);
                if (vl < 32) bw &= (1u << vl) - 1u;
                if (fD) bw = 0;
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
                uint32_t r1 = inc - pc - (s0 > 0 ? before : 0u);
                // a level of one window (warp 0's, in the first round) takes no carry
                const bool one = G <= 32;
                if (lane == 31 && !one)
                    S.win[par][warp] = EncWin{r1 + pc, (starts & 1u) | (starts ? 2u : 0u) | (base < G ? 4u : 0u)};
                __syncthreads();
                const uint32_t cin = one ? 0u : enc_round_carry(S, par, rc_sum);
                par ^= 1u;
                if (s0 < 0) r1 += cin;   // groups of the node that runs in from the window before
                enc_put_bits(rec32, act && !fD, v, S.pos[v] + kk, bw, vl);
                if (act && fD) {
                    flat_emit_d(fD, rec32, S.pos[v] + kk * fD, y, vl);
                } else if (act) {
                    const uint32_t chv = S.ch[v], c0n = chv & 0xFFFFu, c1n = chv >> 16;
                    const bool i0c = !(c0n & 0x8000u), i1c = !(c1n & 0x8000u);
                    const uint32_t ob = smem_addr(bout);
                    const uint32_t lp = ob + 2u * ((i0c ? S.sp[c0n & 0xFFu] : 0u) + (kk - r1));
                    const uint32_t rp = ob + 2u * ((i1c ? S.sp[c1n & 0xFFu] : 0u) + r1);
                    if ((i1c && r1 + pc > S.dem[c1n & 0xFFu]) || (i0c && kk + vl - r1 - pc > S.dem[c0n & 0xFFu]))
                        S.bad = 1;
                    else
                        enc_split(lp, rp, i0c, i1c, y, bw, vl);
                }
            }
            __syncthreads();
        }
        if (t < V) S.pos[t] += S.dem[t] * max(1u, ch_flat_d(S.ch[t]));
        __syncthreads();
        if (S.bad) break;
        P += C;
        if (sub) {
            acc += hcount;
            if (P >= Q1) {
                // plan chunk done in parts: its given counts must be the ones just counted
                if (__syncthreads_or(chunk_hist && acc != __ldg(chunk_hist + ((size_t)b * kEncChunks + c0) * 256 + t))) {
                    if (t == 0) S.bad = 1;
                    break;
                }
                acc = 0;
                sub = 0;   // whole runs again
                c0 += 1;
                k = cEnd - c0;
            }
        } else {
            c0 += k;
            k = cEnd - c0;
        }
    }
    __syncthreads();
    // a chunk of a big block ends where the next one starts: the cursors
    // after the symbols of chunks 0 .. cEnd - 1
    if (cEnd < nw && !S.bad) {
        uint32_t h = 0;
        for (uint32_t c = 0; c < cEnd; c++) h += __ldg(chunk_hist + ((size_t)b * kEncChunks + c) * 256 + t);
        hist[t] = h;
        __syncthreads();
        if (warp == 0) enc_counts(S, hist, S.dem, hc, ps);
        __syncthreads();
        if (t < V) S.nv[t] = S.pos[t] == S.bitsrc[t] + S.dem[t] * max(1u, ch_flat_d(S.ch[t])) ? S.pos[t] - S.bitsrc[t]
                                                                                             : 0xFFFFFFFFu;
        __syncthreads();
    }
    if (t == 0) {
        // every node's cursor ends exactly at the end of its bitmap (of the
        // item's part of it)
        uint32_t bad = S.bad;
        for (int v = 0; v < V && !bad; v++) bad = S.pos[v] != S.bitsrc[v] + S.nv[v];
        if (whole) {
            status[b] = bad ? PIVCO_ERR_INVALID_ARG : PIVCO_OK;
            rec_bytes[b] = bad ? 0 : rec_bound;
        } else if (bad) {
            atomicExch(&status[b], PIVCO_ERR_INVALID_ARG);
            rec_bytes[b] = 0;
        }
    }
    __syncthreads();
}

// The big blocks of a chunked encode (their levels do not fit the buffers):
// checked, their bodies zeroed and their status set OK, and listed; then
// every chunk of theirs is an item of the encode kernel's work list.  One
// CTA per block.
__global__ void __launch_bounds__(kEncThreads) encode_reset_kernel(const uint64_t *__restrict__ blk_off,
                                                                   BlockLayout *__restrict__ layout,
                                                                   uint8_t *__restrict__ out,
                                                                   const uint64_t *__restrict__ out_off,
                                                                   uint64_t *__restrict__ rec_bytes,
                                                                   int32_t *__restrict__ status) {
    const int b = blockIdx.x, t = threadIdx.x;
    const BlockLayout &L = *layout_of(layout, b);
    if (!L.big || L.kind != 2) return;
    const uint64_t n = blk_off[b + 1] - blk_off[b];
    uint8_t *rec = out + out_off[b];
    const uint64_t cap = out_off[b + 1] - out_off[b];
    int st = PIVCO_OK;
    if (L.status != 0) st = L.status;
    else if (L.n != n || (reinterpret_cast<uintptr_t>(rec) & 15)) st = PIVCO_ERR_INVALID_ARG;
    else if (cap < L.rec_bound) st = PIVCO_ERR_CAPACITY;
    if (st != PIVCO_OK) {
        if (t == 0) { status[b] = st; rec_bytes[b] = 0; }
        return;
    }
    // the body and the record's tail, zeroed (the chunks OR their bits in)
    const uint32_t b0 = L.body0, b1 = L.rec_bound;
    const uint32_t h0 = min(b1, (b0 + 15u) & ~15u);
    for (uint32_t i = b0 + t; i < h0; i += kEncThreads) rec[i] = 0;
    for (uint32_t i = h0 + 16 * t; i < b1; i += 16 * kEncThreads)
        *reinterpret_cast<uint4 *>(rec + i) = make_uint4(0u, 0u, 0u, 0u);
    if (t == 0) {
        status[b] = PIVCO_OK;
        rec_bytes[b] = L.rec_bound;
        const uint32_t i = atomicAdd(&layout->list_len, 1u);
        layout_of(layout, (int)i)->list_entry = (uint32_t)b;
    }
}

// One CTA per block (a big block of a chunked encode is left to the chunk
// kernel).
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
    if (chunk_hist && layout_of(layout, (int)blockIdx.x)->big) return;
    encode_item<true, EncSmem>((int)blockIdx.x, 0, kEncChunks, in, blk_off, layout, chunk_hist, out, out_off,
                               rec_bytes, status, S);
}

// The work list of big blocks' chunks, (block, chunk) by (block, chunk):
// persistent CTAs take tickets until the list is done.
__global__ void __launch_bounds__(kEncThreads, kEncChunkCtasPerSm) encode_chunks_kernel(const uint8_t *__restrict__ in,
                                                                                   const uint64_t *__restrict__ blk_off,
                                                                                   BlockLayout *__restrict__ layout,
                                                                                   const uint32_t *__restrict__ chunk_hist,
                                                                                   uint8_t *__restrict__ out,
                                                                                   const uint64_t *__restrict__ out_off,
                                                                                   uint64_t *__restrict__ rec_bytes,
                                                                                   int32_t *__restrict__ status) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    EncSmemBig &S = *reinterpret_cast<EncSmemBig *>(smem_raw);
    __shared__ uint32_t s_tk;
    const uint32_t items = *reinterpret_cast<volatile uint32_t *>(&layout->list_len) * kEncChunks;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tk = atomicAdd(&layout->list_ticket, 1u);
        __syncthreads();
        const uint32_t tk = s_tk;
        if (tk >= items) return;
        const int bb = (int)layout_of(layout, (int)(tk / kEncChunks))->list_entry;
        const uint32_t c = tk % kEncChunks;
        if (c < enc_nchunks(blk_off[bb + 1] - blk_off[bb]))
            encode_item<false, EncSmemBig>(bb, c, c + 1, in, blk_off, layout, chunk_hist, out, out_off, rec_bytes,
                                           status, S);
    }
}

cudaError_t launch_encode(const uint8_t *in, const uint64_t *blk_off, int nblk, BlockLayout *layout,
                          const uint32_t *chunk_hist, uint8_t *out, const uint64_t *out_off, uint64_t *rec_bytes,
                          int32_t *status, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    const int smem = (int)sizeof(EncSmem);
    cudaError_t e = cudaFuncSetAttribute(encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    // the work list of big blocks: emptied, then filled by the reset pass
    e = cudaMemsetAsync(&layout->list_len, 0, 2 * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    if (chunk_hist) {
        encode_reset_kernel<<<nblk, kEncThreads, 0, st>>>(blk_off, layout, out, out_off, rec_bytes, status);
        count_launches(1);
    }
    encode_kernel<<<nblk, kEncThreads, smem, st>>>(in, blk_off, layout, chunk_hist, out, out_off, rec_bytes, status);
    count_launches(1);
    if (chunk_hist) {
        const int smem_big = (int)sizeof(EncSmemBig);
        e = cudaFuncSetAttribute(encode_chunks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_big);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        encode_chunks_kernel<<<sms * kEncChunkCtasPerSm, kEncThreads, smem_big, st>>>(in, blk_off, layout, chunk_hist,
                                                                                      out, out_off, rec_bytes, status);
        count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace pv

namespace pv {
cudaError_t prepare_encode_kernels() {
    cudaError_t e = cudaFuncSetAttribute(encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(EncSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(encode_chunks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(EncSmemBig));
    return e;
}
}  // namespace pv
