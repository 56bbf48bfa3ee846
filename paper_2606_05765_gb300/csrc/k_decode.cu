// Decode side: plan, ANS pass, rank directories and the bottom-up merge
// (Sec. 3; Sec. 5.2 for ANS-coded bitmaps).
//
//   plan       one warp per record: validates the header and body layout,
//              sizes the ANS scratch, builds the block's node table (bitmap
//              source and children of every internal node, from the
//              canonical or the regrouped tree of the code lengths) and
//              splits the block into root tiles whose levels fit a CTA's
//              level buffers; per-block offsets come from two single-pass
//              scans with decoupled look-back.
//   ans        one warp per 16 KiB ANS segment: decodes the bitmap bytes into
//              the workspace scratch.
//   directory  for blocks with several tiles: per-node rank directories
//              (exclusive popcount per superblock) and, from them, every
//              node's bitmap cursor at every tile boundary (the root cursor is
//              the position; a child's cursor is the parent's rank0 / rank1).
//   tiles      one CTA per tile, independent of the other tiles.  With both
//              boundary cursors known, every node's bit range in the tile is
//              known.  Bottom-up, level by level, every node rebuilds its
//              symbol sequence
//                  out_v[k] = bit ? R[rank1(k)] : L[k - rank1(k)]
//              from its children's sequences or leaf constants (the MVV /
//              MCV / MVC / MCC cases of Sec. 3.2), a flat node from its
//              packed indices.  A lane takes one 32-bit bitmap word (32
//              symbols) of one node; ranks come from a segmented warp scan of
//              the words' popcounts and the windows' summaries; 4 output
//              symbols are one byte permute of a left and a right 4-byte
//              window.  The root writes the output.  A tile whose levels do
//              not fit is decoded in shorter chunks whose bit ranges are
//              found top-down from popcounts.
#include "ans_dev.cuh"
#include "lookback.cuh"

namespace pv {

constexpr int kDecThreads = 256;
constexpr int kDecWarps = kDecThreads / 32;
constexpr int kLvlBuf = 24576;               // one level buffer of a tile (bytes)
constexpr int kWSlack = 64;                  // over-read room of the byte windows
constexpr int kTileCtas = 4;                 // tile CTAs per SM the kernels are built for
constexpr uint32_t kNtabHdr = 32;            // node table header (see plan_block)

// bytes of a block's node table: header, then per node u32 bitmap source,
// u32 children and u32 first rank-directory entry, then the block's 256
// symbols in (length, symbol) order (the tables of its flat nodes)
__host__ __device__ inline uint32_t ntab_bytes(uint32_t V) { return (kNtabHdr + 12u * V + 256u + 15u) & ~15u; }

// rank-directory granularity, and whether every coded block gets a directory
// (random access) rather than only those split into several tiles: header
// word 7, the flag in bit 31
__device__ inline uint32_t dec_dir_bits(const uint8_t *ws) { return reinterpret_cast<const uint32_t *>(ws)[7] & 0xFFFFu; }
__device__ inline bool dec_all_dirs(const uint8_t *ws) { return (reinterpret_cast<const uint32_t *>(ws)[7] >> 31) != 0; }

__host__ __device__ inline uint32_t scratch_stride(uint32_t raw) { return ((raw + 15u) & ~15u) + 16u; }

template <typename F, typename G>
__device__ inline uint32_t warp_scan_loop_d(int n, F f, G out) {
    const int lane = threadIdx.x & 31;
    if (n <= 256) {
        // lane l takes items 8l .. 8l + 7: one warp scan of the lanes' sums
        uint32_t x[8], sum = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int i = 8 * lane + j;
            x[j] = i < n ? f(i) : 0u;
            sum += x[j];
        }
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        uint32_t run = inc - sum;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int i = 8 * lane + j;
            if (i < n) out(i, run);
            run += x[j];
        }
        return __shfl_sync(0xffffffffu, inc, 31);
    }
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

__device__ inline int find_node_d(const uint32_t *key, int lo, int hi, uint32_t g) {
    while (hi - lo > 1) {
        const int m = (lo + hi) >> 1;
        if (key[m] <= g) lo = m; else hi = m;
    }
    return lo;
}

// largest b in [0, n) with key[b] <= g (key non-decreasing, key[0] = 0)
__device__ inline int find_block(const uint32_t *key, int n, uint32_t g) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int m = (lo + hi) >> 1;
        if (key[m] <= g) lo = m; else hi = m;
    }
    return lo;
}

// The same search by a whole warp (all lanes, same arguments): 32 probes per
// step, the first around `guess` (where g would sit if the items were spread
// evenly), then 32-way splits of what is left.  key[0] <= g.
__device__ inline int find_block_warp(const uint32_t *key, int n, uint32_t g, int guess) {
    const int lane = threadIdx.x & 31;
    int lo = 0, hi = n;   // the answer is in [lo, hi); key[lo] <= g
    {
        const int s = max(0, min(guess - 15, n - 32));
        const int b = s + lane;
        const uint32_t m = __ballot_sync(0xffffffffu, b < n && key[b] <= g);   // a prefix of the lanes
        const int c = __popc(m), nv = min(32, n - s);
        if (c > 0) lo = s + c - 1;
        if (c < nv) hi = s + c;
    }
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) >> 5;
        const int b = lo + lane * step;
        const uint32_t m = __ballot_sync(0xffffffffu, lane == 0 || (b < hi && key[b] <= g));
        const int c = __popc(m);
        lo += (c - 1) * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Warp-level record parse (plan and ANS passes)
// ---------------------------------------------------------------------------
// bytes of a record staged in shared memory by the parse: the header, the
// length nibbles, n_v, the markers and the alen table of any record
constexpr uint32_t kStage = 2448;
static_assert(kStage >= kNvOff + 5 * 255 + 3 + 4 * 255 && kStage % 16 == 0, "the stage holds a record's tables");
static_assert(kStage >= 2 * kAnsWordWin, "the stage holds the ANS decoder's word window");

struct __align__(16) WarpRec {
    uint8_t stg[kStage];     // the record's first kStage bytes (zeros past its end); after the
                             // parse, the ANS decoder's word window
    uint32_t nv[256];
    uint32_t body_off[256];
    uint32_t alen[256];
    uint32_t soff[256];      // scratch offset of an ANS node within its block
    uint32_t segbase[256];   // first ANS segment of the node within its block
    uint8_t marker[256];
    uint32_t V, n, kind, rb, scratch_bytes, nsegs, flat;
};

__device__ inline bool warp_parse(const uint8_t *grec, uint64_t avail, WarpRec &R) {
    const int lane = threadIdx.x & 31;
    // one coalesced pass stages the tables; everything below reads shared memory
    {
        const uint32_t ns = (uint32_t)(avail < kStage ? avail : kStage);
        if (!(reinterpret_cast<uintptr_t>(grec) & 15)) {
#pragma unroll
            for (uint32_t i = 16 * lane; i < kStage; i += 512) {
                if (i + 16 <= ns) {
                    *reinterpret_cast<uint4 *>(R.stg + i) = __ldg(reinterpret_cast<const uint4 *>(grec + i));
                } else {
                    for (uint32_t j = i; j < i + 16; j++) R.stg[j] = j < ns ? grec[j] : 0;
                }
            }
        } else {
            for (uint32_t i = lane; i < kStage; i += 32) R.stg[i] = i < ns ? grec[i] : 0;
        }
        __syncwarp();
    }
    const uint8_t *rec = R.stg;
    bool ok = avail >= kHdr;
    uint32_t rb = 0, n = 0, V = 0, kind = 0;
    if (ok) {
        rb = ld_le32(rec);
        n = ld_le32(rec + 4);
        V = (uint32_t)rec[8] | ((uint32_t)rec[9] << 8);
        kind = rec[10];
        ok = rec[12] == 'P' && rec[13] == 'V' && rec[14] == 'C' && (rec[15] == '1' || rec[15] == '2') && rb >= kHdr &&
             !(rb & 15u) && rb <= avail;
    }
    const uint32_t flat = ok && rec[15] == '2';
    if (lane == 0) { R.rb = rb; R.n = n; R.kind = kind; R.scratch_bytes = 0; R.nsegs = 0; R.V = 0; R.flat = flat; }
    if (!ok) return false;
    if (kind != 2) {
        const uint32_t aux = rec[11];
        if (kind == 0) return n == 0 && V == 0 && aux == 0 && rb == kHdr;
        return kind == 1 && n != 0 && V == 0 && rb == kHdr;
    }
    if (V < 1 || V > 255 || n == 0 || rec[11] != 0 || rb < kNvOff + 5 * V) return false;
    if (lane == 0) R.V = V;
    const int Vi = (int)V;
    for (int v = lane; v < Vi; v += 32) {
        R.nv[v] = ld_le32(rec + kNvOff + 4 * v);
        const uint8_t m = rec[kNvOff + 4 * V + v];
        R.marker[v] = m;
        // flat markers (0xF0 + D) only in records of the regrouped tree
        if (mark_flat_d(m) ? !flat : (m && m != kMarkRawSel && ((m & 0x7F) < 1 || (m & 0x7F) > 50))) ok = false;
    }
    __syncwarp();
    const uint32_t alen_off = (kNvOff + 5 * V + 3) & ~3u;
    const uint32_t nsel = warp_scan_loop_d(Vi, [&](int v) { return (uint32_t)mark_listed(R.marker[v]); },
                                           [&](int v, uint32_t p) { R.segbase[v] = p; });
    if (alen_off + 4 * nsel > rb) ok = false;
    __syncwarp();
    if (__any_sync(0xffffffffu, !ok)) return false;
    for (int v = lane; v < Vi; v += 32) {
        // raw body bytes: ceil(n_v / 8), ceil(n_v D / 8) for a flat node
        const uint32_t fd = mark_flat_d(R.marker[v]);
        const uint32_t raw = (uint32_t)(((uint64_t)R.nv[v] * (fd ? fd : 1u) + 7) / 8);
        const uint32_t al = mark_listed(R.marker[v]) ? ld_le32(rec + alen_off + 4 * R.segbase[v]) : raw;
        R.alen[v] = al;
        if (R.marker[v] == kMarkRawSel && al != raw) ok = false;
        if (fd && (uint64_t)R.nv[v] * fd > 0xFFFFFFFFull) ok = false;
    }
    __syncwarp();
    const uint32_t base1 = alen_off + 4 * nsel;
    const uint32_t raw_tot = warp_scan_loop_d(Vi, [&](int v) { return mark_listed(R.marker[v]) ? 0u : R.alen[v]; },
                                              [&](int v, uint32_t p) { if (!mark_listed(R.marker[v])) R.body_off[v] = base1 + p; });
    const uint32_t base2 = base1 + raw_tot;
    uint64_t sel_tot = 0;
    {
        // 64-bit: corrupt alen values could wrap 32 bits
        uint64_t carry = 0;
        for (int base = 0; base < Vi; base += 32) {
            const int v = base + lane;
            const uint64_t x = (v < Vi && mark_listed(R.marker[v])) ? R.alen[v] : 0;
            uint64_t inc = x;
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (v < Vi && mark_listed(R.marker[v])) R.body_off[v] = (uint32_t)(base2 + carry + inc - x);
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        sel_tot = carry;
    }
    if ((((uint64_t)base2 + sel_tot + 15) & ~15ull) != rb) ok = false;
    const uint32_t stot = warp_scan_loop_d(Vi, [&](int v) {
        return mark_ans(R.marker[v]) ? scratch_stride((R.nv[v] + 7) / 8) : 0u;
    }, [&](int v, uint32_t p) { R.soff[v] = p; });
    const uint32_t segs = warp_scan_loop_d(Vi, [&](int v) {
        return mark_ans(R.marker[v]) ? ans_seg_count((R.nv[v] + 7) / 8) : 0u;
    }, [&](int v, uint32_t p) { R.segbase[v] = p; });
    for (int v = lane; v < Vi; v += 32)   // every symbol under a node occurs at least once
        if (R.nv[v] < (2u << (mark_flat_d(R.marker[v]) ? mark_flat_d(R.marker[v]) - 1 : 0)) || R.nv[v] > n) ok = false;
    if (lane == 0 && R.nv[0] != n) ok = false;
    if (lane == 0) { R.scratch_bytes = stot; R.nsegs = segs; }
    __syncwarp();
    return __all_sync(0xffffffffu, ok);
}

// ---------------------------------------------------------------------------
// Plan: one warp per record (ticket order), two look-back chains over blocks
//   A: (ANS scratch bytes << 22) | ANS segments
//   B: (node table + directory + cursor bytes << 22) | tiles
// Tuning (from the workspace header): the longest tile and the rank
// directory granularity; neither changes the decoded bytes.
//
// Node table of a coded block (start of its directory region):
//    0 u8 first[17]   first node of each depth (breadth-first node order)
//   17 u8 maxd        depth of the deepest leaf
//   20 u32 ent        rank-directory entries (blocks with several tiles)
//   24 u32 T          root symbols per tile
//   32 u32 src[V]     bit address of node v's bitmap: 8 x record byte offset,
//                     or 8 x block scratch offset | 2^31 for ANS-coded nodes
//      u32 ch[V]      children: child c in bits [16c, 16c + 16), 0x8000 |
//                     symbol for a leaf, else the child's node index; a
//                     flat node's word is ch_flat(D, base)
//      u32 u[V]       node v's first rank-directory entry (blocks with one)
//      u8 sym[256]    the symbols in (length, symbol) order: flat node
//                     symbol x is sym[base + x]
// ---------------------------------------------------------------------------
struct PlanScratch {
    uint32_t cntl[16], lvl[16], run[16];
    int32_t a[17], first[18], start[17];
    int32_t good, maxd, K;
    uint32_t ch[256];
    uint32_t u[256];
    uint8_t sorted[256];
    FlatTree F;
};

__device__ inline void plan_block(int b, const uint8_t *__restrict__ comp, const uint64_t *__restrict__ comp_off,
                                  int nblk, uint8_t *__restrict__ ws, uint64_t ws_bytes, int32_t *__restrict__ status,
                                  WarpRec &R, PlanScratch &Q) {
    const int lane = threadIdx.x & 31;
    uint32_t *hdr32 = reinterpret_cast<uint32_t *>(ws);
    uint64_t *hdr64 = reinterpret_cast<uint64_t *>(ws);
    const DecWs W = dec_ws(ws, nblk);
    const uint32_t dir_bits = dec_dir_bits(ws), tile_max = hdr32[8];
    const bool all_dirs = dec_all_dirs(ws);
    if (lane < 16) { Q.cntl[lane] = 0; Q.lvl[lane] = 0; Q.run[lane] = 0; }
    __syncwarp();
    const uint8_t *rec = comp + comp_off[b];
    // a record starts on a 16-byte boundary (its words are read as words)
    const bool misal = (reinterpret_cast<uintptr_t>(rec) & 15) != 0;
    bool ok = warp_parse(rec, comp_off[b + 1] - comp_off[b], R) && !misal;
    __syncwarp();
    uint32_t ntile = 1, T = ok ? R.n : 0, ent = 0;
    uint64_t dir_bytes = 0;
    const bool coded = ok && R.kind == 2;
    if (coded) {
        // canonical tree of the code lengths: a[d] prefixes of depth d are
        // leaves or under leaves, the others are internal nodes (Sec. 1.1)
        const uint32_t x = ld_le32(R.stg + kLensOff + 4 * lane);
        for (int j = 0; j < 8; j++) {
            const uint32_t l = (x >> (4 * j)) & 15u;
            if (l) atomicAdd(&Q.cntl[l], 1u);
        }
        __syncwarp();
        if (lane == 0) {
            int64_t a = 0;
            int32_t f = 0, base = 0, K = 0, m = 0;
            bool good = true;
            Q.start[0] = 0;
            for (int l = 1; l < 16; l++) { Q.start[l] = base; base += (int32_t)Q.cntl[l]; if (Q.cntl[l]) m = l; }
            K = base;
            for (int d = 0; d <= 16; d++) {
                if (d > 0) a = 2 * a + (d < 16 ? Q.cntl[d] : 0);
                Q.a[d] = (int32_t)a;
                const int64_t open = (int64_t(1) << d) - a;
                if (open < 0) good = false;
                Q.first[d] = f;
                if (d < m) {
                    if (open <= 0) good = false;
                    else f += (int32_t)open;
                } else if (d == m && open != 0) {
                    good = false;   // Kraft equality: the tree is full
                }
            }
            Q.first[17] = f;
            // (a regrouped tree has its own node count, checked below)
            Q.good = good && K >= 2 && f == K - 1 && (R.flat || f == (int32_t)R.V);
            Q.maxd = m;
            Q.K = K;
        }
        __syncwarp();
        const bool good = Q.good != 0;
        // symbols in canonical order (length, then value): rounds of 32 symbols
        for (int j = 0; j < 8; j++) {
            const int sym = 32 * j + lane;
            const uint32_t l = (R.stg[kLensOff + (sym >> 1)] >> (4 * (sym & 1))) & 15u;
            const uint32_t peers = __match_any_sync(0xffffffffu, l);
            const uint32_t r = __popc(peers & ((1u << lane) - 1u));
            if (l && good) Q.sorted[Q.start[l] + Q.run[l] + r] = (uint8_t)sym;
            __syncwarp();
            if (l && r == 0) Q.run[l] += __popc(peers);
            __syncwarp();
        }
        // children of every node and the symbols of each depth
        bool okn = good;
        if (R.flat && good) {
            // the regrouped tree with flat subtrees (Sec. 2.2.3-2.2.4); its
            // flat nodes must be the record's (markers 0xF0 + D)
            flat_tree_build(reinterpret_cast<const int32_t *>(Q.cntl), Q.start, Q.sorted, Q.F);
            okn = Q.F.ok && Q.F.n_nodes == (int32_t)R.V;
            if (okn && lane < 18) Q.first[lane] = lane < Q.F.maxd ? Q.F.first[lane] : Q.F.n_nodes;
            if (okn && lane == 0) Q.maxd = Q.F.maxd;
            for (int v = lane; v < (int)R.V && okn; v += 32) {
                int d = 0;
                uint32_t chv = 0;
                if (!flat_node(Q.F, Q.sorted, v, d, chv)) okn = false;
                const uint32_t D = ch_flat_d(chv);
                if (D != mark_flat_d(R.marker[v]) || (D && (chv & 0xFFu) + (1u << D) > (uint32_t)Q.K)) okn = false;
                if (d >= 1) atomicAdd(&Q.lvl[d], R.nv[v]);
                Q.ch[v] = chv;
            }
        } else {
        int d = 0;   // depth of node v (v grows, so the search goes on from the last one)
        for (int v = lane; v < (int)R.V && good; v += 32) {
            while (d < 15 && Q.first[d + 1] <= v) d++;
            if (d >= 1) atomicAdd(&Q.lvl[d], R.nv[v]);
            const int32_t p = Q.a[d] + (v - Q.first[d]);
            uint32_t code2 = 0;
            for (int c = 0; c < 2; c++) {
                const int32_t cp = 2 * p + c;
                uint32_t code = 0;
                if (cp < Q.a[d + 1]) {             // a leaf of length d + 1
                    const int32_t i = cp - 2 * Q.a[d];
                    if (d + 1 > 15 || i < 0 || i >= (int32_t)Q.cntl[d + 1]) okn = false;
                    else code = 0x8000u | Q.sorted[Q.start[d + 1] + i];
                } else {
                    const int32_t node = Q.first[d + 1] + (cp - Q.a[d + 1]);
                    if (node <= v || node >= (int32_t)R.V) okn = false;
                    else code = (uint32_t)node;
                }
                code2 |= code << (16 * c);
            }
            Q.ch[v] = code2;
        }
        }
        __syncwarp();
        ok = __all_sync(0xffffffffu, okn);
        if (ok) {
            // root symbols per tile: every level of a tile must fit one level
            // buffer (with 4-byte rounding per node), with 20 % headroom
            uint64_t tfit = ~0ull;
            for (int d = 1; d < 16; d++) {
                if (!Q.lvl[d]) continue;
                const uint32_t nodes = (uint32_t)(Q.first[d + 1] - Q.first[d]);
                const uint64_t room = (uint64_t)kLvlBuf > 4ull * nodes + 32 ? kLvlBuf - 4ull * nodes - 32 : 0;
                const uint64_t t = room * R.n / Q.lvl[d] / 5 * 4;
                tfit = t < tfit ? t : tfit;
            }
            if (R.n <= tile_max && tfit >= R.n) {
                T = R.n;
                ntile = 1;
            } else {
                uint64_t t2 = (tfit < (uint64_t)tile_max ? tfit : (uint64_t)tile_max) & ~127ull;
                if (t2 < 128) t2 = 128;
                const uint64_t tmin = ((uint64_t)R.n + (1u << 21) - 1) >> 21;   // at most 2^21 tiles
                if (t2 < tmin) t2 = (tmin + 127) & ~127ull;
                T = (uint32_t)t2;
                ntile = (R.n + T - 1) / T;
            }
            if (ntile > 1 || all_dirs)
                ent = warp_scan_loop_d((int)R.V, [&](int v) { return (R.nv[v] + dir_bits - 1) / dir_bits; },
                                       [&](int v, uint32_t p) { Q.u[v] = p; });
            dir_bytes = ntab_bytes(R.V) +
                        (ent ? ((4ull * ent + 4ull * (ntile + 1) * R.V + 15) & ~15ull) : 0ull);
        }
    }
    const uint64_t sb = ok ? R.scratch_bytes : 0, sg = ok ? R.nsegs : 0;
    if (!ok) { ntile = 1; T = 0; dir_bytes = 0; }
    int to = 0;
    uint64_t ea = 0, eb = 0;
    lookback2_exclusive_warp(W.states_a, W.states_b, b, (sb << 22) | sg, (dir_bytes << 22) | ntile, ea, eb, &to,
                             hdr64[7]);
    if (lane == 0) {
        W.blk_scratch[b] = ea >> 22;
        W.blk_seg[b] = (uint32_t)(ea & ((1u << 22) - 1));
        W.blk_dir[b] = eb >> 22;
        W.blk_tile[b] = (uint32_t)(eb & ((1u << 22) - 1));
        W.blk_T[b] = T;
        W.blk_ntile[b] = ntile;
        status[b] = !ok ? (misal ? PIVCO_ERR_INVALID_ARG : PIVCO_ERR_CORRUPT) : (to ? PIVCO_ERR_TIMEOUT : PIVCO_OK);
        if (b == nblk - 1) {
            hdr64[0] = (ea >> 22) + sb;
            hdr32[2] = (uint32_t)((ea & ((1u << 22) - 1)) + sg);
            hdr64[2] = (eb >> 22) + dir_bytes;
            hdr32[6] = (uint32_t)((eb & ((1u << 22) - 1)) + ntile);
            // totals from a partial prefix are unusable: every later pass
            // gives the whole batch up (abandoned_batch)
            if (to) atomicExch(&hdr32[13], 1u);
        }
    }
    // the node table (only where the workspace holds it: a sizing run may
    // not; and never from a partial prefix, which would place it over
    // another block's table)
    const uint64_t nbase = decode_ws_fixed_bytes(nblk) + (eb >> 22);
    if (ok && coded && !to && nbase + ntab_bytes(R.V) <= ws_bytes) {
        uint8_t *nt = ws + nbase;
        if (lane < 17) nt[lane] = (uint8_t)Q.first[lane];
        if (lane == 17) nt[17] = (uint8_t)Q.maxd;
        if (lane == 0) {
            *reinterpret_cast<uint32_t *>(nt + 20) = ent;
            *reinterpret_cast<uint32_t *>(nt + 24) = T;
        }
        uint32_t *src = reinterpret_cast<uint32_t *>(nt + kNtabHdr);
        for (int v = lane; v < (int)R.V; v += 32) {
            const uint8_t m = R.marker[v];
            src[v] = mark_ans(m) ? (8u * R.soff[v]) | 0x80000000u : 8u * R.body_off[v];
            src[R.V + v] = Q.ch[v];
            src[2 * R.V + v] = ent ? Q.u[v] : 0u;
        }
        uint8_t *sym = nt + kNtabHdr + 12 * R.V;
        for (int i = lane; i < 256; i += 32) sym[i] = Q.sorted[i];
    }
    __syncwarp();
    // the plan is complete (status, offsets, node table); a block of one tile
    // with no ANS segment and no directory can be decoded from here on
    if (lane == 0) {
        const bool simple = ok && !to && ntile == 1 && sg == 0 && !all_dirs;
        __threadfence();
        atomicExch(&W.plan_done[b], simple ? 3u : 1u);
    }
    __syncwarp();
}

__global__ void __launch_bounds__(32) decode_plan_kernel(const uint8_t *__restrict__ comp,
                                                         const uint64_t *__restrict__ comp_off, int nblk,
                                                         uint8_t *__restrict__ ws, uint64_t ws_bytes,
                                                         int32_t *__restrict__ status) {
    __shared__ WarpRec R;
    __shared__ PlanScratch Q;
    __shared__ int s_tile;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(&reinterpret_cast<uint32_t *>(ws)[3], 1u);
    __syncwarp();
    plan_block(s_tile, comp, comp_off, nblk, ws, ws_bytes, status, R, Q);
}

// zero the header, the look-back states and the batch counters; set the
// tuning and the wait bound
__global__ void dec_ws_init_kernel(uint8_t *ws, int nblk, uint32_t dir_bits, uint32_t tile_max, uint64_t limit_ns) {
    const DecWs W = dec_ws(ws, nblk);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nblk; i += gridDim.x * blockDim.x) {
        W.states_a[i] = 0;
        W.states_b[i] = 0;
        W.segs_done[i] = 0;
        W.dir_done[i] = 0;
        W.plan_done[i] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x < 16) {
        uint32_t *h = reinterpret_cast<uint32_t *>(ws);
        h[threadIdx.x] = threadIdx.x == 7 ? dir_bits : (threadIdx.x == 8 ? tile_max : 0u);
        if (threadIdx.x == 14) h[14] = (uint32_t)limit_ns;
        if (threadIdx.x == 15) h[15] = (uint32_t)(limit_ns >> 32);
    }
}

// True when the plan could not place the batch (a look-back wait ran out
// before the last block's prefix was known) or a CTA of the batched queue
// gave up: the workspace totals and offsets are not to be used.  The caller
// marks every block that still reads OK as timed out (grid-stride, all CTAs
// of a pass may do it) and leaves.  A uniform decision: the flag is set
// before the pass starts, or (batched) before all plans are counted done.
__device__ inline bool abandoned_batch(const uint8_t *ws, int32_t *status, int nblk) {
    if (!*reinterpret_cast<const volatile uint32_t *>(ws + 52)) return false;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x)
        if (*reinterpret_cast<volatile int32_t *>(&status[b]) == PIVCO_OK) status[b] = PIVCO_ERR_TIMEOUT;
    return true;
}

cudaError_t launch_decode_plan(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *ws, size_t ws_bytes,
                               int32_t *status, cudaStream_t st, bool all_dirs) {
    if (nblk <= 0) return cudaSuccess;
    const DecTuning tu = current_tuning();
    dec_ws_init_kernel<<<min(1024, div_up(nblk, 256)), 256, 0, st>>>(ws, nblk, tu.dir_bits | (all_dirs ? 1u << 31 : 0u),
                                                                      tu.tile_max, wait_limit_ns());
    decode_plan_kernel<<<nblk, 32, 0, st>>>(comp, comp_off, nblk, ws, ws_bytes, status);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t read_decode_ws_need(const uint8_t *ws, int nblk, size_t *need, cudaStream_t st) {
    uint8_t h[32];
    cudaError_t e = cudaMemcpyAsync(h, ws, 32, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    *need = dec_regions(nblk, h).need;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// ANS pass: one warp per planned segment
// ---------------------------------------------------------------------------
// Decodes block-local ANS segment g (global numbering) into the scratch.
// Returns the block index (or -1 when g is out of range).  R caches the
// parsed record of the last block this warp saw.
__device__ inline int ans_item(uint32_t g, const uint8_t *__restrict__ comp, const uint64_t *__restrict__ comp_off,
                               int nblk, uint8_t *__restrict__ ws, uint64_t ws_bytes, int32_t *__restrict__ status,
                               const AnsTables &A, WarpRec &R, AnsSm &T, int &last_b, bool &last_ok) {
    const int lane = threadIdx.x & 31;
    const DecWs W = dec_ws(ws, nblk);
    const DecRegions G = dec_regions(nblk, ws);
    const uint64_t scratch_cap = ws_bytes > G.scratch ? ws_bytes - G.scratch : 0;
    uint8_t *scratch = ws + G.scratch;
    const int b = find_block(W.blk_seg, nblk, g);
    if (status[b] != PIVCO_OK) return b;
    const uint8_t *rec = comp + comp_off[b];
    if (b != last_b) {
        last_ok = warp_parse(rec, comp_off[b + 1] - comp_off[b], R);
        last_b = b;
    }
    bool ok = last_ok;
    if (ok) {
        const uint32_t j = g - W.blk_seg[b];
        int node = -1;
        for (int v = lane; v < (int)R.V; v += 32) {
            const uint8_t m = R.marker[v];
            if (mark_ans(m)) {
                const uint32_t s0 = R.segbase[v], ns = ans_seg_count((R.nv[v] + 7) / 8);
                if (j >= s0 && j < s0 + ns) node = v;
            }
        }
        for (int o = 16; o; o >>= 1) node = max(node, __shfl_xor_sync(0xffffffffu, node, o));
        if (node < 0) ok = false;
        if (ok) {
            const uint32_t s = j - R.segbase[node];
            const uint32_t raw = (R.nv[node] + 7) / 8;
            const uint8_t mk = R.marker[node];
            const uint64_t sdst = W.blk_scratch[b] + R.soff[node];
            if (sdst + scratch_stride(raw) > scratch_cap) {
                if (lane == 0) status[b] = PIVCO_ERR_CAPACITY;
                __syncwarp();
                return b;
            }
            uint64_t sp = 0;
            uint32_t nw = 0;
            const uint8_t *body = rec + R.body_off[node];
            const uint32_t blen = R.alen[node];
            ok = ans_segment_at(body, blen, raw, s, sp, nw);
            if (ok) {
                load_ans_table(T, A, (mk & 0x7F) - 1, lane, 32);
                __syncwarp();
                const uint32_t sbytes = min(kAnsSeg, raw - s * kAnsSeg), Wl = ans_seg_lanes(sbytes);
                ok = ans_decode_segment(body + sp, body + sp + 4 * Wl, nw, sbytes, T, (mk & 0x80) ? 0xFF : 0,
                                        scratch + sdst + (size_t)s * kAnsSeg, R.stg);
                if (ok && s + 1 == ans_seg_count(raw) && sp + 4ull * Wl + 2ull * nw != blen) ok = false;
                if (s + 1 == ans_seg_count(raw) && lane < 16) scratch[sdst + raw + lane] = 0;
            }
        }
    }
    if (!ok && lane == 0) status[b] = PIVCO_ERR_CORRUPT;
    __syncwarp();
    return b;
}

constexpr int kAnsDecWarps = 4;

__global__ void __launch_bounds__(32 * kAnsDecWarps) ans_decode_planned_kernel(const uint8_t *__restrict__ comp,
                                                                               const uint64_t *__restrict__ comp_off,
                                                                               int nblk, uint8_t *__restrict__ ws,
                                                                               uint64_t ws_bytes,
                                                                               int32_t *__restrict__ status,
                                                                               const __grid_constant__ AnsTables A) {
    __shared__ WarpRec R[kAnsDecWarps];
    __shared__ AnsSm T[kAnsDecWarps];
    if (abandoned_batch(ws, status, nblk)) return;
    const int w = threadIdx.x >> 5;
    const uint32_t total = reinterpret_cast<const uint32_t *>(ws)[2];
    int last_b = -1;
    bool last_ok = false;
    for (uint32_t g = blockIdx.x * kAnsDecWarps + w; g < total; g += gridDim.x * kAnsDecWarps)
        ans_item(g, comp, comp_off, nblk, ws, ws_bytes, status, A, R[w], T[w], last_b, last_ok);
}

cudaError_t launch_ans_decode_planned(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *ws,
                                      size_t ws_bytes, int32_t *status, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    ans_decode_planned_kernel<<<sms * 4, 32 * kAnsDecWarps, 0, st>>>(comp, comp_off, nblk, ws, ws_bytes, status,
                                                                     host_ans_tables());
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// CTA tiles (the bottom-up merge, Sec. 3)
//
// A tile is decoded by one CTA.  Its levels live in two shared-memory level
// buffers; bottom-up, each level is split into windows of 32 groups (a group
// is 32 consecutive symbols of one node, one lane each), and the CTA's warps
// take the windows of a level in rounds, one window per warp per round.  A
// group needs the ones of its node before it: within a window they come from
// a segmented warp scan, across the windows of a round from the windows'
// summaries (one barrier per round), across rounds from a carry every
// thread keeps.  Large tiles (a whole 64 KiB block when its levels fit) need
// no rank directory and amortise the tile's set-up over many symbols.
// ---------------------------------------------------------------------------
constexpr int kTileWarps = kDecWarps;
constexpr int kWnodeMax = 512;                 // window-node entries of all levels below the root

struct WinSum {                                // one window of a round
    uint32_t sum;                              // ones of its last node from that node's start in the window
    uint32_t flags;                            // 1 its first node starts at its first group,
};                                             //   2 a node starts in it, 4 active

struct __align__(16) CtaTile {
    uint8_t buf[2][kLvlBuf + kWSlack];         // level buffers: depth d writes buf[d & 1]
    uint32_t pos[256];                         // bit address of node v's next bit (bit 31: in the ANS scratch)
    uint32_t dem[256];                         // bits of node v in the current chunk
    uint32_t ch[256];                          // children (node table format)
    uint16_t sp[256];                          // byte offset of node v's sequence in its level buffer
    uint16_t gs[256];                          // first 32-symbol group of node v within its level
    uint16_t lg[16];                           // groups of each level
    uint16_t wn_off[16];                       // first window-node entry of each level
    WinSum win[2][kTileWarps];                 // window summaries, two rounds deep
    uint8_t wnode[kWnodeMax];                  // node holding the first group of each window
    uint8_t ftab[256];                         // the block's symbols in (length, symbol) order (flat nodes)
    uint8_t first[17];
    uint8_t maxd;
    uint8_t pad[2];
    int32_t blk, flag;
    uint32_t pad2[2];
};
static_assert(sizeof(CtaTile) % 16 == 0, "tiles must stay 16-byte aligned");

// Byte-permute selectors of a bitmap byte (low 16 bits: its low nibble,
// high 16 bits: its high nibble): a one takes the next byte of the right
// window (bytes 4..7), a zero the next byte of the left window (bytes 0..3).
// A leaf side's window is its symbol in all four bytes, so one table serves
// every kind of children.
__device__ inline void sel_init(uint32_t *sel) {
    const int t = threadIdx.x;
    for (int b8 = t; b8 < 256; b8 += blockDim.x) {
        uint32_t pair = 0;
        for (int h = 0; h < 2; h++) {
            const uint32_t nib = (b8 >> (4 * h)) & 15u;
            uint32_t s = 0, ones = 0, zeros = 0;
            for (int j = 0; j < 4; j++) {
                const uint32_t bit = (nib >> j) & 1u;
                s |= (bit ? 4 + ones : zeros) << (4 * j);
                ones += bit;
                zeros += 1 - bit;
            }
            pair |= s << (16 * h);
        }
        sel[b8] = pair;
    }
}

struct TileSrc {
    const uint8_t *rec;
    const uint8_t *scr;
    uint64_t scr_bytes;
    uint32_t rec_bytes;
};

// 32 bits of a node bitmap from bit address pos + k (bit 31 of pos: scratch)
__device__ inline uint32_t tile_bits(const TileSrc &s, uint32_t pos, uint32_t k) {
    const bool sc = (pos >> 31) != 0;
    const uint64_t e = (uint64_t)(pos & 0x7FFFFFFFu) + k;
    const uint64_t wi = e >> 5;
    const uint32_t sh = (uint32_t)e & 31u;
    const uint32_t *w = reinterpret_cast<const uint32_t *>(sc ? s.scr : s.rec);
    const uint64_t lim = sc ? s.scr_bytes : (uint64_t)s.rec_bytes;
    const uint32_t lo = 4 * wi + 4 <= lim ? __ldcg(w + wi) : 0u;
    const uint32_t hi = (sh && 4 * wi + 8 <= lim) ? __ldcg(w + wi + 1) : 0u;
    return __funnelshift_r(lo, hi, sh);
}

// The two words under 32 bits of a bitmap, loaded ahead of their use
struct BitLd {
    uint32_t lo, hi, sh;
};
__device__ inline BitLd tile_ld(const TileSrc &s, uint32_t pos, uint32_t k) {
    const bool sc = (pos >> 31) != 0;
    const uint64_t e = (uint64_t)(pos & 0x7FFFFFFFu) + k;
    const uint64_t wi = e >> 5;
    BitLd b;
    b.sh = (uint32_t)e & 31u;
    const uint32_t *w = reinterpret_cast<const uint32_t *>(sc ? s.scr : s.rec);
    const uint64_t lim = sc ? s.scr_bytes : (uint64_t)s.rec_bytes;
    b.lo = 4 * wi + 4 <= lim ? __ldcg(w + wi) : 0u;
    b.hi = (b.sh && 4 * wi + 8 <= lim) ? __ldcg(w + wi + 1) : 0u;
    return b;
}
__device__ inline uint32_t tile_word(const BitLd &b) { return __funnelshift_r(b.lo, b.hi, b.sh); }

// popcount of bits [e, e + len) (len <= 256) of the bitmap at bit address
// pos: the covering words are loaded together, then counted
__device__ inline uint32_t tile_popc(const TileSrc &s, uint32_t pos, uint32_t e, uint32_t len) {
    const bool sc = (pos >> 31) != 0;
    const uint64_t a = (uint64_t)(pos & 0x7FFFFFFFu) + e;
    const uint64_t w0 = a >> 5;
    const uint32_t sh = (uint32_t)a & 31u;
    const uint32_t *w = reinterpret_cast<const uint32_t *>(sc ? s.scr : s.rec);
    const uint64_t lim = sc ? s.scr_bytes : (uint64_t)s.rec_bytes;
    const uint32_t nw = (sh + len + 31) >> 5;   // words holding the range (<= 9)
    uint32_t x[9];
#pragma unroll
    for (int i = 0; i < 9; i++) x[i] = ((uint32_t)i < nw && 4 * (w0 + i) + 4 <= lim) ? __ldcg(w + w0 + i) : 0u;
    // all bits of the loaded words, less those before sh in the first and
    // those from sh + len on in the last
    uint32_t c = 0, xl = 0;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        c += __popc(x[i]);
        xl = (uint32_t)i + 1 == nw ? x[i] : xl;
    }
    c -= __popc(x[0] & ((1u << sh) - 1u));
    const uint32_t eb = (sh + len) & 31u;
    if (eb) c -= __popc(xl >> eb);
    return c;
}

// 8 bytes of a level buffer from byte a (reads up to 11 bytes past a)
__device__ inline void win8(const uint8_t *buf, uint32_t a, uint32_t &x0, uint32_t &x1) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(buf + (a & ~3u));
    const uint32_t sh = (a & 3u) * 8u;
    const uint32_t w0 = w[0], w1 = w[1], w2 = w[2];
    x0 = __funnelshift_r(w0, w1, sh);
    x1 = __funnelshift_r(w1, w2, sh);
}

// 32 output symbols of a node from bitmap word w: r0 / r1 zeros / ones of the
// node before this word, i.e. the start of its left / right window.
__device__ inline void merge32(const CtaTile &S, const uint8_t *bin, uint32_t chv, uint32_t r0, uint32_t r1,
                               uint32_t w, const uint32_t *sel, uint32_t (&o)[8]) {
    const uint32_t c0 = chv & 0xFFFFu, c1 = chv >> 16;
    const bool i0 = !(c0 & 0x8000u), i1 = !(c1 & 0x8000u);
    uint32_t la = i0 ? min((uint32_t)S.sp[c0 & 0xFFu] + r0, (uint32_t)kLvlBuf) : 0u;
    uint32_t ra = i1 ? min((uint32_t)S.sp[c1 & 0xFFu] + r1, (uint32_t)kLvlBuf) : 0u;
    const uint32_t kl = (c0 & 0xFFu) * 0x01010101u, kr = (c1 & 0xFFu) * 0x01010101u;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const uint32_t b8 = (w >> (8 * q)) & 0xFFu;
        const uint32_t p0 = __popc(b8 & 15u), p8 = __popc(b8);
        uint32_t L0 = kl, L1 = kl, R0 = kr, R1 = kr;
        if (i0) win8(bin, la, L0, L1);
        if (i1) win8(bin, ra, R0, R1);
        const uint32_t Lh = __funnelshift_rc(L0, L1, 8u * (4u - p0));
        const uint32_t Rh = __funnelshift_rc(R0, R1, 8u * p0);
        const uint32_t sp = sel[b8];
        o[2 * q] = __byte_perm(L0, R0, sp);
        o[2 * q + 1] = __byte_perm(Lh, Rh, sp >> 16);
        la += 8u - p8;
        ra += p8;
    }
}

// 32 output symbols of a flat node (Sec. 2.2.3, merge_flat_D): the D-bit
// indices at bit address pos (a raw body in the record), each mapped through
// the node's symbols tab[0 .. 2^D).
template <int D>
__device__ inline void flat32_t(const TileSrc &s, uint32_t pos, const uint8_t *tab, uint32_t (&o)[8]) {
    const uint64_t e = pos & 0x7FFFFFFFu;
    const uint64_t wi = e >> 5;
    const uint32_t sh = (uint32_t)e & 31u;
    const uint32_t *w = reinterpret_cast<const uint32_t *>(s.rec);
    const uint64_t lim = s.rec_bytes;
    uint32_t x[D + 1], b[D];
#pragma unroll
    for (int k = 0; k <= D; k++) x[k] = 4 * (wi + k) + 4 <= lim ? __ldca(w + wi + k) : 0u;
#pragma unroll
    for (int k = 0; k < D; k++) b[k] = __funnelshift_r(x[k], x[k + 1], sh);
    constexpr uint32_t m = (1u << D) - 1u;
#pragma unroll
    for (int q = 0; q < 8; q++) {
        uint32_t word = 0;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int bit = (4 * q + i) * D, k = bit >> 5, r = bit & 31;
            uint32_t v = b[k] >> r;
            if (r + D > 32) v |= b[k + 1] << (32 - r);
            word |= (uint32_t)tab[v & m] << (8 * i);
        }
        o[q] = word;
    }
}

__device__ inline void flat32(const TileSrc &s, uint32_t D, uint32_t pos, const uint8_t *tab, uint32_t (&o)[8]) {
    switch (D) {
        case 2: flat32_t<2>(s, pos, tab, o); break;
        case 3: flat32_t<3>(s, pos, tab, o); break;
        case 4: flat32_t<4>(s, pos, tab, o); break;
        case 5: flat32_t<5>(s, pos, tab, o); break;
        case 6: flat32_t<6>(s, pos, tab, o); break;
        case 7: flat32_t<7>(s, pos, tab, o); break;
        default: flat32_t<8>(s, pos, tab, o); break;
    }
}

// L1 prefetch of the words under 32 indices of a flat node (<= 36 bytes)
__device__ inline void flat_prefetch(const TileSrc &s, uint32_t D, uint32_t pos) {
    const uint64_t e = pos & 0x7FFFFFFFu;
    const uint64_t b0 = (e >> 5) * 4, b1 = ((e + 32ull * D) >> 5) * 4;
    if (b0 < s.rec_bytes) asm volatile("prefetch.global.L1 [%0];" ::"l"(s.rec + b0));
    if ((b1 >> 7) != (b0 >> 7) && b1 < s.rec_bytes) asm volatile("prefetch.global.L1 [%0];" ::"l"(s.rec + b1));
}

// the children's demands must be the node's zeros and ones
__device__ inline bool children_ok(const CtaTile &S, uint32_t chv, uint32_t dv, uint32_t ones) {
    const uint32_t c0 = chv & 0xFFFFu, c1 = chv >> 16;
    bool ok = true;
    if (!(c0 & 0x8000u)) ok = ok && S.dem[c0] == dv - ones;
    if (!(c1 & 0x8000u)) ok = ok && S.dem[c1] == ones;
    return ok;
}

// up to 32 output bytes at p (any alignment)
__device__ inline void st_out32(uint8_t *p, const uint32_t (&o)[8], uint32_t valid) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    if (valid >= 32 && !(a & 15)) {
        reinterpret_cast<uint4 *>(p)[0] = make_uint4(o[0], o[1], o[2], o[3]);
        reinterpret_cast<uint4 *>(p)[1] = make_uint4(o[4], o[5], o[6], o[7]);
    } else if (!(a & 3)) {
#pragma unroll
        for (int j = 0; j < 8; j++) {
            if (4u * j + 4 <= valid) {
                reinterpret_cast<uint32_t *>(p)[j] = o[j];
            } else {
#pragma unroll
                for (int i = 0; i < 3; i++)
                    if (4u * j + i < valid) p[4 * j + i] = (uint8_t)(o[j] >> (8 * i));
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < 8; j++)
#pragma unroll
            for (int i = 0; i < 4; i++)
                if (4u * j + i < valid) p[4 * j + i] = (uint8_t)(o[j] >> (8 * i));
    }
}

// Spans, groups and window nodes of every level for the current demands,
// by the whole CTA: warp w lays out levels w, w + 8, ... (a level's spans
// and groups are a scan over its own nodes); the levels' window-node tables
// then follow one another in depth order.  False (in every thread) when a
// level (depth >= 1) does not fit a buffer or the window nodes do not fit
// their table.
__device__ inline bool ct_layout(CtaTile &S) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int maxd = S.maxd;
    bool fits = true;
    for (int d = warp; d < maxd; d += kTileWarps) {
        const int f0 = S.first[d], f1 = S.first[d + 1];
        uint64_t carry = 0;
        for (int base = f0; base < f1; base += 32) {
            const int v = base + lane;
            uint64_t x = 0;
            if (v < f1) {
                const uint32_t dv = S.dem[v];
                if (d && dv > (uint32_t)kLvlBuf) fits = false;
                const uint32_t by = d ? ((min(dv, (uint32_t)kLvlBuf) + 3u) & ~3u) : 0u;
                x = ((uint64_t)by << 32) | max(1u, (dv + 31u) >> 5);
            }
            uint64_t inc = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            const uint64_t ex = carry + inc - x;
            if (v < f1) {
                S.sp[v] = (uint16_t)min((uint64_t)kLvlBuf, ex >> 32);
                S.gs[v] = (uint16_t)ex;
            }
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (d && (carry >> 32) > (uint64_t)kLvlBuf) fits = false;
        if ((uint32_t)carry > 0xFFFFu) fits = false;
        if (lane == 0) S.lg[d] = (uint16_t)carry;
    }
    __syncthreads();
    // window-node table offsets: lane d holds level d's windows (none at the root)
    const uint32_t nwin_l = lane >= 1 && lane < maxd ? ((uint32_t)S.lg[lane] + 31) >> 5 : 0u;
    uint32_t wi = nwin_l;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
    }
    if (__shfl_sync(0xffffffffu, wi, 31) > (uint32_t)kWnodeMax) fits = false;
    const uint32_t wn_l = wi - nwin_l;
    for (int d = warp; d < maxd; d += kTileWarps) {
        const uint32_t wn = __shfl_sync(0xffffffffu, wn_l, d), nwin = __shfl_sync(0xffffffffu, nwin_l, d);
        if (lane == 0) S.wn_off[d] = (uint16_t)wn;
        // the node holding the first group of each window of the level: the
        // last node whose first group is at or before it
        const int f0 = S.first[d], f1 = S.first[d + 1];
        for (uint32_t i = lane; i < nwin && wn + i < (uint32_t)kWnodeMax; i += 32) {
            int lo = f0, hi = f1;
            while (hi - lo > 1) {
                const int m = (lo + hi) >> 1;
                if ((uint32_t)S.gs[m] <= 32u * i) lo = m; else hi = m;
            }
            S.wnode[wn + i] = (uint8_t)lo;
        }
    }
    return !__syncthreads_or(!fits);
}

// Demands of a chunk of C root symbols from the current cursors, top-down:
// a node's popcount over its range splits its demand between its children
// (one warp).
__device__ inline void ct_demand(CtaTile &S, const TileSrc &src, uint32_t V, uint32_t C) {
    const int lane = threadIdx.x & 31;
    for (uint32_t v = lane; v < V; v += 32) S.dem[v] = 0;
    __syncwarp();
    if (lane == 0) S.dem[0] = C;
    __syncwarp();
    for (uint32_t v = 0; v < V; v++) {   // breadth-first: parents before children
        if (ch_flat_d(S.ch[v])) continue;   // a flat node has no children to split for
        const uint32_t dv = S.dem[v];
        uint32_t ones = 0;
        for (uint32_t e = 32 * lane; e < dv; e += 1024) {
            uint32_t w = tile_bits(src, S.pos[v], e);
            if (dv - e < 32) w &= (1u << (dv - e)) - 1u;
            ones += __popc(w);
        }
        ones = __reduce_add_sync(0xffffffffu, ones);
        if (lane == 0) {
            const uint32_t chv = S.ch[v];
            const uint32_t c0 = chv & 0xFFFFu, c1 = chv >> 16;
            if (!(c0 & 0x8000u)) S.dem[c0] = dv - ones;
            if (!(c1 & 0x8000u)) S.dem[c1] = ones;
        }
        __syncwarp();
    }
}

// The group of lane `lane` in the window of 32 groups at `base` of a level
// (nodes f0 .. f1-1, G groups): its node counts the nodes that start in the
// window at or before it, after node vcur.
struct WtLoc {
    uint32_t v, kk, dv, starts;
    bool act;
};
__device__ inline WtLoc wt_locate(const CtaTile &S, uint32_t f1, uint32_t G, uint32_t base, uint32_t vcur) {
    const int lane = threadIdx.x & 31;
    const uint32_t le = 0xFFFFFFFFu >> (31 - lane);
    const uint32_t cand = vcur + 1 + lane;
    uint32_t bit = 0;
    if (cand < f1) {
        const uint32_t s = (uint32_t)S.gs[cand] - base;
        if (s < 32) bit = 1u << s;
    }
    WtLoc L;
    L.starts = __reduce_or_sync(0xffffffffu, bit);
    L.v = vcur + __popc(L.starts & le);
    const uint32_t g = base + lane;
    L.kk = (g - S.gs[L.v]) * 32u;
    L.dv = S.dem[L.v];
    L.act = g < G && L.kk < L.dv;
    return L;
}

// The window at group `base` of level d (a warp's window of a round): its
// groups' nodes and the two bitmap words under each group, loaded ahead.
__device__ inline void ct_fetch(const CtaTile &S, const TileSrc &src, int d, uint32_t base, WtLoc &L, BitLd &ld) {
    const int lane = threadIdx.x & 31;
    ld = BitLd{0u, 0u, 0u};
    L = WtLoc{0u, 0u, 0u, 0u, false};
    if (d >= 1) {
        const uint32_t G = S.lg[d];
        if (base < G) {
            const uint32_t u = S.wnode[S.wn_off[d] + (base >> 5)];
            L = wt_locate(S, S.first[d + 1], G, base, (uint32_t)S.gs[u] == base ? u - 1 : u);
            if (L.act) {
                const uint32_t fD = ch_flat_d(S.ch[L.v]);
                if (fD) flat_prefetch(src, fD, S.pos[L.v] + L.kk * fD);
                else ld = tile_ld(src, S.pos[L.v], L.kk);
            }
        }
    } else if (d == 0) {
        L.dv = S.dem[0];
        L.kk = 32u * (base + lane);
        L.act = L.kk < L.dv;
        if (L.act) {
            const uint32_t fD = ch_flat_d(S.ch[0]);
            if (fD) flat_prefetch(src, fD, S.pos[0] + L.kk * fD);
            else ld = tile_ld(src, S.pos[0], L.kk);
        }
    }
}

// One level (depth d >= 1) of the current chunk into its buffer.  nx / nld
// hold the warp's window of this level's first round on entry and of the
// next level's first round on return; par alternates the summary slots.
// The level ends without a barrier: a round reads the level buffer below it
// only after its summary barrier, so the next level's first barrier (or the
// root's) is the one that orders this level's writes before those reads and
// its reads before the next level's writes to the other buffer.  Returns
// false when this thread found the level corrupt (the caller combines).
__device__ inline bool ct_level(CtaTile &S, const TileSrc &src, int d, const uint32_t *sel, WtLoc &nx, BitLd &nld,
                                uint32_t &par) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint8_t *bin = S.buf[(d + 1) & 1];
    uint8_t *bout = S.buf[d & 1];
    const uint32_t G = S.lg[d];
    const uint32_t le = 0xFFFFFFFFu >> (31 - lane);
    uint32_t rc_sum = 0;   // carry into the round: the ones so far of the node running into it
    bool bad = false;
    for (uint32_t r0 = 0; r0 < G; r0 += 32 * kTileWarps) {
        const uint32_t base = r0 + 32 * warp;
        const WtLoc L = nx;
        const BitLd ld = nld;
        if (r0 + 32 * kTileWarps < G) ct_fetch(S, src, d, base + 32 * kTileWarps, nx, nld);
        else ct_fetch(S, src, d - 1, 32 * warp, nx, nld);
        if (base >= G) {
            // past the level's end (its last round only): an empty summary
            // and nothing to merge; the carry into later rounds is not needed
            if (lane == 0) S.win[par][warp] = WinSum{0u, 0u};
            __syncthreads();
            par ^= 1u;
            continue;
        }
        const uint32_t starts = L.starts, v = L.v, kk = L.kk, dv = L.dv;
        const bool act = L.act;
        uint32_t w = 0;
        if (act) {
            w = tile_word(ld);
            if (dv - kk < 32) w &= (1u << (dv - kk)) - 1u;
        }
        const uint32_t pc = __popc(w);
        // ones of the node before this word within the window: segmented scan
        uint32_t inc = pc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const uint32_t sl = starts & le;
        const int s0 = sl ? 31 - __clz(sl) : -1;
        const uint32_t before = __shfl_sync(0xffffffffu, inc, s0 > 0 ? s0 - 1 : 0);
        uint32_t r1 = inc - pc - (s0 > 0 ? before : 0u);
        // a level of one window (warp 0's, in the first round) takes no carry
        const bool one = G <= 32;
        if (lane == 31 && !one) S.win[par][warp] = WinSum{r1 + pc, (starts & 1u) | (starts ? 2u : 0u) | (base < G ? 4u : 0u)};
        __syncthreads();
        // the carry into each window of the round: lane p takes window p's
        // summary; the carry out of a window is a segmented inclusive sum of
        // the windows' sums (a segment starts at a window where a node
        // starts), the first segment continuing the previous round's carry
        uint32_t cin = 0;
        if (!one) {
            const WinSum x = lane < kTileWarps ? S.win[par][lane] : WinSum{0u, 0u};
            uint32_t val = x.sum, seg = (x.flags >> 1) & 1u;
#pragma unroll
            for (int o = 1; o < kTileWarps; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, val, o), f = __shfl_up_sync(0xffffffffu, seg, o);
                if (lane >= o && !seg) { val += y; seg |= f; }
            }
            if (!seg) val += rc_sum;
            const uint32_t prev = __shfl_up_sync(0xffffffffu, val, 1);
            // the head node runs in from the window before unless it starts here
            const uint32_t c = (x.flags & 1u) ? 0u : (lane ? prev : rc_sum);
            cin = __shfl_sync(0xffffffffu, c, warp);
            const uint32_t act = __ballot_sync(0xffffffffu, (x.flags & 4u) != 0);   // window 0 always is
            const int last = 31 - __clz(act);
            rc_sum = __shfl_sync(0xffffffffu, val, last);
        }
        par ^= 1u;
        if (s0 < 0) r1 += cin;   // groups of the node that runs in from the previous window
        if (act) {
            const uint32_t chv = S.ch[v], fD = ch_flat_d(chv);
            uint32_t o[8];
            if (fD) {
                flat32(src, fD, S.pos[v] + kk * fD, S.ftab + (chv & 0xFFu), o);
            } else {
                if (kk + 32 >= dv && !children_ok(S, chv, dv, r1 + pc)) bad = true;
                merge32(S, bin, chv, kk - r1, r1, w, sel, o);
            }
            uint8_t *p = bout + S.sp[v] + kk;
            // spans are 4-byte aligned: 32-bit stores, the ones inside the node's span
            uint32_t *p4 = reinterpret_cast<uint32_t *>(p);
#pragma unroll
            for (int j = 0; j < 8; j++)
                if (4u * j < dv - kk) p4[j] = o[j];
        }
    }
    return !bad;
}

// The root level of the current chunk into the output.
__device__ inline bool ct_root(CtaTile &S, const TileSrc &src, uint8_t *out, const uint32_t *sel, WtLoc nx,
                               BitLd nld, uint32_t &par) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint8_t *bin = S.buf[1];
    const uint32_t dv = S.dem[0], chv = S.ch[0];
    const uint32_t G = (dv + 31) >> 5;
    uint32_t rc = 0;   // ones of the root before the round
    for (uint32_t r0 = 0; r0 < G; r0 += 32 * kTileWarps) {
        const uint32_t base = r0 + 32 * warp;
        const WtLoc L = nx;
        const BitLd ld = nld;
        if (r0 + 32 * kTileWarps < G) ct_fetch(S, src, 0, base + 32 * kTileWarps, nx, nld);
        const uint32_t kk = L.kk;
        const bool act = L.act;
        uint32_t w = 0;
        if (act) {
            w = tile_word(ld);
            if (dv - kk < 32) w &= (1u << (dv - kk)) - 1u;
        }
        const uint32_t pc = __popc(w);
        uint32_t inc = pc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) S.win[par][warp].sum = inc;
        __syncthreads();
        // the windows' sums (lane p: window p; an empty window's is 0): the
        // ones before this warp's window and the round's total
        uint32_t cin;
        {
            const uint32_t ws = lane < kTileWarps ? S.win[par][lane].sum : 0u;
            uint32_t wi = ws;
#pragma unroll
            for (int o = 1; o < kTileWarps; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            cin = rc + __shfl_sync(0xffffffffu, wi - ws, warp);
            rc += __shfl_sync(0xffffffffu, wi, kTileWarps - 1);
        }
        par ^= 1u;
        if (act) {
            const uint32_t r1 = cin + inc - pc;
            uint32_t o[8];
            if (const uint32_t fD = ch_flat_d(chv)) flat32(src, fD, S.pos[0] + kk * fD, S.ftab + (chv & 0xFFu), o);
            else merge32(S, bin, chv, kk - r1, r1, w, sel, o);
            st_out32(out + kk, o, min(32u, dv - kk));
        }
    }
    return children_ok(S, chv, dv, rc);
}

// fills n bytes at p with x (whole CTA)
__device__ inline void cta_fill(uint8_t *p, uint32_t n, uint8_t x) {
    const int t = threadIdx.x;
    const uint32_t head = min(n, (uint32_t)((16 - (reinterpret_cast<uintptr_t>(p) & 15)) & 15));
    if (t < (int)head) p[t] = x;
    const uint32_t body = (n - head) / 16;
    const uint32_t x4 = x * 0x01010101u;
    uint4 *q = reinterpret_cast<uint4 *>(p + head);
    for (uint32_t i = t; i < body; i += blockDim.x) q[i] = make_uint4(x4, x4, x4, x4);
    for (uint32_t i = head + 16 * body + t; i < n; i += blockDim.x) p[i] = x;
}

// Decodes tile gt of the queue with the whole CTA (every thread calls it
// with the same arguments).  b: the tile's block when the caller knows it.
__device__ inline void cta_tile(uint32_t gt, const uint8_t *__restrict__ comp, const uint64_t *__restrict__ comp_off,
                                int nblk, uint8_t *__restrict__ out, const uint64_t *__restrict__ out_off,
                                const uint8_t *__restrict__ ws, uint64_t ws_bytes, int32_t *__restrict__ status,
                                CtaTile &S, const uint32_t *sel, int b = -1) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const DecWs W = dec_ws(const_cast<uint8_t *>(ws), nblk);
    const DecRegions G = dec_regions(nblk, ws);
    // one block and one status for the whole CTA (every decision below that
    // chooses a path with barriers is the same in every thread)
    if (warp == 0) {
        if (b < 0) {
            const uint32_t ttot = reinterpret_cast<const uint32_t *>(ws)[6];
            b = find_block_warp(W.blk_tile, nblk, gt, (int)((uint64_t)gt * (uint32_t)nblk / max(ttot, 1u)));
        }
        if (lane == 0) { S.blk = b; S.flag = *reinterpret_cast<volatile int32_t *>(&status[b]); }
    }
    __syncthreads();
    b = S.blk;
    const int32_t st0 = S.flag;   // (nothing in the tile writes blk or flag again)
    if (st0 != PIVCO_OK) return;
    const uint32_t k = gt - W.blk_tile[b], ntile = W.blk_ntile[b], T = W.blk_T[b];
    const uint8_t *rec = comp + comp_off[b];
    uint8_t *dst = out + out_off[b];
    const uint64_t ocap = out_off[b + 1] - out_off[b];
    const uint32_t rb = ld_le32(rec), n = ld_le32(rec + 4);
    const uint32_t V = (uint32_t)rec[8] | ((uint32_t)rec[9] << 8), kind = rec[10], aux = rec[11];
    if (n != ocap) {                     // the plan validated magic / size / layout
        if (t == 0) status[b] = PIVCO_ERR_CAPACITY;
        return;
    }
    if (kind == 0) return;
    const uint32_t P0 = k * T, P1 = min(n, P0 + T);
    if (kind == 1) {
        cta_fill(dst + P0, P1 - P0, (uint8_t)aux);
        return;
    }
    const uint64_t nbase = G.dir + W.blk_dir[b], ntb = ntab_bytes(V);
    const uint8_t *nt = ws + nbase;
    const uint32_t ent = nbase + ntb <= ws_bytes ? *reinterpret_cast<const uint32_t *>(nt + 20) : 0u;
    const uint32_t *cursors = reinterpret_cast<const uint32_t *>(nt + ntb) + ent;
    if (nbase + ntb > ws_bytes ||
        (ntile > 1 && nbase + ntb + 4ull * ent + 4ull * (ntile + 1) * V > ws_bytes)) {
        if (t == 0) status[b] = PIVCO_ERR_CAPACITY;
        return;
    }
    const uint32_t *nsrc = reinterpret_cast<const uint32_t *>(nt + kNtabHdr);
    const uint32_t *nv = reinterpret_cast<const uint32_t *>(rec + kNvOff);
    if (t < 17) S.first[t] = nt[t];
    if (t == 17) S.maxd = nt[17];
    if (t < 64) reinterpret_cast<uint32_t *>(S.ftab)[t] = reinterpret_cast<const uint32_t *>(nt + kNtabHdr + 12 * V)[t];
    const uint64_t sbase = G.scratch + W.blk_scratch[b];
    TileSrc src;
    src.rec = rec;
    src.rec_bytes = rb;
    src.scr = ws + sbase;
    src.scr_bytes = ws_bytes > sbase ? ws_bytes - sbase : 0;
    int bad = V > 255;   // the plan has checked it
    if ((uint32_t)t < V) {
        const uint32_t v = t;
        const uint32_t nvv = __ldg(nv + v);
        const uint32_t cs = ntile > 1 ? cursors[(size_t)k * V + v] : 0u;
        const uint32_t e = ntile > 1 ? cursors[(size_t)(k + 1) * V + v] : nvv;
        const uint32_t s0 = nsrc[v], chv = nsrc[V + v];
        const uint32_t bpe = max(1u, ch_flat_d(chv));   // bits per symbol of the node's body
        if (e < cs || e > nvv || bpe > 8 || (uint64_t)(s0 & 0x7FFFFFFFu) + (uint64_t)nvv * bpe >= 0x80000000ull ||
            (bpe > 1 && ((s0 >> 31) || (chv & 0xFFu) + (1u << bpe) > 256u)))
            bad = 1;
        S.pos[v] = s0 + cs * bpe;
        S.dem[v] = e - cs;
        S.ch[v] = chv;
    }
    __syncthreads();
    if (t == 0 && S.dem[0] != P1 - P0) bad = 1;
    if ((uint32_t)t < V) {   // a child never has more symbols than its parent
        const uint32_t chv = S.ch[t], c0 = chv & 0xFFFFu, c1 = chv >> 16;
        const uint32_t dc = ((c0 & 0x8000u) ? 0u : S.dem[c0]) + ((c1 & 0x8000u) ? 0u : S.dem[c1]);
        if (dc > S.dem[t]) bad = 1;
    }
    // the node table's levels: at most 16, first nodes non-decreasing up to V
    if (t == 0 && (S.maxd < 1 || S.maxd > 16 || S.first[0] != 0 || S.first[S.maxd] != V)) bad = 1;
    if (t >= 1 && t <= 16 && t <= S.maxd && S.first[t] < S.first[t - 1]) bad = 1;
    if (__syncthreads_or(bad)) {
        if (t == 0) status[b] = PIVCO_ERR_CORRUPT;
        return;
    }
    // the whole tile at once when its levels fit, else chunks found top-down
    uint32_t P = P0, C = P1 - P0, par = 0;
    bool chunked = false;
    while (P < P1) {
        if (chunked) {
            if (warp == 0) ct_demand(S, src, V, C);
            __syncthreads();
        }
        const bool fits = ct_layout(S);
        if (!fits) {
            chunked = true;
            C = max(32u, (C / 2) & ~31u);
            continue;
        }
        bool ok = true;
        WtLoc nx;
        BitLd nld;
        ct_fetch(S, src, (int)S.maxd - 1, 32 * warp, nx, nld);
        for (int d = (int)S.maxd - 1; d >= 1; d--) ok = ct_level(S, src, d, sel, nx, nld, par) && ok;
        ok = ct_root(S, src, dst + P, sel, nx, nld, par) && ok;
        if (__syncthreads_or(!ok)) {
            if (t == 0) status[b] = PIVCO_ERR_CORRUPT;
            return;
        }
        if ((uint32_t)t < V) S.pos[t] += S.dem[t] * max(1u, ch_flat_d(S.ch[t]));
        __syncthreads();
        P += C;
        C = min(C, P1 - P);
    }
    if (chunked && (uint32_t)t < V) {   // the chunks must end exactly at the tile's end cursors
        const uint32_t ce = ntile > 1 ? cursors[(size_t)(k + 1) * V + t] : __ldg(nv + t);
        if (S.pos[t] != nsrc[t] + ce * max(1u, ch_flat_d(S.ch[t]))) bad = 1;
    }
    // the last tile checks the pad bits of every body
    if (k + 1 == ntile && (uint32_t)t < V) {
        const uint32_t nb = __ldg(nv + t) * max(1u, ch_flat_d(S.ch[t]));
        if ((nb & 7) && (tile_bits(src, nsrc[t], nb & ~7u) & 0xFFu) >> (nb & 7)) bad = 1;
    }
    if (__syncthreads_or(bad) && t == 0) status[b] = PIVCO_ERR_CORRUPT;
}

// ---------------------------------------------------------------------------
// Rank directory and tile-boundary cursors of one block (whole CTA).  They
// follow the block's node table in its directory region:
//   dir[u_v + i]   ones of node v before its superblock i (dir_bits bits each)
//   cur[k V + v]   node v's bitmap cursor at tile boundary k (k = 0..ntile)
// The root's cursor at boundary k is k T; top-down, a child's cursor is the
// parent's rank0 / rank1 there (Sec. 3.2's running counts, made random-access).
// The superblocks of all nodes, node after node, are cut into one contiguous
// part per warp; each warp scans its part, and the parts' carries are added
// to the first node of the following parts.
// ---------------------------------------------------------------------------
struct DirSmem {
    uint32_t u[256];        // first superblock of node v
    uint32_t nv[256];
    uint32_t src[256];
    uint32_t ch[256];
    uint32_t first_node[kDecWarps], last_node[kDecWarps], tail[kDecWarps], add[kDecWarps];
    uint8_t first[17];
    uint8_t maxd;
    int32_t bad;
};

__device__ inline void dir_cta(int b, const uint8_t *__restrict__ comp, const uint64_t *__restrict__ comp_off,
                               int nblk, uint8_t *__restrict__ ws, uint64_t ws_bytes, int32_t *__restrict__ status,
                               DirSmem &D) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const DecWs W = dec_ws(ws, nblk);
    const DecRegions G = dec_regions(nblk, ws);
    const uint32_t dir_bits = dec_dir_bits(ws);
    const uint32_t ntile = W.blk_ntile[b], T = W.blk_T[b];
    if (ntile <= 1 && !dec_all_dirs(ws)) return;
    // one decision for the whole CTA (every thread reaches the same barriers)
    if (__syncthreads_or(*reinterpret_cast<volatile int32_t *>(&status[b]) != PIVCO_OK)) return;
    const uint8_t *rec = comp + comp_off[b];
    const uint32_t rb = ld_le32(rec);
    const uint32_t V = (uint32_t)rec[8] | ((uint32_t)rec[9] << 8);
    const uint64_t nbase = G.dir + W.blk_dir[b], ntb = ntab_bytes(V);
    const uint8_t *nt = ws + nbase;
    const uint32_t ent = nbase + ntb <= ws_bytes ? *reinterpret_cast<const uint32_t *>(nt + 20) : 0u;
    if (nbase + ntb + 4ull * ent + 4ull * (ntile + 1) * V > ws_bytes) {
        __syncthreads();
        if (t == 0) status[b] = PIVCO_ERR_CAPACITY;
        return;
    }
    uint32_t *dirp = reinterpret_cast<uint32_t *>(ws + nbase + ntb);
    uint32_t *cur = dirp + ent;
    const uint32_t *nsrc = reinterpret_cast<const uint32_t *>(nt + kNtabHdr);
    const uint32_t *nv = reinterpret_cast<const uint32_t *>(rec + kNvOff);
    const uint64_t sbase = G.scratch + W.blk_scratch[b];
    TileSrc src;
    src.rec = rec;
    src.rec_bytes = rb;
    src.scr = ws + sbase;
    src.scr_bytes = ws_bytes > sbase ? ws_bytes - sbase : 0;
    if (t < 17) D.first[t] = nt[t];
    if (t == 17) D.maxd = nt[17];
    if (t == 0) D.bad = 0;
    for (uint32_t v = t; v < V; v += kDecThreads) {
        D.nv[v] = __ldg(nv + v);
        D.src[v] = nsrc[v];
        D.ch[v] = nsrc[V + v];
    }
    __syncthreads();
    if (warp == 0) {
        const uint32_t tot = warp_scan_loop_d((int)V, [&](int v) { return (D.nv[v] + dir_bits - 1) / dir_bits; },
                                              [&](int v, uint32_t p) { D.u[v] = p; });
        if (lane == 0 && tot != ent) D.bad = 1;
    }
    __syncthreads();
    if (D.bad) {
        if (t == 0) status[b] = PIVCO_ERR_CORRUPT;
        __syncthreads();
        return;
    }
    // phase 1: superblock popcounts scanned within each node, per part
    const uint32_t le = 0xFFFFFFFFu >> (31 - lane);
    const uint32_t g0 = (uint32_t)((uint64_t)ent * warp / kDecWarps), g1 = (uint32_t)((uint64_t)ent * (warp + 1) / kDecWarps);
    {
        uint32_t vcur = (uint32_t)find_node_d(D.u, 0, (int)V, g0), carry = 0;
        if (lane == 0) D.first_node[warp] = vcur;
        for (uint32_t base = g0; base < g1; base += 32) {
            const uint32_t cand = vcur + 1 + lane;
            uint32_t bit = 0;
            if (cand < V) {
                const uint32_t s = D.u[cand] - base;
                if (s < 32) bit = 1u << s;
            }
            const uint32_t starts = __reduce_or_sync(0xffffffffu, bit);
            const uint32_t v = vcur + __popc(starts & le);
            const uint32_t g = base + lane;
            uint32_t pc = 0;
            if (g < g1) {
                const uint32_t e0 = (g - D.u[v]) * dir_bits, nvv = D.nv[v];
                pc = tile_popc(src, D.src[v], e0, min(dir_bits, nvv - e0));
            }
            uint32_t inc = pc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            const uint32_t sl = starts & le;
            const int sa = sl ? 31 - __clz(sl) : -1;
            const uint32_t before = __shfl_sync(0xffffffffu, inc, sa > 0 ? sa - 1 : 0);
            const uint32_t ex = inc - pc - (sa > 0 ? before : 0u) + (sa < 0 ? carry : 0u);
            if (g < g1) dirp[g] = ex;
            // the last lane inside the part carries its node's count onwards
            const int last = (int)min(31u, g1 - 1 - base);
            carry = __shfl_sync(0xffffffffu, ex + pc, last);
            vcur = __shfl_sync(0xffffffffu, v, last);
        }
        if (lane == 0) { D.last_node[warp] = vcur; D.tail[warp] = carry; }
    }
    __syncthreads();
    // phase 2: ones of each part's first node in the parts before it
    if (t == 0) {
        D.add[0] = 0;
        for (int w = 1; w < kDecWarps; w++) {
            const uint32_t v0 = D.first_node[w];
            uint32_t a = 0;
            if ((uint64_t)ent * w / kDecWarps > (uint64_t)ent * (w - 1) / kDecWarps && D.last_node[w - 1] == v0)
                a = D.tail[w - 1] + (D.first_node[w - 1] == v0 ? D.add[w - 1] : 0u);
            else if ((uint64_t)ent * w / kDecWarps == (uint64_t)ent * (w - 1) / kDecWarps)
                a = D.add[w - 1];   // an empty part passes its predecessor's sum through
            D.add[w] = a;
        }
    }
    __syncthreads();
    if (D.add[warp]) {
        const uint32_t v0 = D.first_node[warp], a = D.add[warp];
        const uint32_t gend = min(g1, D.u[v0] + (D.nv[v0] + dir_bits - 1) / dir_bits);
        for (uint32_t g = g0 + lane; g < gend; g += 32) dirp[g] += a;
    }
    // boundary 0: all cursors 0; boundary ntile: n_v; the root at boundary k: k T
    for (uint32_t v = t; v < V; v += kDecThreads) { cur[v] = 0; cur[(size_t)ntile * V + v] = D.nv[v]; }
    for (uint32_t k = 1 + t; k < ntile; k += kDecThreads) cur[(size_t)k * V] = k * T;
    __syncthreads();
    // phase 3: cursors top-down, depth by depth
    int bad = 0;
    for (int d = 0; d < (int)D.maxd; d++) {
        const uint32_t f0 = D.first[d], nd = D.first[d + 1] - f0;
        for (uint32_t i = t; i < (ntile - 1) * nd; i += kDecThreads) {
            const uint32_t k = 1 + i / nd, v = f0 + i % nd;
            const uint32_t c = cur[(size_t)k * V + v], nvv = D.nv[v];
            if (c > nvv) { bad = 1; continue; }
            if (ch_flat_d(D.ch[v])) continue;   // no children below a flat node
            const uint32_t nsb = (nvv + dir_bits - 1) / dir_bits;
            uint32_t sb = c / dir_bits;
            if (sb >= nsb) sb = nsb - 1;
            const uint32_t ones = dirp[D.u[v] + sb] + tile_popc(src, D.src[v], sb * dir_bits, c - sb * dir_bits);
            const uint32_t chv = D.ch[v], c0 = chv & 0xFFFFu, c1 = chv >> 16;
            if (!(c0 & 0x8000u)) cur[(size_t)k * V + c0] = c - ones;
            if (!(c1 & 0x8000u)) cur[(size_t)k * V + c1] = ones;
        }
        __syncthreads();
    }
    bad = __syncthreads_or(bad);
    if (t == 0 && bad) status[b] = PIVCO_ERR_CORRUPT;
    __syncthreads();
}

// Warp version of the directory pass, for blocks with at most kDirWarpMax
// superblocks: one warp sweeps every node's superblocks in one flat pass
// (segmented scan per node), then finds the cursors top-down.  u / nv /
// first / maxd are the warp's scratch.
constexpr uint32_t kDirWarpMax = 8192;

// superblock count of block b's rank directory (0: the block has none: one
// tile, and no directory asked for every block; or no node table at all: a
// block that is not coded, or whose plan failed, has an empty region, and
// its record is not read)
__device__ inline uint32_t dir_entries(int b, const uint8_t *comp, const uint64_t *comp_off, int nblk,
                                       const uint8_t *ws, uint64_t ws_bytes) {
    const DecWs W = dec_ws(const_cast<uint8_t *>(ws), nblk);
    if (W.blk_ntile[b] <= 1 && !dec_all_dirs(ws)) return 0;
    const uint64_t d0 = W.blk_dir[b];
    const uint64_t d1 = b + 1 < nblk ? W.blk_dir[b + 1] : reinterpret_cast<const uint64_t *>(ws)[2];
    if (d1 <= d0) return 0;
    const DecRegions G = dec_regions(nblk, ws);
    const uint8_t *rec = comp + comp_off[b];
    const uint32_t V = (uint32_t)rec[8] | ((uint32_t)rec[9] << 8);
    const uint64_t nbase = G.dir + d0;
    return nbase + ntab_bytes(V) <= ws_bytes ? *reinterpret_cast<const uint32_t *>(ws + nbase + 20) : 0xFFFFFFFFu;
}

__device__ inline void dir_warp(int b, const uint8_t *__restrict__ comp, const uint64_t *__restrict__ comp_off,
                                int nblk, uint8_t *__restrict__ ws, uint64_t ws_bytes, int32_t *__restrict__ status,
                                uint32_t *u, uint32_t *nvs, uint8_t *first, uint8_t &maxd, uint32_t *sm,
                                uint32_t sm_words) {
    const int lane = threadIdx.x & 31;
    const DecWs W = dec_ws(ws, nblk);
    const DecRegions G = dec_regions(nblk, ws);
    const uint32_t dir_bits = dec_dir_bits(ws);
    const uint32_t ntile = W.blk_ntile[b], T = W.blk_T[b];
    if ((ntile <= 1 && !dec_all_dirs(ws)) || *reinterpret_cast<volatile int32_t *>(&status[b]) != PIVCO_OK) return;
    const uint8_t *rec = comp + comp_off[b];
    const uint32_t rb = ld_le32(rec);
    const uint32_t V = (uint32_t)rec[8] | ((uint32_t)rec[9] << 8);
    const uint64_t nbase = G.dir + W.blk_dir[b], ntb = ntab_bytes(V);
    const uint8_t *nt = ws + nbase;
    const uint32_t ent = nbase + ntb <= ws_bytes ? *reinterpret_cast<const uint32_t *>(nt + 20) : 0u;
    if (nbase + ntb + 4ull * ent + 4ull * (ntile + 1) * V > ws_bytes) {
        if (lane == 0) status[b] = PIVCO_ERR_CAPACITY;
        return;
    }
    uint32_t *dirp = reinterpret_cast<uint32_t *>(ws + nbase + ntb);
    uint32_t *cur = dirp + ent;
    const uint32_t *gsrc = reinterpret_cast<const uint32_t *>(nt + kNtabHdr);
    const uint32_t *nv = reinterpret_cast<const uint32_t *>(rec + kNvOff);
    const uint64_t sbase = G.scratch + W.blk_scratch[b];
    TileSrc src;
    src.rec = rec;
    src.rec_bytes = rb;
    src.scr = ws + sbase;
    src.scr_bytes = ws_bytes > sbase ? ws_bytes - sbase : 0;
    if (lane < 17) first[lane] = nt[lane];
    if (lane == 17) maxd = nt[17];
    // the nodes' bitmap addresses and children in shared memory (sm[0..512),
    // sm_words >= 512); the tile cursors too (sm[512..)) when they fit,
    // copied out at the end
    uint32_t *nsrc = sm, *nch = sm + 256;
    const bool cur_sm = (uint64_t)(ntile + 1) * V + 512 <= sm_words;
    const uint32_t tot = warp_scan_loop_d((int)V, [&](int v) { return (__ldg(nv + v) + dir_bits - 1) / dir_bits; },
                                          [&](int v, uint32_t p) {
                                              u[v] = p;
                                              nvs[v] = __ldg(nv + v);
                                              nsrc[v] = gsrc[v];
                                              nch[v] = gsrc[V + v];
                                          });
    __syncwarp();
    if (tot != ent) {
        if (lane == 0) status[b] = PIVCO_ERR_CORRUPT;
        return;
    }
    const uint32_t le = 0xFFFFFFFFu >> (31 - lane);
    uint32_t vcur = 0, carry = 0;
    // four windows of 32 superblocks per step: their nodes first (shared
    // memory only), then all their bitmap loads, then the scans
    constexpr int kU = 4;
    for (uint32_t base = 0; base < ent; base += 32 * kU) {
        uint32_t vv[kU], st[kU], pc[kU];
#pragma unroll
        for (int r = 0; r < kU; r++) {
            const uint32_t cand = vcur + 1 + lane, bb = base + 32 * r;
            uint32_t bit = 0;
            if (cand < V) {
                const uint32_t sd = u[cand] - bb;
                if (sd < 32) bit = 1u << sd;
            }
            st[r] = __reduce_or_sync(0xffffffffu, bit);
            vv[r] = vcur + __popc(st[r] & le);
            vcur = __shfl_sync(0xffffffffu, vv[r], 31);
        }
#pragma unroll
        for (int r = 0; r < kU; r++) {
            const uint32_t g = base + 32 * r + lane;
            pc[r] = 0;
            if (g < ent) {
                const uint32_t v = vv[r], e0 = (g - u[v]) * dir_bits;
                pc[r] = tile_popc(src, nsrc[v], e0, min(dir_bits, nvs[v] - e0));
            }
        }
#pragma unroll
        for (int r = 0; r < kU; r++) {
            const uint32_t g = base + 32 * r + lane;
            uint32_t inc = pc[r];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            const uint32_t sl = st[r] & le;
            const int sa = sl ? 31 - __clz(sl) : -1;
            const uint32_t before = __shfl_sync(0xffffffffu, inc, sa > 0 ? sa - 1 : 0);
            const uint32_t ex = inc - pc[r] - (sa > 0 ? before : 0u) + (sa < 0 ? carry : 0u);
            if (g < ent) dirp[g] = ex;
            carry = __shfl_sync(0xffffffffu, ex + pc[r], 31);
        }
    }
    uint32_t *cw = cur_sm ? sm + 512 : cur;
    for (uint32_t v = lane; v < V; v += 32) { cw[v] = 0; cw[(size_t)ntile * V + v] = nvs[v]; }
    for (uint32_t k = 1 + lane; k < ntile; k += 32) cw[(size_t)k * V] = k * T;
    __syncwarp();
    int bad = 0;
    for (int d = 0; d < (int)maxd; d++) {
        const uint32_t f0 = first[d], nd = first[d + 1] - f0;
        for (uint32_t i = lane; i < (ntile - 1) * nd; i += 32) {
            const uint32_t k = 1 + i / nd, v = f0 + i % nd;
            const uint32_t c = cw[(size_t)k * V + v], nvv = nvs[v];
            if (c > nvv) { bad = 1; continue; }
            if (ch_flat_d(nch[v])) continue;   // no children below a flat node
            const uint32_t nsb = (nvv + dir_bits - 1) / dir_bits;
            uint32_t sb = c / dir_bits;
            if (sb >= nsb) sb = nsb - 1;
            const uint32_t ones = dirp[u[v] + sb] + tile_popc(src, nsrc[v], sb * dir_bits, c - sb * dir_bits);
            const uint32_t chv = nch[v], c0 = chv & 0xFFFFu, c1 = chv >> 16;
            if (!(c0 & 0x8000u)) cw[(size_t)k * V + c0] = c - ones;
            if (!(c1 & 0x8000u)) cw[(size_t)k * V + c1] = ones;
        }
        __syncwarp();
    }
    if (cur_sm)
        for (uint32_t i = lane; i < (ntile + 1) * V; i += 32) cur[i] = cw[i];
    if (__any_sync(0xffffffffu, bad) && lane == 0) status[b] = PIVCO_ERR_CORRUPT;
    __syncwarp();
}

struct DirWarpSmem {
    uint32_t u[256], nv[256], sm[512];
    uint8_t first[17];
    uint8_t maxd;
    uint8_t pad[14];
};

struct TileSmem {
    uint32_t sel[256];
    CtaTile tile;
};

// Plain tile pass: every CTA takes tiles by ticket (workspace header word 12).
// Plain directory pass: CTAs take the blocks with many superblocks, then
// every warp takes the blocks with few.
__global__ void __launch_bounds__(kDecThreads, 2) decode_dir_kernel(const uint8_t *__restrict__ comp,
                                                                    const uint64_t *__restrict__ comp_off, int nblk,
                                                                    uint8_t *__restrict__ ws, uint64_t ws_bytes,
                                                                    int32_t *__restrict__ status) {
    __shared__ DirSmem D;
    __shared__ DirWarpSmem DW[kDecWarps];
    if (abandoned_batch(ws, status, nblk)) return;
    for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
        const uint32_t e = dir_entries(b, comp, comp_off, nblk, ws, ws_bytes);
        if (e > kDirWarpMax) dir_cta(b, comp, comp_off, nblk, ws, ws_bytes, status, D);
    }
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * kDecWarps + warp, nw = gridDim.x * kDecWarps;
    DirWarpSmem &M = DW[warp];
    for (int b = gw; b < nblk; b += nw) {
        const uint32_t e = dir_entries(b, comp, comp_off, nblk, ws, ws_bytes);
        if (e && e <= kDirWarpMax)
            dir_warp(b, comp, comp_off, nblk, ws, ws_bytes, status, M.u, M.nv, M.first, M.maxd, M.sm, 512);
    }
}

__global__ void __launch_bounds__(kDecThreads, kTileCtas) decode_kernel(const uint8_t *__restrict__ comp,
                                                                        const uint64_t *__restrict__ comp_off,
                                                                        int nblk, uint8_t *__restrict__ out,
                                                                        const uint64_t *__restrict__ out_off,
                                                                        uint8_t *__restrict__ ws, uint64_t ws_bytes,
                                                                        int32_t *__restrict__ status) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    TileSmem &S = *reinterpret_cast<TileSmem *>(smem_raw);
    __shared__ uint32_t s_it;
    if (abandoned_batch(ws, status, nblk)) return;
    sel_init(S.sel);
    uint32_t *hdr = reinterpret_cast<uint32_t *>(ws);
    const uint32_t total_tiles = hdr[6];
    for (;;) {
        if (threadIdx.x == 0) s_it = atomicAdd(&hdr[12], 1u);
        __syncthreads();
        const uint32_t it = s_it;
        __syncthreads();
        if (it >= total_tiles) break;
        cta_tile(it, comp, comp_off, nblk, out, out_off, ws, ws_bytes, status, S.tile, S.sel);
    }
}

// ---------------------------------------------------------------------------
// Batched decode: one persistent launch over a work queue keyed by
// (block, stage).  Every item is taken by a whole CTA, in queue order:
//   plans      4 blocks per item, one warp each (ticket order = block order,
//              as the plan's look-back needs)
//   ANS        4 segments per item, one warp each
//   directory  8 blocks per item: each warp builds its block's directory if
//              it has few superblocks, then the whole CTA builds those of the
//              blocks with many, one after another
//   tiles      one tile per item (cta_tile)
// An item only waits (bounded) on items earlier in the queue: the ANS and
// later items on all plans; a directory on its block's ANS segments; a tile
// on its block's ANS segments and directory.  The CTAs that took those items
// are running, so every wait ends.
// ---------------------------------------------------------------------------
__device__ inline bool wait_geq(const uint32_t *p, uint32_t want, uint64_t limit_ns) {
    if (*reinterpret_cast<const volatile uint32_t *>(p) >= want) { __threadfence(); return true; }
    const uint64_t t0 = globaltimer_ns();
    unsigned ns = 64;
    while (*reinterpret_cast<const volatile uint32_t *>(p) < want) {
        if (globaltimer_ns() - t0 > limit_ns) return false;
        __nanosleep(ns);
        if (ns < 2048) ns <<= 1;
    }
    __threadfence();
    return true;
}

constexpr int kPlanWarps = 4;   // warps per plan or ANS item (their shared memory bounds the CTA's)
struct PlanAnsSmem {
    WarpRec R[kPlanWarps];
    PlanScratch Q[kPlanWarps];
    AnsSm T[kPlanWarps];
};
struct DirAllSmem {
    DirSmem dir;
    DirWarpSmem dw[kDecWarps];
};
union BatchUnion {
    PlanAnsSmem pa;
    DirAllSmem d;
    CtaTile tile;
};
struct BatchSmem {
    uint32_t sel[256];
    BatchUnion u;
    int32_t blk, ok;
    uint32_t pad[2];
};
static_assert(sizeof(PlanAnsSmem) <= sizeof(CtaTile), "plans fit the tiles' shared memory");
// kTileCtas CTAs per SM: dynamic + static shared memory + 1 KiB reserved each, of 228 KiB
static_assert(kTileCtas * (sizeof(BatchSmem) + 128 + 1024) <= 228 * 1024, "tile CTAs per SM");

// One request's (batch's) queue: where its records, output and workspace are.
struct BatchQueue {
    const uint8_t *comp;
    const uint64_t *comp_off;
    uint8_t *out;
    const uint64_t *out_off;
    uint8_t *ws;
    uint64_t ws_bytes;
    int32_t *status;
    int nblk;
};

// the wait bound of a batch's queue (workspace header)
__device__ inline uint64_t wait_bound(const BatchQueue &q) { return reinterpret_cast<const uint64_t *>(q.ws)[7]; }

__device__ inline uint32_t batch_nplan(int nblk) { return (uint32_t)((nblk + kPlanWarps - 1) / kPlanWarps); }
__device__ inline uint32_t batch_ndir(int nblk) { return (uint32_t)((nblk + kDecWarps - 1) / kDecWarps); }

// Items of a batch's queue once all plans are done (header written by the last plan):
// plans, first tiles (one per block), ANS segments, directories, tiles.
__device__ inline uint32_t batch_items_total(const BatchQueue &q) {
    const uint32_t *hdr = reinterpret_cast<const uint32_t *>(q.ws);
    return batch_nplan(q.nblk) + (uint32_t)q.nblk + (hdr[2] + kPlanWarps - 1) / kPlanWarps + batch_ndir(q.nblk) +
           hdr[6];
}

enum : int { kItemDone = 0, kItemNone = 1, kItemStop = 2 };

// Runs item `item` of the queue with the whole CTA.  kItemDone: processed;
// kItemNone: past the last item; kItemStop: the wait for the plans expired
// or the plans could not place the batch (every block is marked), the CTA
// must stop.
__device__ inline int batch_item(const BatchQueue &q, uint32_t item, BatchSmem &B, const AnsTables &A, int &last_b,
                                 bool &last_ok) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int nblk = q.nblk;
    uint32_t *hdr = reinterpret_cast<uint32_t *>(q.ws);
    const DecWs W = dec_ws(q.ws, nblk);
    const uint32_t nplan = batch_nplan(nblk);
    if (item < nplan) {
        // ---- plans ----
        const int b = (int)(item * kPlanWarps + warp);
        if (warp < kPlanWarps && b < nblk) {
            plan_block(b, q.comp, q.comp_off, nblk, q.ws, q.ws_bytes, q.status, B.u.pa.R[warp], B.u.pa.Q[warp]);
            // a CTA that has given up on the queue (below) may have marked
            // the blocks before this plan wrote its status: re-mark it, so a
            // block whose later items may never run does not read as done
            __threadfence();
            if (lane == 0 && *reinterpret_cast<volatile uint32_t *>(&hdr[13]) &&
                *reinterpret_cast<volatile int32_t *>(&q.status[b]) == PIVCO_OK)
                q.status[b] = PIVCO_ERR_TIMEOUT;
        }
        __syncthreads();
        if (t == 0) { __threadfence(); atomicAdd(&hdr[10], 1u); }
        return kItemDone;
    }
    if (item < nplan + (uint32_t)nblk) {
        // ---- first tiles: block b's only tile as soon as its own plan is
        // complete, when it needs no ANS segment and no directory (its node
        // table and offsets are then all it reads); other blocks' tiles come
        // after the directories ----
        const int b = (int)(item - nplan);
        if (t == 0) {
            const int okw = wait_geq(&W.plan_done[b], 1u, wait_bound(q));
            if (!okw) q.status[b] = PIVCO_ERR_TIMEOUT;
            B.ok = okw ? (int)*reinterpret_cast<volatile uint32_t *>(&W.plan_done[b]) : 0;
        }
        __syncthreads();
        const int pd = B.ok;
        __syncthreads();
        if (pd & 2) cta_tile(W.blk_tile[b], q.comp, q.comp_off, nblk, q.out, q.out_off, q.ws, q.ws_bytes, q.status,
                             B.u.tile, B.sel, b);
        __syncthreads();
        return kItemDone;
    }
    // everything after the plans and first tiles needs all plans
    int ok = 1;
    if (t == 0) {
        ok = wait_geq(&hdr[10], nplan, wait_bound(q));
        // the last plan could not place the batch: nothing after the plans runs
        if (ok && *reinterpret_cast<volatile uint32_t *>(&hdr[13])) ok = 0;
    }
    if (__syncthreads_or(!ok)) {
        // this CTA leaves the queue: every block not yet failed is marked, as
        // its items may now never run (the flag makes plans still running
        // mark theirs, the fences order the flag against their status writes)
        if (t == 0) {
            atomicExch(&hdr[13], 1u);
            __threadfence();
            for (int b = 0; b < nblk; b++)
                if (*reinterpret_cast<volatile int32_t *>(&q.status[b]) == PIVCO_OK) q.status[b] = PIVCO_ERR_TIMEOUT;
        }
        __syncthreads();
        return kItemStop;
    }
    const uint32_t total_segs = hdr[2];
    const uint32_t nseg_items = (total_segs + kPlanWarps - 1) / kPlanWarps;
    uint32_t it = item - nplan - (uint32_t)nblk;
    if (it < nseg_items) {
        // ---- ANS segments ----
        const uint32_t g = it * kPlanWarps + warp;
        if (warp < kPlanWarps && g < total_segs) {
            const int b = ans_item(g, q.comp, q.comp_off, nblk, q.ws, q.ws_bytes, q.status, A, B.u.pa.R[warp],
                                   B.u.pa.T[warp], last_b, last_ok);
            if (lane == 0) { __threadfence(); atomicAdd(&W.segs_done[b], 1u); }
        }
        __syncthreads();
        last_b = -1;   // the cached record may be overwritten by a later item
        return kItemDone;
    }
    it -= nseg_items;
    const uint32_t ndir = batch_ndir(nblk);
    if (it < ndir) {
        // ---- directories of blocks 8 it .. 8 it + 7 ----
        const int bw = (int)(it * kDecWarps + warp);
        const uint32_t e = bw < nblk ? dir_entries(bw, q.comp, q.comp_off, nblk, q.ws, q.ws_bytes) : 0u;
        if (e && e <= kDirWarpMax) {
            const uint32_t nsegs = (bw + 1 < nblk ? W.blk_seg[bw + 1] : total_segs) - W.blk_seg[bw];
            int okw = 1;
            if (lane == 0) {
                okw = wait_geq(&W.segs_done[bw], nsegs, wait_bound(q));
                if (!okw) q.status[bw] = PIVCO_ERR_TIMEOUT;
            }
            if (__shfl_sync(0xffffffffu, okw, 0)) {
                DirWarpSmem &M = B.u.d.dw[warp];
                dir_warp(bw, q.comp, q.comp_off, nblk, q.ws, q.ws_bytes, q.status, M.u, M.nv, M.first, M.maxd, M.sm,
                         512);
            }
            __syncwarp();
            if (lane == 0) { __threadfence(); atomicExch(&W.dir_done[bw], 1u); }
        }
        const bool big = e > kDirWarpMax;
        for (int w = 0; w < kDecWarps; w++) {
            if (!__syncthreads_or(warp == w && big)) continue;
            const int b = (int)(it * kDecWarps + w);
            const uint32_t nsegs = (b + 1 < nblk ? W.blk_seg[b + 1] : total_segs) - W.blk_seg[b];
            int okw = 1;
            if (t == 0) okw = wait_geq(&W.segs_done[b], nsegs, wait_bound(q));
            if (__syncthreads_or(!okw)) {
                if (t == 0) q.status[b] = PIVCO_ERR_TIMEOUT;
            } else {
                dir_cta(b, q.comp, q.comp_off, nblk, q.ws, q.ws_bytes, q.status, B.u.d.dir);
            }
            __syncthreads();
            if (t == 0) { __threadfence(); atomicExch(&W.dir_done[b], 1u); }
        }
        __syncthreads();
        return kItemDone;
    }
    it -= ndir;
    if (it >= hdr[6]) return kItemNone;
    // ---- tile it: after its block's ANS segments and directory (a tile
    // decoded among the first tiles is skipped) ----
    if (warp == 0) {
        const int b = find_block_warp(W.blk_tile, nblk, it, (int)((uint64_t)it * (uint32_t)nblk / max(hdr[6], 1u)));
        if (lane == 0) {
            int okw = 1;
            if (W.plan_done[b] & 2u) {
                okw = 0;
            } else {
                const uint32_t nsegs = (b + 1 < nblk ? W.blk_seg[b + 1] : total_segs) - W.blk_seg[b];
                okw = wait_geq(&W.segs_done[b], nsegs, wait_bound(q));
                if (okw && W.blk_ntile[b] > 1) okw = wait_geq(&W.dir_done[b], 1u, wait_bound(q));
                if (!okw) q.status[b] = PIVCO_ERR_TIMEOUT;
            }
            B.blk = b;
            B.ok = okw;
        }
    }
    __syncthreads();
    const int b = B.blk, okw = B.ok;
    __syncthreads();
    if (okw) cta_tile(it, q.comp, q.comp_off, nblk, q.out, q.out_off, q.ws, q.ws_bytes, q.status, B.u.tile, B.sel, b);
    __syncthreads();
    return kItemDone;
}

__global__ void __launch_bounds__(kDecThreads, kTileCtas) decode_batch_kernel(const uint8_t *__restrict__ comp,
                                                                              const uint64_t *__restrict__ comp_off,
                                                                              int nblk, uint8_t *__restrict__ out,
                                                                              const uint64_t *__restrict__ out_off,
                                                                              uint8_t *__restrict__ ws, uint64_t ws_bytes,
                                                                              int32_t *__restrict__ status,
                                                                              const __grid_constant__ AnsTables A) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    BatchSmem &B = *reinterpret_cast<BatchSmem *>(smem_raw);
    __shared__ uint32_t s_item;
    const BatchQueue q{comp, comp_off, out, out_off, ws, ws_bytes, status, nblk};
    uint32_t *hdr = reinterpret_cast<uint32_t *>(ws);
    sel_init(B.sel);
    int last_b = -1;
    bool last_ok = false;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&hdr[9], 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        const int r = batch_item(q, item, B, A, last_b, last_ok);
        if (r != kItemDone) return;
    }
}

// ---------------------------------------------------------------------------
// Serving: a device-resident request loop over the batch queue items.
// Requests are published by the host in sequence order into a ring (entry r
// at ring[r % kServeRing], the count in flags->tail, host memory mapped into
// the device).  Every CTA repeatedly takes the next item of request ctl->cur;
// when that request has no items left it moves ctl->cur on, so the items of
// consecutive requests overlap on the device and a request published while
// others run is picked up by the first CTA that frees up.  The CTA that
// finishes a request's last item writes its worst block status and then its
// done flag into mapped host memory.  A CTA leaves when it has found nothing
// to do for idle_ns, when its launch has lived life_ns (checked between
// items), or on flags->stop; the host then launches the loop again if work
// remains.  A request's ring entry and memory are reused only after a launch
// that started later has ended with ctl->cur past it, so no CTA can still
// touch them.
// ---------------------------------------------------------------------------
__device__ inline uint32_t ld_acquire_sys_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ inline void st_release_sys_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Counts one finished item of request r; the item that completes the
// request's queue writes its worst block status, then its done flag.
__device__ inline void serve_item_done(const BatchQueue &q, uint32_t r, ServeFlags *flags) {
    uint32_t *hdr = reinterpret_cast<uint32_t *>(q.ws);
    __threadfence();
    const uint32_t n = atomicAdd(&hdr[11], 1u) + 1;
    if (*reinterpret_cast<volatile uint32_t *>(&hdr[10]) < batch_nplan(q.nblk)) return;   // totals not known yet
    __threadfence();
    if (n != batch_items_total(q)) return;
    int32_t worst = PIVCO_OK;
    for (int b = 0; b < q.nblk && worst == PIVCO_OK; b++) worst = *reinterpret_cast<volatile int32_t *>(&q.status[b]);
    flags->worst[r % kServeRing] = worst;
    __threadfence_system();
    st_release_sys_u32(&flags->done[r % kServeRing], r + 1);
}

__global__ void __launch_bounds__(kDecThreads, kTileCtas) serve_loop_kernel(ServeCtl *__restrict__ ctl,
                                                                            const ServeDesc *__restrict__ ring,
                                                                            ServeFlags *flags, uint64_t idle_ns,
                                                                            uint64_t life_ns,
                                                                            const __grid_constant__ AnsTables A) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    BatchSmem &B = *reinterpret_cast<BatchSmem *>(smem_raw);
    __shared__ ServeDesc D;
    __shared__ uint32_t s_cmd, s_item, s_r;
    const int t = threadIdx.x;
    sel_init(B.sel);
    int last_b = -1;
    bool last_ok = false;
    uint32_t have = 0xFFFFFFFFu;   // request whose ring entry is in D (thread 0's view)
    uint32_t used = 0xFFFFFFFFu;   // request of the last item (all threads)
    const uint64_t t0 = globaltimer_ns();
    uint64_t idle_since = 0;
    for (;;) {
        if (t == 0) {
            uint32_t cmd = 0;   // 0 work, 1 nothing yet, 2 leave
            const uint64_t now = globaltimer_ns();
            const uint32_t r = *reinterpret_cast<volatile uint32_t *>(&ctl->cur);
            const uint32_t tail = ld_acquire_sys_u32(&flags->tail);
            if (ld_acquire_sys_u32(&flags->stop) || now - t0 > life_ns) {
                cmd = 2;
            } else if (r >= tail) {
                if (!idle_since) idle_since = now;
                cmd = now - idle_since > idle_ns ? 2u : 1u;
            } else {
                idle_since = 0;
                if (r != have) {
                    D = ring[r % kServeRing];
                    if (D.seq != r) cmd = 1;   // not written yet (cannot happen once published)
                    else have = r;
                }
                if (cmd == 0) {
                    s_item = atomicAdd(&reinterpret_cast<uint32_t *>(D.ws)[9], 1u);
                    s_r = r;
                }
            }
            s_cmd = cmd;
        }
        __syncthreads();
        const uint32_t cmd = s_cmd, item = s_item, r = s_r;
        __syncthreads();
        if (cmd == 2) return;
        if (cmd == 1) {
            if (t == 0) __nanosleep(1000);
            continue;
        }
        if (r != used) { last_b = -1; used = r; }
        const BatchQueue q{D.comp, D.comp_off, D.out, D.out_off, D.ws, D.ws_bytes, D.status, D.nblk};
        const int res = batch_item(q, item, B, A, last_b, last_ok);
        if (res != kItemNone) {
            if (t == 0) serve_item_done(q, r, flags);
            if (res == kItemStop) return;
            __syncthreads();
            continue;
        }
        // the request has no items left: move on to the next one
        if (t == 0) atomicCAS(&ctl->cur, r, r + 1);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Random access (NEXT to the bottom-up merge): the symbol at one position of
// one block by a top-down walk, Sec. 2.1's traversal made random-access the
// way a wavelet tree answers access (Sec. 7.2): at node v the position's bit
// picks the child, and the position becomes its rank among the positions of
// that bit, rank1(B_v, x) = the directory's ones before x's superblock plus
// the popcount of the superblock's bits before x.  The workspace comes from
// the plan with a directory for every coded block, the ANS pass and the
// directory pass (pivco_access_prepare).  One thread per query.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) access_kernel(const uint8_t *__restrict__ comp,
                                                     const uint64_t *__restrict__ comp_off, int nblk,
                                                     const uint32_t *__restrict__ qblk, const uint32_t *__restrict__ qpos,
                                                     int nq, uint8_t *__restrict__ sym, int32_t *__restrict__ qstatus,
                                                     const uint8_t *__restrict__ ws, uint64_t ws_bytes,
                                                     const int32_t *__restrict__ status) {
    const DecWs W = dec_ws(const_cast<uint8_t *>(ws), nblk);
    const DecRegions G = dec_regions(nblk, ws);
    const uint32_t dir_bits = dec_dir_bits(ws);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        const uint32_t b = qblk[q], x0 = qpos[q];
        uint8_t out = 0;
        int32_t st = PIVCO_OK;
        if (b >= (uint32_t)nblk) {
            st = PIVCO_ERR_INVALID_ARG;
        } else if ((st = status[b]) == PIVCO_OK) {
            const uint8_t *rec = comp + comp_off[b];   // validated by the plan
            const uint32_t n = ld_le32(rec + 4), kind = rec[10];
            if (x0 >= n) {
                st = PIVCO_ERR_INVALID_ARG;
            } else if (kind == 1) {
                out = rec[11];
            } else {
                const uint32_t rb = ld_le32(rec), V = (uint32_t)rec[8] | ((uint32_t)rec[9] << 8);
                const uint64_t nbase = G.dir + W.blk_dir[b], ntb = ntab_bytes(V);
                const uint8_t *nt = ws + nbase;
                const uint32_t ent = nbase + ntb <= ws_bytes ? *reinterpret_cast<const uint32_t *>(nt + 20) : 0u;
                if (!ent || nbase + ntb + 4ull * ent > ws_bytes) {
                    st = PIVCO_ERR_INVALID_ARG;   // no directory: the workspace was not prepared for access
                } else {
                    const uint32_t *nsrc = reinterpret_cast<const uint32_t *>(nt + kNtabHdr);
                    const uint32_t *nch = nsrc + V, *nu = nsrc + 2 * V;
                    const uint32_t *dirp = reinterpret_cast<const uint32_t *>(nt + ntb);
                    const uint32_t *nv = reinterpret_cast<const uint32_t *>(rec + kNvOff);
                    const uint64_t sbase = G.scratch + W.blk_scratch[b];
                    TileSrc src;
                    src.rec = rec;
                    src.rec_bytes = rb;
                    src.scr = ws + sbase;
                    src.scr_bytes = ws_bytes > sbase ? ws_bytes - sbase : 0;
                    uint32_t v = 0, x = x0;
                    st = PIVCO_ERR_CORRUPT;   // unless a leaf is reached within the code-length limit
                    for (int d = 0; d <= (int)kMaxLen && v < V; d++) {
                        const uint32_t nvv = __ldg(nv + v);
                        if (x >= nvv) break;
                        if (const uint32_t D = ch_flat_d(nch[v])) {
                            // a flat node: the D-bit index of the position, then its symbol
                            const uint32_t xi = tile_bits(src, nsrc[v], x * D) & ((1u << D) - 1u);
                            out = nt[kNtabHdr + 12 * V + (nch[v] & 0xFFu) + xi];
                            st = PIVCO_OK;
                            break;
                        }
                        const uint32_t bit = tile_bits(src, nsrc[v], x) & 1u;
                        const uint32_t sb = x / dir_bits;
                        const uint32_t ones = dirp[nu[v] + sb] + tile_popc(src, nsrc[v], sb * dir_bits, x - sb * dir_bits);
                        const uint32_t c = (nch[v] >> (16 * bit)) & 0xFFFFu;
                        x = bit ? ones : x - ones;
                        if (c & 0x8000u) {
                            out = (uint8_t)c;
                            st = PIVCO_OK;
                            break;
                        }
                        v = c;
                    }
                }
            }
        }
        sym[q] = out;
        if (qstatus) qstatus[q] = st;
    }
}

cudaError_t launch_access_prepare(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *ws, size_t ws_bytes,
                                  int32_t *status, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    cudaError_t e = launch_decode_plan(comp, comp_off, nblk, ws, ws_bytes, status, st, true);
    if (e == cudaSuccess) e = launch_ans_decode_planned(comp, comp_off, nblk, ws, ws_bytes, status, st);
    if (e == cudaSuccess) e = launch_decode_dir(comp, comp_off, nblk, ws, ws_bytes, status, st);
    return e;
}

cudaError_t launch_access(const uint8_t *comp, const uint64_t *comp_off, int nblk, const uint32_t *qblk,
                          const uint32_t *qpos, int nq, uint8_t *sym, int32_t *qstatus, const uint8_t *ws,
                          size_t ws_bytes, const int32_t *status, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = min(div_up(nq, 256), sms * 8);
    access_kernel<<<grid, 256, 0, st>>>(comp, comp_off, nblk, qblk, qpos, nq, sym, qstatus, ws, ws_bytes, status);
    count_launches(1);
    return cudaGetLastError();
}

// Host: an upper bound, from host copies of the records, of the workspace the
// decode of these blocks needs under tuning `tu` (never below what the plan
// computes for valid records): the scratch of every ANS-coded node exactly,
// and rank directories plus tile cursors for the most tiles the plan can
// choose (a level of a valid record holds at most n symbols).
size_t decode_ws_bound(const uint8_t *comp, const uint64_t *comp_off, int nblk, const DecTuning &tu) {
    uint64_t dir = 0, scratch = 0;
    // the shortest tile the plan can choose: a level of at most 128 nodes and
    // at most n symbols in a buffer, 20 % headroom, a multiple of 128
    const uint64_t t_fit = ((uint64_t)(kLvlBuf - 4 * 128 - 32) / 5 * 4) & ~127ull;
    uint64_t t_min = tu.tile_max < t_fit ? tu.tile_max : t_fit;
    if (t_min < 128) t_min = 128;
    for (int b = 0; b < nblk; b++) {
        const uint8_t *rec = comp + comp_off[b];
        const uint64_t avail = comp_off[b + 1] > comp_off[b] ? comp_off[b + 1] - comp_off[b] : 0;
        if (avail < kNvOff || rec[10] != 2) continue;
        const uint32_t n = (uint32_t)rec[4] | ((uint32_t)rec[5] << 8) | ((uint32_t)rec[6] << 16) | ((uint32_t)rec[7] << 24);
        const uint32_t V = (uint32_t)rec[8] | ((uint32_t)rec[9] << 8);
        if (V < 1 || V > 255 || kNvOff + 5 * V > avail) continue;
        uint64_t ent = 0;
        for (uint32_t v = 0; v < V; v++) {
            const uint8_t *p = rec + kNvOff + 4 * v;
            const uint32_t nv = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
            const uint8_t m = rec[kNvOff + 4 * V + v];
            ent += (nv + (uint64_t)tu.dir_bits - 1) / tu.dir_bits;
            if (mark_ans(m)) scratch += scratch_stride((nv + 7) / 8);
        }
        uint64_t ntile = ((uint64_t)n + t_min - 1) / t_min;
        if (ntile > (1u << 21)) ntile = 1u << 21;
        dir += ntab_bytes(V) + ((4 * ent + 4 * (ntile + 1) * V + 15) & ~(uint64_t)15);
    }
    return ((decode_ws_fixed_bytes(nblk) + dir + 255) & ~(size_t)255) + scratch + 256;
}

// Host: an upper bound of the same workspace from the blocks' sizes alone
// (no record is read): every block taken as 255 nodes carrying at most 15
// bits per symbol, all of them ANS-coded.  For callers that place records
// they have not seen yet.
size_t decode_ws_size_bound(const uint64_t *blk_off, int nblk, const DecTuning &tu) {
    const uint64_t t_fit = ((uint64_t)(kLvlBuf - 4 * 128 - 32) / 5 * 4) & ~127ull;
    uint64_t t_min = tu.tile_max < t_fit ? tu.tile_max : t_fit;
    if (t_min < 128) t_min = 128;
    uint64_t dir = 0, scratch = 0;
    for (int b = 0; b < nblk; b++) {
        const uint64_t n = blk_off[b + 1] - blk_off[b];
        if (n < 2) continue;   // empty and one-symbol blocks have no nodes
        const uint64_t ent = 15 * n / tu.dir_bits + 255;
        uint64_t ntile = (n + t_min - 1) / t_min;
        if (ntile > (1u << 21)) ntile = 1u << 21;
        dir += ntab_bytes(255) + ((4 * ent + 4 * (ntile + 1) * 255 + 15) & ~(uint64_t)15);
        scratch += 15 * n / 8 + 255ull * 48;
    }
    return ((decode_ws_fixed_bytes(nblk) + dir + 255) & ~(size_t)255) + scratch + 256;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static int merge_grid(const void *fn, int smem) {
    int dev = 0, sms = 148, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kDecThreads, smem);
    const uint32_t want = current_tuning().ctas_per_sm;
    if (want && (int)want < occ) occ = (int)want;
    if (occ < 1) occ = 1;
    return sms * occ;
}

cudaError_t launch_decode_dir(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *ws, size_t ws_bytes,
                              int32_t *status, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = nblk < sms * 4 ? nblk : sms * 4;
    decode_dir_kernel<<<grid, kDecThreads, 0, st>>>(comp, comp_off, nblk, ws, ws_bytes, status);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_decode(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *out,
                          const uint64_t *out_off, uint8_t *ws, size_t ws_bytes, int32_t *status, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    cudaError_t e = launch_decode_plan(comp, comp_off, nblk, ws, ws_bytes, status, st);
    if (e != cudaSuccess) return e;
    e = launch_ans_decode_planned(comp, comp_off, nblk, ws, ws_bytes, status, st);
    if (e != cudaSuccess) return e;
    return launch_decode_merge(comp, comp_off, nblk, out, out_off, ws, ws_bytes, status, st);
}

cudaError_t launch_decode_merge(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *out,
                                const uint64_t *out_off, uint8_t *ws, size_t ws_bytes, int32_t *status,
                                cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    cudaError_t e = launch_decode_dir(comp, comp_off, nblk, ws, ws_bytes, status, st);
    if (e != cudaSuccess) return e;
    const int smem = (int)sizeof(TileSmem);
    e = cudaFuncSetAttribute(decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    decode_kernel<<<merge_grid((const void *)decode_kernel, smem), kDecThreads, smem, st>>>(
        comp, comp_off, nblk, out, out_off, ws, ws_bytes, status);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_serve_loop(ServeCtl *ctl, const ServeDesc *ring, ServeFlags *flags, uint64_t idle_ns,
                              uint64_t life_ns, cudaStream_t st) {
    const int smem = (int)sizeof(BatchSmem);
    cudaError_t e = cudaFuncSetAttribute(serve_loop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    serve_loop_kernel<<<merge_grid((const void *)serve_loop_kernel, smem), kDecThreads, smem, st>>>(
        ctl, ring, flags, idle_ns, life_ns, host_ans_tables());
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_decode_batch(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *out,
                                const uint64_t *out_off, uint8_t *ws, size_t ws_bytes, int32_t *status,
                                cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    const DecTuning tu = current_tuning();
    dec_ws_init_kernel<<<min(1024, div_up(nblk, 256)), 256, 0, st>>>(ws, nblk, tu.dir_bits, tu.tile_max,
                                                                      wait_limit_ns());
    const int smem = (int)sizeof(BatchSmem);
    cudaError_t e = cudaFuncSetAttribute(decode_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    decode_batch_kernel<<<merge_grid((const void *)decode_batch_kernel, smem), kDecThreads, smem, st>>>(
        comp, comp_off, nblk, out, out_off, ws, ws_bytes, status, host_ans_tables());
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace pv

namespace pv {
// dynamic shared-memory limits of the decode kernels (set before any capture)
cudaError_t prepare_decode_kernels() {
    cudaError_t e = cudaFuncSetAttribute(decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(decode_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BatchSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(serve_loop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BatchSmem));
    return e;
}
}  // namespace pv
