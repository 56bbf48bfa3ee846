// Internal definitions shared by the library's kernels (not part of the ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/pivco.h"

namespace pv {

// ---------------------------------------------------------------------------
// Record format constants (App. D, adapted; documented in include/pivco.h)
// ---------------------------------------------------------------------------
constexpr uint32_t kHdr = 16;        // fixed header
constexpr uint32_t kLensOff = 16;    // 128 bytes of 4-bit lengths
constexpr uint32_t kNvOff = 144;     // u32 n_v[n_int]
constexpr uint32_t kMaxLen = 15;     // 4-bit length field
constexpr uint8_t kMarkRawSel = 0xFF;
constexpr uint8_t kMarkFlat = 0xF0;  // a flat node of depth D (2..8) has marker 0xF0 + D

// depth D of a flat node's marker (0 for any other marker)
__host__ __device__ inline uint32_t mark_flat_d(uint32_t m) { return (m >= 0xF2u && m <= 0xF8u) ? m - 0xF0u : 0u; }
// a node with an entry in the record's alen table: ANS coded, or selected and kept raw
__host__ __device__ inline bool mark_listed(uint32_t m) { return m != 0 && !mark_flat_d(m); }
// a node whose body is an ANS stream
__host__ __device__ inline bool mark_ans(uint32_t m) { return mark_listed(m) && m != kMarkRawSel; }

// Children word of a node (node tables of encoder and decoder): child c in
// bits [16c, 16c + 16), 0x8000 | symbol for a leaf, else the child's node
// index.  A flat node (Sec. 2.2.3) is 0x80008000 | D << 24 | base: both
// halves read as leaves, D in bits 24..30, base (the index of its first
// symbol in the block's (length, symbol) order) in bits 0..7.
__host__ __device__ inline uint32_t ch_flat(uint32_t D, uint32_t base) { return 0x80008000u | (D << 24) | base; }
__host__ __device__ inline uint32_t ch_flat_d(uint32_t chv) { return (chv >> 24) & 0x7Fu; }
constexpr uint32_t kAnsSeg = 16384;  // bitmap bytes per ANS segment
constexpr uint32_t kAnsScale = 15;
constexpr uint32_t kAnsM = 1u << kAnsScale;
constexpr uint32_t kAnsL = 1u << 16;

__host__ __device__ inline uint32_t ans_seg_count(uint32_t nbytes) { return (nbytes + kAnsSeg - 1) / kAnsSeg; }
__host__ __device__ inline uint32_t ans_seg_lanes(uint32_t seg_bytes) {
    uint32_t w = (seg_bytes + 511) / 512;
    return w < 1 ? 1 : (w > 32 ? 32 : w);
}

// ---------------------------------------------------------------------------
// Static ANS tables, passed by value to kernels (Sec. 5.2: 50 tables for skew
// 50..99 %).  Byte frequencies depend only on the byte's popcount class k.
// Bytes are ordered by (k, value) in the cumulative table.
// ---------------------------------------------------------------------------
struct AnsTables {
    uint16_t q[50][9];        // frequency of one byte of class k (of 2^15)
    uint16_t start[50][10];   // cumulative start of class k; start[t][9] = 2^15
    uint32_t magic[50][9];    // ceil(2^32 / q) for exact division (q >= 2); 0 when q == 1
    int32_t fseh_q16[50];     // expected bits per bitmap bit, Q16
    uint8_t rank_in_class[256];   // index of byte b among bytes of its class
    uint8_t class_member[256];    // bytes sorted by (popcount, value)
    uint8_t class_base[10];       // first index of class k in class_member
};
const AnsTables &host_ans_tables();

// ---------------------------------------------------------------------------
// Per-block layout written by build_layout and read by the encoders.
// ---------------------------------------------------------------------------
struct BlockLayout {
    uint32_t n;            // symbols
    uint32_t rec_bound;    // record bytes with every node raw
    uint32_t body0;        // byte offset of the first body
    uint32_t body_end;     // byte offset just past the last body
    uint16_t n_int;        // internal nodes
    uint8_t kind;          // 0 empty, 1 constant, 2 coded
    uint8_t csym;          // kind 1 symbol
    uint8_t max_depth;     // longest code length
    uint8_t n_sel;         // nodes selected for ANS
    uint8_t status;        // PIVCO_* of layout construction
    uint8_t flat;          // regrouped tree with flat subtrees (record tag PVC2)
    uint8_t depth_first[17];   // first node id at depth d (breadth-first); [d+1]-[d] = count
    uint8_t big;               // the levels of the whole block do not fit the encoder's buffers
    uint8_t pad1[14];
    uint16_t tree_a[17];       // leaf-covered prefix count at depth d (TreeShape::a)
    uint16_t pad2[15];
    uint16_t code[256];    // code of symbol s (lens[s] bits, MSB = first decision; canonical or regrouped)
    uint8_t len[256];      // code length of symbol s
    uint32_t nv[256];      // symbols through node v
    uint32_t body_off[256];    // byte offset of node v's body in the record (raw layout)
    int16_t child[256][2];     // >= 0 internal id; < 0 leaf, symbol = -c - 1
    uint8_t sel[256];          // ANS candidate marker (table id | 0x80 XOR), 0 if not selected
    uint8_t depth[256];
    uint8_t fd[256];           // D of a flat node, 0 for an ordinary node
    uint8_t fbase[256];        // flat node: index of its first symbol in (length, symbol) order
    uint8_t pad3[8];
    // (from here on not staged by the encoder, which loads it straight into its tables)
    uint8_t ci[256];           // code index of symbol s: its place in the order of codes (left-aligned)
    uint8_t nlo[256];          // the leaves under node v are code indices nlo[v] .. nhi1[v]
    uint8_t nhi1[256];
    // scratch of the chunked encoder (the work list of big blocks; written
    // by the encode call, not by the plan): entry i of the list lives in
    // block i's layout, its length and the chunk ticket in block 0's
    uint32_t list_entry;
    uint32_t list_len;
    uint32_t list_ticket;
    uint32_t pad4;
};
static_assert(offsetof(BlockLayout, ci) % 16 == 0 && offsetof(BlockLayout, nhi1) + 256 == offsetof(BlockLayout, ci) + 768,
              "the canonical tables are one 16-byte aligned run");
static_assert(sizeof(BlockLayout) <= 8192, "layout too large");
constexpr int32_t kLayoutBytes = 8192;
// block b's layout record: records are kLayoutBytes apart (not sizeof(BlockLayout))
__host__ __device__ inline BlockLayout *layout_of(BlockLayout *layout, int b) {
    return reinterpret_cast<BlockLayout *>(reinterpret_cast<uint8_t *>(layout) + (size_t)b * kLayoutBytes);
}
__host__ __device__ inline const BlockLayout *layout_of(const BlockLayout *layout, int b) {
    return reinterpret_cast<const BlockLayout *>(reinterpret_cast<const uint8_t *>(layout) + (size_t)b * kLayoutBytes);
}

// ---------------------------------------------------------------------------
// Canonical tree from code lengths (Sec. 1 canonical coding, App. D).
// For a full canonical code the leaves at each depth occupy the smallest
// prefix values; a[d] counts the d-bit values covered by leaves of length
// <= d, and the internal nodes at depth d are exactly the prefixes
// a[d] .. 2^d - 1.  Nodes are numbered breadth-first (depth, prefix).
// ---------------------------------------------------------------------------
struct TreeShape {
    int32_t cnt[kMaxLen + 2];      // symbols of each length
    int32_t a[kMaxLen + 2];        // leaf-covered prefix count at depth d
    int32_t first[kMaxLen + 2];    // first node id at depth d
    int32_t len_base[kMaxLen + 2]; // index of the first symbol of length l in sorted order
    int32_t n_int;
    int32_t max_len;
    int32_t K;
    int32_t ok;
};

// Builds the tree shape and the per-symbol canonical codes.  Must be called
// by all threads of the CTA (blockDim.x >= 256).  lens/codes/sorted are in
// shared memory; `sorted` receives the symbols ordered by (length, value).
__device__ inline void build_tree_shape(const uint8_t *lens, TreeShape &ts, uint16_t *codes, uint8_t *sorted,
                                        int32_t *rank_scratch /* 256 */) {
    const int t = threadIdx.x;
    if (t < kMaxLen + 2) ts.cnt[t] = 0;
    __syncthreads();
    if (t < 256) {
        // symbols of each length: one ballot per length per warp
        const uint32_t l = lens[t];
        for (uint32_t k = 1; k <= kMaxLen; k++) {
            const uint32_t c = __popc(__ballot_sync(0xffffffffu, l == k));
            if ((t & 31) == 0 && c) atomicAdd(&ts.cnt[k], (int32_t)c);
        }
    }
    __syncthreads();
    if (t == 0) {
        int32_t a = 0, first = 0, base = 0, K = 0, ml = 0;
        bool ok = true;
        ts.a[0] = 0;
        ts.first[0] = 0;
        for (int l = 1; l <= (int)kMaxLen; l++) {
            ts.len_base[l] = base;
            base += ts.cnt[l];
            K += ts.cnt[l];
            if (ts.cnt[l]) ml = l;
        }
        // open[d] = 2^d - a[d] internal nodes at depth d; a[d] = 2 a[d-1] + cnt[d]
        for (int d = 0; d <= (int)kMaxLen; d++) {
            if (d > 0) a = 2 * a + ts.cnt[d];
            ts.a[d] = a;
            int64_t open = (int64_t(1) << d) - a;
            if (open < 0) ok = false;
            ts.first[d] = first;
            if (d < ml) {
                if (open <= 0) ok = false;
                first += (int32_t)open;
            } else if (d == ml && open != 0) {
                ok = false;     // Kraft equality: the tree is full
            }
        }
        ts.first[kMaxLen + 1] = first;
        ts.n_int = first;
        ts.max_len = ml;
        ts.K = K;
        ts.ok = ok && K >= 2 && first == K - 1;
    }
    __syncthreads();
    // rank of s among symbols of the same length (by value): lanes of equal
    // length within the warp, plus the counts of that length in earlier warps
    if (t < 128) rank_scratch[t] = 0;
    __syncthreads();
    int32_t rank_in_warp = 0;
    if (t < 256) {
        const uint32_t l = lens[t];
        const uint32_t peers = __match_any_sync(0xffffffffu, l);
        rank_in_warp = __popc(peers & ((1u << (t & 31)) - 1u));
        if (rank_in_warp == 0) rank_scratch[(t >> 5) * 16 + (l & 15)] = __popc(peers);
    }
    __syncthreads();
    if (t < 256) {
        const uint8_t l = lens[t];
        if (l && ts.ok) {
            int32_t r = rank_in_warp;
            for (int w = 0; w < (t >> 5); w++) r += rank_scratch[w * 16 + l];
            sorted[ts.len_base[l] + r] = (uint8_t)t;
            codes[t] = (uint16_t)(2 * ts.a[l - 1] + r);
        } else {
            codes[t] = 0;
        }
    }
    __syncthreads();
}

// depth of internal node v
__device__ inline int node_depth(const TreeShape &ts, int v) {
    int d = 0;
    while (d < ts.max_len && ts.first[d + 1] <= v) d++;
    return d;
}

// child b of internal node v at depth d: >= 0 internal id, < 0 leaf -(sym+1)
__device__ inline int node_child(const TreeShape &ts, const uint8_t *sorted, int v, int d, int b) {
    const int32_t p = ts.a[d] + (v - ts.first[d]);
    const int32_t q = 2 * p + b;
    if (q < ts.a[d + 1]) return -(int)sorted[ts.len_base[d + 1] + (q - 2 * ts.a[d])] - 1;
    return ts.first[d + 1] + (q - ts.a[d + 1]);
}

// ---------------------------------------------------------------------------
// Regrouped tree with flat subtrees (Sec. 2.2.3-2.2.4).  Each length class l
// (symbols ascending) is cut into groups of the largest power of two left,
// first 2^D symbols first; a group is an item of length l - D.  The items
// form a canonical tree ordered by (item length, first symbol): a[d] counts
// the d-bit prefixes covered by items of length <= d, the items of length d
// hold prefixes 2 a[d-1] .. a[d] - 1 by rank, the prefixes a[d] .. 2^d - 1
// are ordinary nodes.  An item of two symbols is an ordinary node with two
// leaves, one of 2^D >= 4 a flat node, one of a single symbol a leaf.  Nodes
// are numbered breadth-first (depth, prefix): at each depth the item nodes
// (by rank) come before the item tree's own nodes.  Symbol x of item i has
// the code (code_i << D) | x.
// ---------------------------------------------------------------------------
constexpr int kMaxItems = 144;    // 15 length classes x at most 9 groups each
struct FlatTree {
    int32_t a[18];
    int32_t first[18];            // first node id at depth d
    int32_t nin[18];              // item nodes (pairs and flat groups) at depth d
    int32_t icnt[18];             // items of length d
    int32_t nitems, maxd, n_nodes, ok;
    uint8_t it_of[16][9];         // item of length d and rank r
    uint8_t in_of[16][9];         // k-th item node of depth d
    uint8_t item_ld[16][9];       // item of length class l made of 2^D symbols
    uint8_t iD[kMaxItems], il[kMaxItems], irank[kMaxItems], ik[kMaxItems];
    uint16_t iso[kMaxItems];      // index of the item's first symbol in (length, symbol) order
    uint16_t ioff[kMaxItems];     // symbols of the items before it in code order
};

// Builds the item tree of the code lengths (one warp, all lanes).  cnt[l]:
// symbols of length l (l = 1..15); start[l]: index of the first of them in
// `sorted` (the symbols in (length, symbol) order).  F.ok = 0 unless the items
// make a full tree.
__device__ inline void flat_tree_build(const int32_t *cnt, const int32_t *start, const uint8_t *sorted, FlatTree &F) {
    const int lane = threadIdx.x & 31;
    // lane l makes the items of length class l: one per set bit D of its
    // count, largest first, each taking the next 2^D symbols of the class
    const int c = (lane >= 1 && lane <= (int)kMaxLen) ? cnt[lane] : 0;
    bool ok = c >= 0 && c <= 256 && (c >> (lane < 9 ? lane + 1 : 9)) == 0;   // at most 2^l symbols of length l
    const int mine = __popc((uint32_t)c & 0x1FFu);
    int base = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, base, o);
        if (lane >= o) base += y;
    }
    const int total = __shfl_sync(0xffffffffu, base, 31);
    base -= mine;
    if (lane < 18) F.icnt[lane] = 0;
    __syncwarp();
    if (ok && total <= kMaxItems) {
        int i = base, acc = 0;
        for (int D = 8; D >= 0; D--) {
            if (!((c >> D) & 1)) continue;
            F.iD[i] = (uint8_t)D;
            F.il[i] = (uint8_t)(lane - D);
            F.iso[i] = (uint16_t)(start[lane] + acc);
            F.item_ld[lane][D] = (uint8_t)i;
            atomicAdd(&F.icnt[lane - D], 1);
            acc += 1 << D;
            i++;
        }
    }
    ok = __all_sync(0xffffffffu, ok) && total <= kMaxItems;
    const int n = ok ? total : 0;
    __syncwarp();
    // rank of an item among the items of its length, by first symbol
    for (int i = lane; i < n; i += 32) {
        const uint32_t fs = sorted[F.iso[i]];
        int r = 0;
        for (int j = 0; j < n; j++) r += F.il[j] == F.il[i] && sorted[F.iso[j]] < fs;
        F.irank[i] = (uint8_t)r;
        if (r < 9) F.it_of[F.il[i]][r] = (uint8_t)i;
        else ok = false;
    }
    int maxil = 0;
    for (int i = lane; i < n; i += 32) maxil = max(maxil, (int)F.il[i]);
    maxil = __reduce_max_sync(0xffffffffu, (uint32_t)maxil);
    ok = __all_sync(0xffffffffu, ok);
    __syncwarp();
    // depth d = lane: Kraft equality at the item level (a[d] d-bit prefixes
    // covered by items of length <= d), the item nodes of depth d in rank
    // order, then the item tree's own nodes
    int cnt_d = 0;
    if (lane < 18) {
        int64_t a = 0;
        for (int j = 0; j <= lane; j++) a = 2 * a + F.icnt[j];
        F.a[lane] = (int32_t)(a > 0x7FFFFFFF ? 0x7FFFFFFF : a);
        if (lane <= 15 && a > (int64_t(1) << lane)) ok = false;
        if (lane < maxil && a >= (int64_t(1) << lane)) ok = false;
        if (lane == maxil && a != (int64_t(1) << lane)) ok = false;
        int k = 0;
        if (lane <= maxil && lane < 16)
            for (int r = 0; r < F.icnt[lane] && r < 9; r++) {
                const int i = F.it_of[lane][r];
                if (F.iD[i] >= 1) { F.in_of[lane][k] = (uint8_t)i; F.ik[i] = (uint8_t)k; k++; }
            }
        F.nin[lane] = k;
        const int64_t open = lane < maxil ? (int64_t(1) << lane) - a : 0;
        cnt_d = lane < 17 ? k + (int)(open > 0 ? open : 0) : 0;
    }
    ok = __all_sync(0xffffffffu, ok);
    int f = cnt_d;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, f, o);
        if (lane >= o) f += y;
    }
    if (lane < 18) F.first[lane] = f - cnt_d;
    const int n_nodes = __shfl_sync(0xffffffffu, f, 31);
    const uint32_t used = __ballot_sync(0xffffffffu, cnt_d > 0);
    // code order of the items: by (length, rank); the symbols of the items
    // before each one
    if (ok) {
        for (int i = lane; i < n; i += 32) {
            uint32_t off = 0;
            for (int j = 0; j < n; j++)
                if (F.il[j] < F.il[i] || (F.il[j] == F.il[i] && F.irank[j] < F.irank[i])) off += 1u << F.iD[j];
            F.ioff[i] = (uint16_t)off;
        }
    }
    if (lane == 0) {
        F.nitems = n;
        F.maxd = used ? 32 - __clz(used) : 0;
        F.n_nodes = n_nodes;
        F.ok = ok && n_nodes >= 1 && n_nodes <= 255;
    }
    __syncwarp();
}

// Symbol number r (0-based) of length class l: its item (l, D) is the group
// whose range holds r, D the highest bit where the class count has a one
// and r a zero; x = r's low D bits is its index in the group.
__device__ inline void flat_sym(const FlatTree &F, const int32_t *cnt, int l, int r, int &item, uint32_t &x) {
    const uint32_t c = (uint32_t)cnt[l], m = c & ~(uint32_t)r;
    const int D = m ? 31 - __clz(m) : 0;
    item = F.item_ld[l][D];
    x = (uint32_t)r & ((1u << D) - 1u);
}

// code of item i's prefix (its item length F.il[i] bits)
__device__ inline uint32_t flat_item_code(const FlatTree &F, int i) {
    const int l = F.il[i];
    return l ? (uint32_t)(2 * F.a[l - 1] + F.irank[i]) : 0u;
}

// Node v of the regrouped tree: its depth and children word (ch_flat for a
// flat node).  Returns false for ids or children out of range.
__device__ inline bool flat_node(const FlatTree &F, const uint8_t *sorted, int v, int &depth, uint32_t &chv) {
    int d = 0;
    while (d < F.maxd - 1 && F.first[d + 1] <= v) d++;
    depth = d;
    chv = 0;
    if (v < 0 || v >= F.n_nodes) return false;
    const int k = v - F.first[d];
    if (k < F.nin[d]) {
        const int i = F.in_of[d][k];
        if (F.iD[i] == 1) chv = ((0x8000u | sorted[F.iso[i] + 1]) << 16) | (0x8000u | sorted[F.iso[i]]);
        else chv = ch_flat(F.iD[i], F.iso[i]);
        return true;
    }
    const int32_t p = F.a[d] + (k - F.nin[d]);
    for (int b = 0; b < 2; b++) {
        const int32_t q = 2 * p + b;
        uint32_t code;
        if (d + 1 > 15) return false;
        if (q < F.a[d + 1]) {
            const int32_t r = q - 2 * F.a[d];
            if (r < 0 || r >= F.icnt[d + 1] || r >= 9) return false;
            const int i = F.it_of[d + 1][r];
            code = F.iD[i] == 0 ? (0x8000u | sorted[F.iso[i]]) : (uint32_t)(F.first[d + 1] + F.ik[i]);
        } else {
            code = (uint32_t)(F.first[d + 1] + F.nin[d + 1] + (q - F.a[d + 1]));
        }
        if (!(code & 0x8000u) && (code <= (uint32_t)v || code >= (uint32_t)F.n_nodes)) return false;
        chv |= code << (16 * b);
    }
    return true;
}

// ---------------------------------------------------------------------------
// Small utilities
// ---------------------------------------------------------------------------
__device__ inline uint32_t ld_le32(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
__device__ inline void st_le32(uint8_t *p, uint32_t v) {
    p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); p[2] = (uint8_t)(v >> 16); p[3] = (uint8_t)(v >> 24);
}
__device__ inline uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr uint64_t kWaitLimitNs = 1000000000ull;   // default bound of a device wait: 1 s
uint64_t wait_limit_ns();                          // the current bound (pivco_set_wait_limit)

__host__ __device__ inline uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
// kernels launched by this library (reported through pivco_launch_count)
void count_launches(int n);
inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

// Launchers implemented in the kernel translation units.
// Warp chunks of an encoded block: a block of n symbols is cut into
// nw = min(8, max(1, n / 4096)) contiguous chunks, chunk w starting at
// floor(n w / nw) rounded down to a multiple of 32.  The encoder gives chunk w
// to its warp w; the chunked histogram counts each chunk on its own.
constexpr uint32_t kEncChunks = 8;
constexpr int kEBuf = 13824;         // symbols per encoder level buffer (a skew80 64 KiB block in one chunk)
constexpr uint32_t kEncMinChunk = 4096;
__host__ __device__ inline uint32_t enc_nchunks(uint64_t n) {
    const uint64_t c = n / kEncMinChunk;
    return (uint32_t)(c < 1 ? 1 : (c > kEncChunks ? kEncChunks : c));
}
__host__ __device__ inline uint32_t enc_chunk_start(uint64_t n, uint32_t w, uint32_t nw) {
    return w >= nw ? (uint32_t)n : (uint32_t)((n * w / nw) & ~31ull);
}
cudaError_t launch_histogram_chunks(const uint8_t *in, const uint64_t *blk_off, int nblk, uint32_t *hist,
                                    uint32_t *chunk_hist, cudaStream_t st);
struct BlockLayout;
cudaError_t launch_block_plan(const uint8_t *in, const uint64_t *blk_off, int nblk, const pivco_params &p,
                              uint32_t *hist, uint32_t *chunk_hist, uint8_t *lens, BlockLayout *layout,
                              uint64_t *rec_bound, int32_t *status, cudaStream_t st);

cudaError_t launch_histogram(const uint8_t *in, const uint64_t *blk_off, int nblk, uint32_t *hist,
                             int slices, cudaStream_t st);
cudaError_t launch_code_lengths(const uint32_t *hist, int nblk, int max_len, uint8_t *lens, int32_t *status,
                                cudaStream_t st);
cudaError_t launch_build_layout(const uint32_t *hist, const uint8_t *lens, int nblk, const pivco_params &p,
                                BlockLayout *layout, uint64_t *rec_bound, int32_t *status, cudaStream_t st);
cudaError_t launch_scan(const uint64_t *in, int n, uint64_t *out, void *ws, int32_t *status, cudaStream_t st);
size_t scan_ws_bytes(int n);
cudaError_t launch_encode(const uint8_t *in, const uint64_t *blk_off, int nblk, BlockLayout *layout,
                          const uint32_t *chunk_hist, uint8_t *out, const uint64_t *out_off, uint64_t *rec_bytes,
                          int32_t *status, cudaStream_t st);
cudaError_t launch_ans_encode_blocks(const BlockLayout *layout, int nblk, uint8_t *out, const uint64_t *out_off,
                                     uint64_t *rec_bytes, uint8_t *ws, size_t ws_bytes, int32_t *status,
                                     cudaStream_t st);
cudaError_t launch_ans_encode(const uint8_t *bm, const uint64_t *bm_off, const uint8_t *table, int nbm,
                              uint8_t *bodies, const uint64_t *body_off, uint64_t *body_bytes, int32_t *status,
                              cudaStream_t st);
cudaError_t launch_ans_decode(const uint8_t *bodies, const uint64_t *body_off, const uint8_t *table, int nbm,
                              uint8_t *bm, const uint64_t *bm_off, int32_t *status, cudaStream_t st);
// ---------------------------------------------------------------------------
// Decode workspace (written by the decode plan, read by the later passes):
//   header (64 B): u64 scratch bytes @0, u32 ANS segments @8, u32 ticket @12,
//                  u64 directory+cursor bytes @16, u32 tiles @24,
//                  u32 directory granularity (bits) @28, u32 longest tile @32,
//                  u32 batch queue ticket @36, u32 batch plans done @40,
//                  u32 items done (serving) @44, u32 tile ticket @48,
//                  u32 abandoned @52 (a CTA gave up on the queue),
//                  u64 wait bound in ns @56
//   per block: u64 look-back states A[nblk], B[nblk]; u64 scratch offset[nblk];
//              u64 directory offset[nblk]; u32 first segment[nblk];
//              u32 first tile[nblk]; u32 tile length[nblk]; u32 tiles[nblk];
//              u32 ANS segments done[nblk]; u32 directory done[nblk]
//   then: rank directories and tile-boundary cursors, ANS-decoded bitmaps.
// ---------------------------------------------------------------------------
struct DecWs {
    uint64_t *states_a, *states_b, *blk_scratch, *blk_dir;
    uint32_t *blk_seg, *blk_tile, *blk_T, *blk_ntile, *segs_done, *dir_done;
    uint32_t *plan_done;   // 1 | 2 (one tile, no ANS, no directory) once the block's plan is complete
};
__host__ __device__ inline size_t decode_ws_fixed_bytes(int nblk) {
    const size_t f = 64 + 32ull * nblk + 28ull * nblk;
    return (f + 255) & ~(size_t)255;
}

// Launch tuning of the decode (never changes the decoded bytes)
struct DecTuning {
    uint32_t tile_max;      // longest root tile (symbols), a multiple of 128, <= 2^20
    uint32_t dir_bits;      // rank directory granularity (bits), a multiple of 32, <= 1024
    uint32_t ctas_per_sm;   // persistent merge CTAs per SM (0: as many as fit)
};
DecTuning current_tuning();   // a copy, taken under the tuning lock
void set_tuning(const DecTuning &t);
__host__ __device__ inline DecWs dec_ws(uint8_t *ws, int nblk) {
    DecWs w;
    w.states_a = reinterpret_cast<uint64_t *>(ws + 64);
    w.states_b = w.states_a + nblk;
    w.blk_scratch = w.states_b + nblk;
    w.blk_dir = w.blk_scratch + nblk;
    w.blk_seg = reinterpret_cast<uint32_t *>(w.blk_dir + nblk);
    w.blk_tile = w.blk_seg + nblk;
    w.blk_T = w.blk_tile + nblk;
    w.blk_ntile = w.blk_T + nblk;
    w.segs_done = w.blk_ntile + nblk;
    w.dir_done = w.segs_done + nblk;
    w.plan_done = w.dir_done + nblk;
    return w;
}
struct DecRegions {
    size_t dir, scratch, need;
};
__host__ __device__ inline DecRegions dec_regions(int nblk, const uint8_t *ws_header) {
    const uint64_t scratch = *reinterpret_cast<const uint64_t *>(ws_header);
    const uint64_t dir = *reinterpret_cast<const uint64_t *>(ws_header + 16);
    DecRegions r;
    r.dir = decode_ws_fixed_bytes(nblk);
    r.scratch = (r.dir + dir + 255) & ~(size_t)255;
    r.need = r.scratch + scratch;
    return r;
}
// ---- serving (device-resident request loop) ----
constexpr uint32_t kServeRing = 4096;       // ring entries (requests admitted and not yet retired)
struct ServeDesc {                          // one published request (device memory)
    const uint8_t *comp;
    const uint64_t *comp_off;
    uint8_t *out;
    const uint64_t *out_off;
    uint8_t *ws;
    uint64_t ws_bytes;
    int32_t *status;
    int32_t nblk;
    uint32_t seq;
};
static_assert(sizeof(ServeDesc) == 64, "ring entry layout");
struct ServeCtl {                           // device memory
    uint32_t cur;                           // requests before cur hand out no more items
    uint32_t pad[63];
};
struct ServeFlags {                         // pinned host memory mapped into the device
    uint32_t tail;                          // requests published (host writes)
    uint32_t stop;                          // nonzero: every CTA leaves (host writes)
    uint32_t pad[30];
    uint32_t done[kServeRing];              // seq + 1 once request seq is decoded (device writes)
    int32_t worst[kServeRing];              // its first non-OK block status, else 0 (device writes)
};
cudaError_t launch_serve_loop(ServeCtl *ctl, const ServeDesc *ring, ServeFlags *flags, uint64_t idle_ns,
                              uint64_t life_ns, cudaStream_t st);
size_t decode_ws_bound(const uint8_t *comp, const uint64_t *comp_off, int nblk, const DecTuning &tu);
size_t decode_ws_size_bound(const uint64_t *blk_off, int nblk, const DecTuning &tu);

cudaError_t launch_decode_plan(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *ws,
                               size_t ws_bytes, int32_t *status, cudaStream_t st, bool all_dirs = false);
cudaError_t launch_access_prepare(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *ws,
                                  size_t ws_bytes, int32_t *status, cudaStream_t st);
cudaError_t launch_access(const uint8_t *comp, const uint64_t *comp_off, int nblk, const uint32_t *qblk,
                          const uint32_t *qpos, int nq, uint8_t *sym, int32_t *qstatus, const uint8_t *ws,
                          size_t ws_bytes, const int32_t *status, cudaStream_t st);
cudaError_t launch_zero_bytes(uint8_t *p, size_t n, cudaStream_t st);
cudaError_t launch_ans_decode_planned(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *ws,
                                      size_t ws_bytes, int32_t *status, cudaStream_t st);
cudaError_t launch_decode_merge(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *out,
                                const uint64_t *out_off, uint8_t *ws, size_t ws_bytes, int32_t *status,
                                cudaStream_t st);
cudaError_t launch_decode_dir(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *ws, size_t ws_bytes,
                              int32_t *status, cudaStream_t st);
cudaError_t launch_golomb_plan(const uint8_t *in, const uint64_t *blk_off, int nblk, uint64_t *rec_size,
                               int32_t *status, cudaStream_t st);
cudaError_t launch_golomb_encode(const uint8_t *in, const uint64_t *blk_off, int nblk, uint8_t *out,
                                 const uint64_t *out_off, uint64_t *rec_bytes, int32_t *status, cudaStream_t st);
cudaError_t launch_golomb_decode(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *out,
                                 const uint64_t *out_off, int32_t *status, cudaStream_t st);
cudaError_t prepare_golomb_kernels();
cudaError_t prepare_decode_kernels();
cudaError_t prepare_encode_kernels();
cudaError_t prepare_ans_kernels();
cudaError_t launch_decode_batch(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *out,
                                const uint64_t *out_off, uint8_t *ws, size_t ws_bytes, int32_t *status,
                                cudaStream_t st);
cudaError_t read_decode_ws_need(const uint8_t *ws, int nblk, size_t *need, cudaStream_t st);
cudaError_t launch_decode(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *out,
                          const uint64_t *out_off, uint8_t *ws, size_t ws_bytes, int32_t *status,
                          cudaStream_t st);

}  // namespace pv
