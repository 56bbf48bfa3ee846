// Decode side: plan, ANS pass, rank directories and the bottom-up merge
// (Sec. 3; Sec. 5.2 for ANS-coded bitmaps).
//
//   plan       one warp per record: validates the header and body layout,
//              sizes the ANS scratch, and splits the block into root tiles
//              whose levels fit the merge's buffers; per-block offsets come
//              from two single-pass scans with decoupled look-back.
//   ans        one warp per 16 KiB ANS segment: decodes the bitmap bytes into
//              the workspace scratch.
//   directory  for blocks with several tiles: per-node rank directories
//              (exclusive popcount per 256-bit superblock) and, from them,
//              every node's bitmap cursor at every tile boundary (the root
//              cursor is the position; a child's cursor is the parent's
//              rank0 / rank1 there).
//   merge      one CTA per tile (persistent).  With both boundary cursors
//              known, each node's bit range for the tile is known; its
//              128-bit units are popcounted in one flat pass and scanned per
//              node (the tile's rank directory).  Bottom-up, every node
//              rebuilds its symbol sequence
//                  out_v[k] = bit ? R[rank1(k)] : L[k - rank1(k)]
//              from its children's sequences or leaf constants (MVV / MCV /
//              MVC / MCC of Table 8), 4 symbols per lane with one byte
//              permute.  The root writes the output.  A tile whose levels do
//              not fit is decoded in shorter chunks whose bit ranges are
//              found top-down from popcounts.
#include "ans_dev.cuh"
#include "lookback.cuh"
#include "tma.cuh"

namespace pv {

constexpr int kDecThreads = 256;
constexpr int kDecWarps = kDecThreads / 32;
constexpr int kDUnit = 128;
constexpr int kDLvlCap = 14336;              // level buffer capacity (depths >= 1)
constexpr int kDLvlBytes = kDLvlCap + 16;    // slack for 4-byte windows
constexpr int kDMaxRoot = 65536;             // longest chunk
constexpr int kDRecSmem = 24576;             // records up to this size are staged in shared memory
constexpr int kDMaxUnits = kDMaxRoot / kDUnit + 14 * (kDLvlCap / kDUnit) + 256;

__host__ __device__ inline uint32_t scratch_stride(uint32_t raw) { return ((raw + 15u) & ~15u) + 16u; }

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

// ---------------------------------------------------------------------------
// Warp-level record parse (plan and ANS passes)
// ---------------------------------------------------------------------------
struct WarpRec {
    uint32_t nv[256];
    uint32_t body_off[256];
    uint32_t alen[256];
    uint32_t soff[256];      // scratch offset of an ANS node within its block
    uint32_t segbase[256];   // first ANS segment of the node within its block
    uint8_t marker[256];
    uint32_t V, n, kind, rb, scratch_bytes, nsegs;
};

__device__ inline bool warp_parse(const uint8_t *rec, uint64_t avail, WarpRec &R) {
    const int lane = threadIdx.x & 31;
    bool ok = avail >= kHdr;
    uint32_t rb = 0, n = 0, V = 0, kind = 0;
    if (ok) {
        rb = ld_le32(rec);
        n = ld_le32(rec + 4);
        V = (uint32_t)rec[8] | ((uint32_t)rec[9] << 8);
        kind = rec[10];
        ok = rec[12] == 'P' && rec[13] == 'V' && rec[14] == 'C' && rec[15] == '1' && rb >= kHdr && !(rb & 15u) &&
             rb <= avail;
    }
    if (lane == 0) { R.rb = rb; R.n = n; R.kind = kind; R.scratch_bytes = 0; R.nsegs = 0; R.V = 0; }
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
        if (m && m != kMarkRawSel && ((m & 0x7F) < 1 || (m & 0x7F) > 50)) ok = false;
    }
    __syncwarp();
    const uint32_t alen_off = (kNvOff + 5 * V + 3) & ~3u;
    const uint32_t nsel = warp_scan_loop_d(Vi, [&](int v) { return (uint32_t)(R.marker[v] != 0); },
                                           [&](int v, uint32_t p) { R.segbase[v] = p; });
    if (alen_off + 4 * nsel > rb) ok = false;
    __syncwarp();
    if (__any_sync(0xffffffffu, !ok)) return false;
    for (int v = lane; v < Vi; v += 32) {
        const uint32_t raw = (R.nv[v] + 7) / 8;
        const uint32_t al = R.marker[v] ? ld_le32(rec + alen_off + 4 * R.segbase[v]) : raw;
        R.alen[v] = al;
        if (R.marker[v] == kMarkRawSel && al != raw) ok = false;
    }
    __syncwarp();
    const uint32_t base1 = alen_off + 4 * nsel;
    const uint32_t raw_tot = warp_scan_loop_d(Vi, [&](int v) { return R.marker[v] ? 0u : R.alen[v]; },
                                              [&](int v, uint32_t p) { if (!R.marker[v]) R.body_off[v] = base1 + p; });
    const uint32_t base2 = base1 + raw_tot;
    uint64_t sel_tot = 0;
    {
        // 64-bit: corrupt alen values could wrap 32 bits
        uint64_t carry = 0;
        for (int base = 0; base < Vi; base += 32) {
            const int v = base + lane;
            const uint64_t x = (v < Vi && R.marker[v]) ? R.alen[v] : 0;
            uint64_t inc = x;
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (v < Vi && R.marker[v]) R.body_off[v] = (uint32_t)(base2 + carry + inc - x);
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        sel_tot = carry;
    }
    if ((((uint64_t)base2 + sel_tot + 15) & ~15ull) != rb) ok = false;
    const uint32_t stot = warp_scan_loop_d(Vi, [&](int v) {
        return (R.marker[v] && R.marker[v] != kMarkRawSel) ? scratch_stride((R.nv[v] + 7) / 8) : 0u;
    }, [&](int v, uint32_t p) { R.soff[v] = p; });
    const uint32_t segs = warp_scan_loop_d(Vi, [&](int v) {
        return (R.marker[v] && R.marker[v] != kMarkRawSel) ? ans_seg_count((R.nv[v] + 7) / 8) : 0u;
    }, [&](int v, uint32_t p) { R.segbase[v] = p; });
    for (int v = lane; v < Vi; v += 32)
        if (R.nv[v] < 2 || R.nv[v] > n) ok = false;
    if (lane == 0 && R.nv[0] != n) ok = false;
    if (lane == 0) { R.scratch_bytes = stot; R.nsegs = segs; }
    __syncwarp();
    return __all_sync(0xffffffffu, ok);
}

// ---------------------------------------------------------------------------
// Plan: one warp per record (ticket order), two look-back chains over blocks
//   A: (ANS scratch bytes << 22) | ANS segments
//   B: (directory + cursor bytes << 22) | tiles
// Tuning (from the workspace header): the longest tile and the rank
// directory granularity; neither changes the decoded bytes.
// ---------------------------------------------------------------------------
struct PlanScratch {
    uint32_t cntl[16], first[17], lvl[16];
};

__device__ inline void plan_block(int b, const uint8_t *__restrict__ comp, const uint64_t *__restrict__ comp_off,
                                  int nblk, uint8_t *__restrict__ ws, int32_t *__restrict__ status, WarpRec &R,
                                  PlanScratch &Q) {
    const int lane = threadIdx.x & 31;
    uint32_t *hdr32 = reinterpret_cast<uint32_t *>(ws);
    uint64_t *hdr64 = reinterpret_cast<uint64_t *>(ws);
    const DecWs W = dec_ws(ws, nblk);
    const uint32_t dir_bits = hdr32[7], tile_max = hdr32[8];
    if (lane < 16) { Q.cntl[lane] = 0; Q.lvl[lane] = 0; }
    __syncwarp();
    const uint8_t *rec = comp + comp_off[b];
    bool ok = warp_parse(rec, comp_off[b + 1] - comp_off[b], R);
    __syncwarp();
    uint32_t ntile = 1, T = ok ? R.n : 0;
    uint64_t dir_bytes = 0;
    if (ok && R.kind == 2) {
        // node depths from the code lengths (canonical tree shape)
        const uint32_t x = ld_le32(rec + kLensOff + 4 * lane);
        for (int j = 0; j < 8; j++) {
            const uint32_t l = (x >> (4 * j)) & 15u;
            if (l) atomicAdd(&Q.cntl[l], 1u);
        }
        __syncwarp();
        if (lane == 0) {
            int64_t a = 0, f = 0;
            int ml = 0;
            for (int l = 1; l < 16; l++) if (Q.cntl[l]) ml = l;
            Q.first[0] = 0;
            for (int d = 0; d < 16; d++) {
                if (d > 0) a = 2 * a + Q.cntl[d];
                const int64_t open = (int64_t(1) << d) - a;
                if (d < ml) f += open > 0 ? open : 0;
                Q.first[d + 1] = (uint32_t)(f > 255 ? 255 : f);
            }
        }
        __syncwarp();
        if (Q.first[15] != R.V) ok = false;
        for (int v = lane; v < (int)R.V && ok; v += 32) {
            int d = 0;
            while (d < 15 && Q.first[d + 1] <= (uint32_t)v) d++;
            if (d >= 1) atomicAdd(&Q.lvl[d], R.nv[v]);
        }
        __syncwarp();
        ok = __all_sync(0xffffffffu, ok);
        if (ok) {
            uint64_t mx = 1;
            for (int d = 1; d < 16; d++) mx = Q.lvl[d] > mx ? Q.lvl[d] : mx;
            const uint64_t fit = (uint64_t)(kDLvlCap - 4 * 256) * R.n / mx;
            uint64_t t2 = 0;
            if (fit < R.n) t2 = fit / 5 * 4;   // several tiles: 20 % headroom against uneven statistics
            else if (R.n > tile_max) t2 = tile_max;
            if (t2) {
                t2 = t2 > (uint64_t)tile_max ? (uint64_t)tile_max : t2;
                T = (uint32_t)(t2 < (uint64_t)kDUnit ? kDUnit : (t2 & ~(uint64_t)(kDUnit - 1)));
                ntile = (R.n + T - 1) / T;
                const uint32_t ent = warp_scan_loop_d((int)R.V, [&](int v) { return (R.nv[v] + dir_bits - 1) / dir_bits; },
                                                      [&](int, uint32_t) {});
                dir_bytes = ((4ull * ent + 4ull * (ntile + 1) * R.V) + 15) & ~15ull;
            }
        }
    }
    const uint64_t sb = ok ? R.scratch_bytes : 0, sg = ok ? R.nsegs : 0;
    if (!ok) { ntile = 1; T = 0; dir_bytes = 0; }
    if (lane == 0) {
        int to = 0;
        const uint64_t ea = lookback_exclusive(W.states_a, b, (sb << 22) | sg, &to);
        const uint64_t eb = lookback_exclusive(W.states_b, b, (dir_bytes << 22) | ntile, &to);
        W.blk_scratch[b] = ea >> 22;
        W.blk_seg[b] = (uint32_t)(ea & ((1u << 22) - 1));
        W.blk_dir[b] = eb >> 22;
        W.blk_tile[b] = (uint32_t)(eb & ((1u << 22) - 1));
        W.blk_T[b] = T;
        W.blk_ntile[b] = ntile;
        status[b] = !ok ? PIVCO_ERR_CORRUPT : (to ? PIVCO_ERR_TIMEOUT : PIVCO_OK);
        if (b == nblk - 1) {
            hdr64[0] = (ea >> 22) + sb;
            hdr32[2] = (uint32_t)((ea & ((1u << 22) - 1)) + sg);
            hdr64[2] = (eb >> 22) + dir_bytes;
            hdr32[6] = (uint32_t)((eb & ((1u << 22) - 1)) + ntile);
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(32) decode_plan_kernel(const uint8_t *__restrict__ comp,
                                                         const uint64_t *__restrict__ comp_off, int nblk,
                                                         uint8_t *__restrict__ ws, int32_t *__restrict__ status) {
    __shared__ WarpRec R;
    __shared__ PlanScratch Q;
    __shared__ int s_tile;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(&reinterpret_cast<uint32_t *>(ws)[3], 1u);
    __syncwarp();
    plan_block(s_tile, comp, comp_off, nblk, ws, status, R, Q);
}

// zero the header, the look-back states and the batch counters; set the tuning
__global__ void dec_ws_init_kernel(uint8_t *ws, int nblk, uint32_t dir_bits, uint32_t tile_max) {
    const DecWs W = dec_ws(ws, nblk);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nblk; i += gridDim.x * blockDim.x) {
        W.states_a[i] = 0;
        W.states_b[i] = 0;
        W.segs_done[i] = 0;
        W.dir_done[i] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x < 16) {
        uint32_t *h = reinterpret_cast<uint32_t *>(ws);
        h[threadIdx.x] = threadIdx.x == 7 ? dir_bits : (threadIdx.x == 8 ? tile_max : 0u);
    }
}

cudaError_t launch_decode_plan(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *ws, size_t ws_bytes,
                               int32_t *status, cudaStream_t st) {
    (void)ws_bytes;
    if (nblk <= 0) return cudaSuccess;
    const DecTuning &tu = current_tuning();
    dec_ws_init_kernel<<<min(1024, div_up(nblk, 256)), 256, 0, st>>>(ws, nblk, tu.dir_bits, tu.tile_max);
    decode_plan_kernel<<<nblk, 32, 0, st>>>(comp, comp_off, nblk, ws, status);
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
            if (m && m != kMarkRawSel) {
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
                                        scratch + sdst + (size_t)s * kAnsSeg);
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
// Shared-memory state of one CTA working on one block (directory and merge)
// ---------------------------------------------------------------------------
struct DecSmem {
    uint8_t rec[kDRecSmem];          // record copy (bulk copy destination, 16-aligned)
    uint8_t buf[2][kDLvlBytes];      // level buffers (depth d uses buf[d & 1])
    uint32_t ubase[kDMaxUnits];      // unit popcount, then the unit's rank base within its node
    uint8_t umap[kDMaxUnits];        // unit -> node
    uint32_t sel[4][16];             // byte-permute selectors by (node kind, 4 bits)
    uint32_t cur[256];               // bits of node v consumed before the current chunk
    uint32_t dem[256];               // bits of node v used by the current chunk
    uint32_t span[256];              // span of node v in its level buffer
    uint32_t ustart[256];            // first unit of node v
    uint32_t nv[256];
    uint32_t src_off[256];           // bitmap start: record byte offset or scratch offset
    uint32_t alen[256];
    uint32_t lvl_units[17];
    int32_t first[17];
    int16_t child[256][2];
    uint8_t depth[256];
    uint8_t src_kind[256];           // 0: record (shared copy), 1: record (global), 2: scratch
    uint8_t lens[256];
    uint8_t sorted[256];
    uint8_t marker[256];
    uint16_t codes[256];
    int32_t rank_scratch[256];
    TreeShape ts;
    uint64_t mbar;
    int32_t flag;                    // 1 corrupt, 2 capacity
    int32_t overflow;
    uint32_t chunk;
    uint32_t item;                   // batch queue item of this CTA
};

__device__ inline uint32_t bits32_g(const uint8_t *base, uint64_t bit, uint64_t limit) {
    const uint64_t wi = bit >> 5;
    const uint32_t sh = (uint32_t)(bit & 31);
    const uint32_t *w = reinterpret_cast<const uint32_t *>(base);
    const uint32_t lo = (4 * wi + 4 <= limit) ? __ldg(w + wi) : 0u;
    const uint32_t hi = (sh && 4 * wi + 8 <= limit) ? __ldg(w + wi + 1) : 0u;
    return sh ? __funnelshift_r(lo, hi, sh) : lo;
}
__device__ inline uint32_t bits32_s(const uint8_t *base, uint32_t bit, uint32_t limit) {
    const uint32_t wi = bit >> 5, sh = bit & 31;
    const uint32_t *w = reinterpret_cast<const uint32_t *>(base);
    const uint32_t lo = (4 * wi + 4 <= limit) ? w[wi] : 0u;
    const uint32_t hi = (4 * wi + 8 <= limit) ? w[wi + 1] : 0u;
    return __funnelshift_r(lo, hi, sh);
}

struct NodeSrc {
    const uint8_t *rec_g;
    const uint8_t *scratch;
    uint64_t scratch_lim;
    uint32_t rb;
};

// bits [c, c + 32) of node v's bitmap
__device__ inline uint32_t node_bits(const DecSmem &S, const NodeSrc &src, int v, uint32_t c) {
    const uint8_t k = S.src_kind[v];
    if (k == 0) return bits32_s(S.rec, 8u * S.src_off[v] + c, src.rb);
    if (k == 1) return bits32_g(src.rec_g, 8ull * S.src_off[v] + c, src.rb);
    const uint64_t off = S.src_off[v];
    return bits32_g(src.scratch + off, c, src.scratch_lim > off ? src.scratch_lim - off : 0);
}

__device__ inline uint32_t mask_valid(uint32_t w, int64_t valid) {
    return valid >= 32 ? w : (valid <= 0 ? 0u : (w & ((1u << valid) - 1u)));
}

// 4 bytes at any byte offset of a level buffer (reads up to 7 bytes past p)
__device__ inline uint32_t lds4(const uint8_t *p) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uint32_t *w = reinterpret_cast<const uint32_t *>(a & ~uintptr_t(3));
    return __funnelshift_r(w[0], w[1], (uint32_t)(a & 3) * 8);
}

// popcount of bits [0, c) of node v (c <= n_v) from its rank directory
__device__ inline uint32_t rank1_dir(const DecSmem &S, const NodeSrc &src, const uint32_t *dir, int v, uint32_t c,
                                     uint32_t dir_bits) {
    const uint32_t nsb = (S.nv[v] + dir_bits - 1) / dir_bits;
    uint32_t sb = c / dir_bits;
    if (sb >= nsb) sb = nsb - 1;
    const uint32_t base = sb * dir_bits;
    uint32_t r = dir[sb];
    for (uint32_t e = base; e < c; e += 32) r += __popc(mask_valid(node_bits(S, src, v, e), (int64_t)c - e));
    return r;
}

// Per-block setup shared by the directory and merge: tree from the code
// lengths, node table and bitmap sources.  Returns 0 ok, 1 corrupt, 2
// workspace too small.  in_smem: the record is being bulk-copied into S.rec.
__device__ inline int block_setup(DecSmem &S, const uint8_t *rec_g, uint32_t rb, uint32_t n, uint32_t V, bool in_smem,
                                  uint64_t scratch_lim) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t < 128) {
        const uint8_t x = rec_g[kLensOff + t];
        S.lens[2 * t] = x & 15;
        S.lens[2 * t + 1] = x >> 4;
    }
    __syncthreads();
    build_tree_shape(S.lens, S.ts, S.codes, S.sorted, S.rank_scratch);
    if (!S.ts.ok || (uint32_t)S.ts.n_int != V) return 1;
    if (t < 17) S.first[t] = S.ts.first[t];
    if (t < (int)V) {
        const int d = node_depth(S.ts, t);
        S.depth[t] = (uint8_t)d;
        S.child[t][0] = (int16_t)node_child(S.ts, S.sorted, t, d, 0);
        S.child[t][1] = (int16_t)node_child(S.ts, S.sorted, t, d, 1);
        S.nv[t] = ld_le32(rec_g + kNvOff + 4 * t);
        S.marker[t] = rec_g[kNvOff + 4 * V + t];
    }
    __syncthreads();
    int bad = 0;
    if (t < (int)V) {
        const uint32_t nvv = S.nv[t];
        if (nvv < 2) bad = 1;
        for (int c = 0; c < 2; c++) {
            const int ch = S.child[t][c];
            if (ch >= 0 && S.nv[ch] > nvv) bad = 1;
        }
    }
    if (t == 0 && S.nv[0] != n) bad = 1;
    if (warp == 0) {
        const int Vi = (int)V;
        const uint32_t alen_off = (kNvOff + 5 * V + 3) & ~3u;
        const uint32_t nsel = warp_scan_loop_d(Vi, [&](int v) { return (uint32_t)(S.marker[v] != 0); },
                                               [&](int v, uint32_t p) { S.src_off[v] = p; });
        __syncwarp();
        for (int v = lane; v < Vi; v += 32) {
            const uint32_t raw = (S.nv[v] + 7) / 8;
            const uint32_t al = S.marker[v] ? ld_le32(rec_g + alen_off + 4 * S.src_off[v]) : raw;
            S.alen[v] = al;
            if (S.marker[v] == kMarkRawSel && al != raw) bad = 1;
            S.src_kind[v] = (S.marker[v] && S.marker[v] != kMarkRawSel) ? 2 : (in_smem ? 0 : 1);
        }
        __syncwarp();
        const uint32_t base1 = alen_off + 4 * nsel;
        const uint32_t raw_tot = warp_scan_loop_d(Vi, [&](int v) { return S.marker[v] ? 0u : S.alen[v]; },
                                                  [&](int v, uint32_t p) { if (!S.marker[v]) S.src_off[v] = base1 + p; });
        const uint32_t base2 = base1 + raw_tot;
        const uint32_t sel_tot = warp_scan_loop_d(Vi, [&](int v) { return S.marker[v] ? S.alen[v] : 0u; },
                                                  [&](int v, uint32_t p) { if (S.marker[v] == kMarkRawSel) S.src_off[v] = base2 + p; });
        const uint32_t scr_tot = warp_scan_loop_d(Vi, [&](int v) {
            return S.src_kind[v] == 2 ? scratch_stride((S.nv[v] + 7) / 8) : 0u;
        }, [&](int v, uint32_t p) { if (S.src_kind[v] == 2) S.src_off[v] = p; });
        if (lane == 0) {
            if (((base2 + sel_tot + 15u) & ~15u) != rb) bad = 1;
            if (scr_tot > scratch_lim) bad |= 2;
        }
    }
    bad = __syncthreads_or(bad);
    return (bad & 1) ? 1 : (bad ? 2 : 0);
}

// ---------------------------------------------------------------------------
// Rank directories and tile-boundary cursors of one block (whole CTA)
// ---------------------------------------------------------------------------
__device__ inline void dir_block(int b, const uint8_t *__restrict__ comp, const uint64_t *__restrict__ comp_off,
                                 int nblk, uint8_t *__restrict__ ws, uint64_t ws_bytes, int32_t *__restrict__ status,
                                 DecSmem &S) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const DecWs W = dec_ws(ws, nblk);
    const DecRegions G = dec_regions(nblk, ws);
    const uint32_t dir_bits = reinterpret_cast<const uint32_t *>(ws)[7];
    const uint32_t ntile = W.blk_ntile[b];
    if (ntile <= 1 || status[b] != PIVCO_OK) return;
    const uint8_t *rec_g = comp + comp_off[b];
    const uint32_t rb = ld_le32(rec_g), n = ld_le32(rec_g + 4);
    const uint32_t V = (uint32_t)rec_g[8] | ((uint32_t)rec_g[9] << 8);
    const uint64_t slim = ws_bytes > G.scratch + W.blk_scratch[b] ? ws_bytes - G.scratch - W.blk_scratch[b] : 0;
    const int bad = block_setup(S, rec_g, rb, n, V, false, slim);
    if (bad || G.dir + W.blk_dir[b] + 4ull * (ntile + 1) * V > ws_bytes) {
        if (t == 0) status[b] = bad == 1 ? PIVCO_ERR_CORRUPT : PIVCO_ERR_CAPACITY;
        __syncthreads();
        return;
    }
    NodeSrc src;
    src.rec_g = rec_g;
    src.rb = rb;
    src.scratch = ws + G.scratch + W.blk_scratch[b];
    src.scratch_lim = slim;
    uint32_t *dir = reinterpret_cast<uint32_t *>(ws + G.dir + W.blk_dir[b]);
    // superblocks per node
    if (warp == 0) {
        const uint32_t tot = warp_scan_loop_d((int)V, [&](int v) { return (S.nv[v] + dir_bits - 1) / dir_bits; },
                                              [&](int v, uint32_t p) { S.ustart[v] = p; });
        if (lane == 0) S.lvl_units[0] = tot;
    }
    __syncthreads();
    const uint32_t nsb = S.lvl_units[0];
    uint32_t *cursors = dir + nsb;
    if (G.dir + W.blk_dir[b] + 4ull * nsb + 4ull * (ntile + 1) * V > ws_bytes) {
        if (t == 0) status[b] = PIVCO_ERR_CAPACITY;
        __syncthreads();
        return;
    }
    for (uint32_t g = t; g < nsb; g += kDecThreads) {
        const int v = find_node_d(S.ustart, 0, (int)V, g);
        const uint32_t e0 = (g - S.ustart[v]) * dir_bits, nvv = S.nv[v];
        uint32_t pc = 0;
        for (uint32_t e = e0; e < e0 + dir_bits && e < nvv; e += 32)
            pc += __popc(mask_valid(node_bits(S, src, v, e), (int64_t)nvv - e));
        dir[g] = pc;
    }
    __syncthreads();
    for (int v = warp; v < (int)V; v += kDecWarps) {
        const uint32_t u0 = S.ustart[v], nu = (S.nv[v] + dir_bits - 1) / dir_bits;
        warp_scan_loop_d((int)nu, [&](int i) { return dir[u0 + i]; }, [&](int i, uint32_t p) { dir[u0 + i] = p; });
    }
    // boundary 0: all cursors 0; boundary ntile: n_v; root cursor at boundary k: k * T
    for (uint32_t v = t; v < V; v += kDecThreads) { cursors[v] = 0; cursors[(size_t)ntile * V + v] = S.nv[v]; }
    const uint32_t T = W.blk_T[b];
    for (uint32_t k = 1 + t; k < ntile; k += kDecThreads) cursors[(size_t)k * V] = k * T;
    __syncthreads();
    // top-down by depth: children's cursors from the parent's rank at its cursor
    const int maxd = S.ts.max_len;
    int bad2 = 0;
    for (int d = 0; d < maxd; d++) {
        const uint32_t f0 = S.first[d], nd = S.first[d + 1] - f0;
        for (uint32_t i = t; i < (ntile - 1) * nd; i += kDecThreads) {
            const uint32_t k = 1 + i / nd;
            const int v = (int)(f0 + i % nd);
            const uint32_t c = cursors[(size_t)k * V + v];
            if (c > S.nv[v]) { bad2 = 1; continue; }
            const uint32_t ones = rank1_dir(S, src, dir + S.ustart[v], v, c, dir_bits);
            const int c0 = S.child[v][0], c1 = S.child[v][1];
            if (c0 >= 0) cursors[(size_t)k * V + c0] = c - ones;
            if (c1 >= 0) cursors[(size_t)k * V + c1] = ones;
        }
        __syncthreads();
    }
    bad2 = __syncthreads_or(bad2);
    if (t == 0 && bad2) status[b] = PIVCO_ERR_CORRUPT;
    __syncthreads();
}

__global__ void __launch_bounds__(kDecThreads, 3) decode_dir_kernel(const uint8_t *__restrict__ comp,
                                                                    const uint64_t *__restrict__ comp_off, int nblk,
                                                                    uint8_t *__restrict__ ws, uint64_t ws_bytes,
                                                                    int32_t *__restrict__ status) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    DecSmem &S = *reinterpret_cast<DecSmem *>(smem_raw);
    const DecWs W = dec_ws(ws, nblk);
    for (int b = blockIdx.x; b < nblk; b += gridDim.x)
        if (W.blk_ntile[b] > 1) dir_block(b, comp, comp_off, nblk, ws, ws_bytes, status, S);
}

cudaError_t launch_decode_dir(const uint8_t *comp, const uint64_t *comp_off, int nblk, uint8_t *ws, size_t ws_bytes,
                              int32_t *status, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    const int smem = (int)sizeof(DecSmem);
    cudaError_t e = cudaFuncSetAttribute(decode_dir_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = nblk < sms * 3 ? nblk : sms * 3;
    decode_dir_kernel<<<grid, kDecThreads, smem, st>>>(comp, comp_off, nblk, ws, ws_bytes, status);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Merge
// ---------------------------------------------------------------------------
// merge every node of depth d for the current chunk: units g in [g0, g1)
__device__ inline void merge_level(DecSmem &S, const NodeSrc &src, int d, uint32_t g0, uint32_t g1, uint8_t *dst,
                                   uint32_t P, bool out4) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint8_t *bin = S.buf[(d + 1) & 1];
    uint8_t *bout = S.buf[d & 1];
    for (uint32_t g = g0 + warp; g < g1; g += kDecWarps) {
        const int v = S.umap[g];
        const uint32_t k0 = (g - S.ustart[v]) * kDUnit, k = k0 + 4 * lane;
        const uint32_t dv = S.dem[v], q = lane >> 3;
        const int64_t e = (int64_t)k0 + 32 * q;
        const uint32_t wq = e < dv ? mask_valid(node_bits(S, src, v, S.cur[v] + (uint32_t)e), (int64_t)dv - e) : 0u;
        const uint32_t w0 = __shfl_sync(0xffffffffu, wq, 0), w1 = __shfl_sync(0xffffffffu, wq, 8),
                       w2 = __shfl_sync(0xffffffffu, wq, 16);
        if (k >= dv) continue;
        const uint32_t r1 = S.ubase[g] + (q > 0 ? __popc(w0) : 0) + (q > 1 ? __popc(w1) : 0) + (q > 2 ? __popc(w2) : 0) +
                            __popc(wq & ((1u << (4 * (lane & 7))) - 1u));
        const uint32_t nib = (wq >> (4 * (lane & 7))) & 15u;
        const int c0 = S.child[v][0], c1 = S.child[v][1];
        const uint32_t xl = c0 >= 0 ? lds4(bin + S.span[c0] + (k - r1)) : (uint32_t)(-c0 - 1) * 0x01010101u;
        const uint32_t xr = c1 >= 0 ? lds4(bin + S.span[c1] + r1) : (uint32_t)(-c1 - 1) * 0x01010101u;
        const uint32_t o = __byte_perm(xl, xr, S.sel[(c0 >= 0) | ((c1 >= 0) << 1)][nib]);
        if (d > 0) {
            *reinterpret_cast<uint32_t *>(bout + S.span[v] + k) = o;
        } else {
            uint8_t *op = dst + P + k;
            if (out4 && k + 4 <= dv) *reinterpret_cast<uint32_t *>(op) = o;
            else for (uint32_t j = 0; j < 4 && k + j < dv; j++) op[j] = (uint8_t)(o >> (8 * j));
        }
    }
}

// One-time CTA setup of the merge: the mbarrier and the byte-permute selectors.
// Selector of output byte j for 4 bits `nib`: a one takes the next byte of the
// right window (bytes 4..7), a zero the next byte of the left window (bytes
// 0..3); a leaf side always takes its constant.
__device__ inline void merge_cta_init(DecSmem &S) {
    const int t = threadIdx.x;
    if (t == 0) mbar_init(&S.mbar, 1);
    if (t < 64) {
        const int kindsel = t >> 4, nib = t & 15;
        const bool lint = kindsel & 1, rint = kindsel & 2;
        uint32_t s = 0, ones = 0, zeros = 0;
        for (int j = 0; j < 4; j++) {
            const uint32_t bit = (nib >> j) & 1u;
            const uint32_t idx = bit ? (rint ? 4 + ones : 4) : (lint ? zeros : 0);
            s |= idx << (4 * j);
            ones += bit;
            zeros += 1 - bit;
        }
        S.sel[kindsel][nib] = s;
    }
    __syncthreads();
}

// unit popcounts and per-node scans of the current chunk's units [g0, g1) of
// the nodes [f0, f1); sets the children's demands when set_children, else
// checks them.  Returns nonzero on inconsistency.
__device__ inline int rank_units(DecSmem &S, const NodeSrc &src, int f0, int f1, uint32_t g0, uint32_t g1,
                                 bool set_children) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (uint32_t g = g0 + t; g < g1; g += kDecThreads) {
        const int v = find_node_d(S.ustart, f0, f1, g);
        const uint32_t k0 = (g - S.ustart[v]) * kDUnit, dv = S.dem[v], c = S.cur[v];
        uint32_t pc = 0;
#pragma unroll
        for (uint32_t q = 0; q < 4; q++) {
            const int64_t e = (int64_t)k0 + 32 * q;
            if (e < dv) pc += __popc(mask_valid(node_bits(S, src, v, c + (uint32_t)e), (int64_t)dv - e));
        }
        S.ubase[g] = pc;
        S.umap[g] = (uint8_t)v;
    }
    __syncthreads();
    int bad = 0;
    for (int v = f0 + warp; v < f1; v += kDecWarps) {
        const uint32_t dv = S.dem[v];
        uint32_t ones = 0;
        if (dv) {
            const uint32_t u0 = S.ustart[v], nu = (dv + kDUnit - 1) / kDUnit;
            ones = warp_scan_loop_d((int)nu, [&](int i) { return S.ubase[u0 + i]; },
                                    [&](int i, uint32_t p) { S.ubase[u0 + i] = p; });
        }
        if (lane < 2) {
            const int ch = S.child[v][lane];
            if (ch >= 0) {
                const uint32_t dc = lane ? ones : dv - ones;
                if (set_children) {
                    S.dem[ch] = dc;
                    if ((uint64_t)S.cur[ch] + dc > S.nv[ch]) bad = 1;
                } else if (S.dem[ch] != dc) {
                    bad = 1;
                }
            }
        }
    }
    return __syncthreads_or(bad);
}

// Decodes tile gt (whole CTA).  Returns false when a bounded wait expired
// (the CTA must stop; the affected blocks are marked).
__device__ inline bool tile_item(uint32_t gt, const uint8_t *__restrict__ comp, const uint64_t *__restrict__ comp_off,
                                 int nblk, uint8_t *__restrict__ out, const uint64_t *__restrict__ out_off,
                                 const uint8_t *__restrict__ ws, uint64_t ws_bytes, int32_t *__restrict__ status,
                                 DecSmem &S, uint32_t &phase) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const DecWs W = dec_ws(const_cast<uint8_t *>(ws), nblk);
    const DecRegions G = dec_regions(nblk, ws);
    const uint32_t dir_bits = reinterpret_cast<const uint32_t *>(ws)[7];
    const int b = find_block(W.blk_tile, nblk, gt);
    if (status[b] != PIVCO_OK) return true;   // the plan / ANS / directory pass already failed this block
    const uint32_t k = gt - W.blk_tile[b], ntile = W.blk_ntile[b], T = W.blk_T[b];
    const uint8_t *rec_g = comp + comp_off[b];
    uint8_t *dst = out + out_off[b];
    const uint64_t ocap = out_off[b + 1] - out_off[b];
    const uint32_t rb = ld_le32(rec_g), n = ld_le32(rec_g + 4);
    const uint32_t V = (uint32_t)rec_g[8] | ((uint32_t)rec_g[9] << 8), kind = rec_g[10], aux = rec_g[11];
    if ((comp_off[b] & 15) || n != ocap) {   // the plan validated magic / size / layout
        if (t == 0) status[b] = n != ocap ? PIVCO_ERR_CAPACITY : PIVCO_ERR_CORRUPT;
        return true;
    }
    if (kind == 0) return true;
    if (kind == 1) {
        for (uint32_t i = t; i < n; i += kDecThreads) dst[i] = (uint8_t)aux;
        return true;
    }
    const uint32_t P0 = k * T, P1 = min(n, P0 + T);
    // ---- record into shared memory (overlaps the tree construction) ----
    const bool in_smem = rb <= (uint32_t)kDRecSmem;
    if (in_smem && t == 0) {
        fence_proxy_async_smem();
        mbar_expect_tx(&S.mbar, rb);
        bulk_g2s(S.rec, rec_g, rb, &S.mbar);
    }
    const uint64_t slim = ws_bytes > G.scratch + W.blk_scratch[b] ? ws_bytes - G.scratch - W.blk_scratch[b] : 0;
    const int bad = block_setup(S, rec_g, rb, n, V, in_smem, slim);
    int timed_out = in_smem ? !mbar_wait(&S.mbar, phase) : 0;
    timed_out = __syncthreads_or(timed_out);
    if (timed_out) {
        mbar_wait(&S.mbar, phase);   // one more bounded wait for the copy before the CTA leaves
        if (t == 0) status[b] = PIVCO_ERR_TIMEOUT;
        return false;
    }
    if (in_smem) phase ^= 1;
    if (bad) {
        if (t == 0) status[b] = bad == 1 ? PIVCO_ERR_CORRUPT : PIVCO_ERR_CAPACITY;
        __syncthreads();
        return true;
    }
    NodeSrc src;
    src.rec_g = rec_g;
    src.rb = rb;
    src.scratch = ws + G.scratch + W.blk_scratch[b];
    src.scratch_lim = slim;
    const bool out4 = (reinterpret_cast<uintptr_t>(dst) & 3) == 0;
    const int maxd = S.ts.max_len;
    // ---- this tile's bit range of every node ----
    const uint32_t *cursors = nullptr;   // tile-boundary cursors follow the node directories
    if (warp == 0 && ntile > 1) {
        const uint32_t ent = warp_scan_loop_d((int)V, [&](int v) { return (S.nv[v] + dir_bits - 1) / dir_bits; },
                                              [&](int, uint32_t) {});
        if (lane == 0) S.lvl_units[16] = ent;
    }
    __syncthreads();
    if (ntile > 1) cursors = reinterpret_cast<const uint32_t *>(ws + G.dir + W.blk_dir[b]) + S.lvl_units[16];
    for (uint32_t v = t; v < V; v += kDecThreads) {
        const uint32_t cs = ntile > 1 ? cursors[(size_t)k * V + v] : 0u;
        const uint32_t ce = ntile > 1 ? cursors[(size_t)(k + 1) * V + v] : S.nv[v];
        S.cur[v] = cs;
        S.dem[v] = ce >= cs ? ce - cs : 0u;
        S.alen[v] = (ce < cs || ce > S.nv[v]) ? 1u : 0u;   // reused as a per-node error mark
    }
    if (t == 0) { S.flag = 0; S.overflow = 0; }
    __syncthreads();
    for (uint32_t v = t; v < V; v += kDecThreads)
        if (S.alen[v]) S.flag = 1;
    if (t == 0 && S.dem[0] != P1 - P0) S.flag = 1;
    // ---- fast path: spans and units of every depth at once ----
    for (int d = warp; d < maxd; d += kDecWarps) {
        const int f0 = S.first[d], f1 = S.first[d + 1];
        uint64_t carry = 0;
        for (int base = f0; base < f1; base += 32) {
            const int v = base + lane;
            const uint32_t dv = v < f1 ? S.dem[v] : 0u;
            const uint64_t x = ((uint64_t)((dv + kDUnit - 1) / kDUnit) << 32) | ((dv + 3u) & ~3u);
            uint64_t inc = x;
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            const uint64_t ex = carry + inc - x;
            if (v < f1) { S.span[v] = (uint32_t)ex; S.ustart[v] = (uint32_t)(ex >> 32); }
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (lane == 0) {
            S.lvl_units[d] = (uint32_t)(carry >> 32);
            if (d > 0 && (uint32_t)carry > (uint32_t)kDLvlCap) S.overflow = 1;
        }
    }
    __syncthreads();
    if (t == 0) {
        uint32_t acc = 0;
        for (int d = 0; d < maxd; d++) { const uint32_t u = S.lvl_units[d]; S.lvl_units[d] = acc; acc += u; }
        S.lvl_units[maxd] = acc;
        if (acc > (uint32_t)kDMaxUnits) S.overflow = 1;
    }
    __syncthreads();
    if (S.flag) {
        if (t == 0) status[b] = PIVCO_ERR_CORRUPT;
        __syncthreads();
        return true;
    }
    if (!S.overflow) {
        for (uint32_t v = t; v < V; v += kDecThreads) S.ustart[v] += S.lvl_units[S.depth[v]];
        __syncthreads();
        if (rank_units(S, src, 0, (int)V, 0, S.lvl_units[maxd], false)) {
            if (t == 0) status[b] = PIVCO_ERR_CORRUPT;
            __syncthreads();
            return true;
        }
        for (int d = maxd - 1; d >= 0; d--) {
            merge_level(S, src, d, S.lvl_units[d], S.lvl_units[d + 1], dst, P0, out4);
            __syncthreads();
        }
    } else {
        // ---- fallback: chunks whose bit ranges are found top-down ----
        if (t == 0) S.chunk = max((uint32_t)kDUnit, ((P1 - P0) / 2) & ~(uint32_t)(kDUnit - 1));
        __syncthreads();
        for (uint32_t P = P0; P < P1;) {
            const uint32_t cc = min(S.chunk, P1 - P);
            if (t == 0) { S.dem[0] = cc; S.lvl_units[0] = 0; S.overflow = 0; }
            __syncthreads();
            for (int d = 0; d < maxd; d++) {
                const int f0 = S.first[d], f1 = S.first[d + 1];
                if (warp == 0) {
                    const uint32_t u0 = S.lvl_units[d];
                    uint64_t carry = 0;
                    for (int base = f0; base < f1; base += 32) {
                        const int v = base + lane;
                        const uint32_t dv = v < f1 ? S.dem[v] : 0u;
                        const uint64_t x = ((uint64_t)((dv + kDUnit - 1) / kDUnit) << 32) | ((dv + 3u) & ~3u);
                        uint64_t inc = x;
                        for (int o = 1; o < 32; o <<= 1) {
                            const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
                            if (lane >= o) inc += y;
                        }
                        const uint64_t ex = carry + inc - x;
                        if (v < f1) { S.span[v] = (uint32_t)ex; S.ustart[v] = u0 + (uint32_t)(ex >> 32); }
                        carry += __shfl_sync(0xffffffffu, inc, 31);
                    }
                    if (lane == 0) {
                        S.lvl_units[d + 1] = u0 + (uint32_t)(carry >> 32);
                        if (d > 0 && (uint32_t)carry > (uint32_t)kDLvlCap) S.overflow = 1;
                        if (S.lvl_units[d + 1] > (uint32_t)kDMaxUnits) S.overflow = 1;
                    }
                }
                __syncthreads();
                if (S.overflow) break;
                if (rank_units(S, src, f0, f1, S.lvl_units[d], S.lvl_units[d + 1], true)) {
                    if (t == 0) S.flag = 1;
                }
                __syncthreads();
                if (S.flag) break;
            }
            if (S.flag) break;
            if (S.overflow) {
                if (t == 0) S.chunk = max((uint32_t)kDUnit, (S.chunk / 4 * 3) & ~(uint32_t)(kDUnit - 1));
                __syncthreads();
                continue;
            }
            for (int d = maxd - 1; d >= 0; d--) {
                merge_level(S, src, d, S.lvl_units[d], S.lvl_units[d + 1], dst, P, out4);
                __syncthreads();
            }
            for (uint32_t v = t; v < V; v += kDecThreads) S.cur[v] += S.dem[v];
            P += cc;
            __syncthreads();
        }
        // the chunks must end exactly at the tile's end cursors
        if (!S.flag) {
            for (uint32_t v = t; v < V; v += kDecThreads) {
                const uint32_t ce = ntile > 1 ? cursors[(size_t)(k + 1) * V + v] : S.nv[v];
                if (S.cur[v] != ce) S.flag = 1;
            }
        }
        __syncthreads();
        if (S.flag) {
            if (t == 0) status[b] = PIVCO_ERR_CORRUPT;
            __syncthreads();
            return true;
        }
    }
    // the last tile checks the pad bits of every bitmap
    if (k + 1 == ntile) {
        int bad_end = 0;
        for (uint32_t v = t; v < V && !bad_end; v += kDecThreads) {
            if (S.nv[v] & 7) {
                const uint32_t last = node_bits(S, src, (int)v, S.nv[v] & ~7u) & 0xFFu;
                if (last >> (S.nv[v] & 7)) bad_end = 1;
            }
        }
        bad_end = __syncthreads_or(bad_end);
        if (t == 0 && bad_end) status[b] = PIVCO_ERR_CORRUPT;
    }
    __syncthreads();
    return true;
}

__global__ void __launch_bounds__(kDecThreads, 3) decode_kernel(const uint8_t *__restrict__ comp,
                                                                const uint64_t *__restrict__ comp_off,
                                                                int nblk, uint8_t *__restrict__ out,
                                                                const uint64_t *__restrict__ out_off,
                                                                const uint8_t *__restrict__ ws, uint64_t ws_bytes,
                                                                int32_t *__restrict__ status) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    DecSmem &S = *reinterpret_cast<DecSmem *>(smem_raw);
    merge_cta_init(S);
    uint32_t phase = 0;
    const uint32_t total_tiles = reinterpret_cast<const uint32_t *>(ws)[6];
    for (uint32_t gt = blockIdx.x; gt < total_tiles; gt += gridDim.x)
        if (!tile_item(gt, comp, comp_off, nblk, out, out_off, ws, ws_bytes, status, S, phase)) return;
}

// ---------------------------------------------------------------------------
// Batched decode: one persistent launch over a work queue keyed by
// (block, stage).  Items, in queue order:
//   plans      8 blocks per item, one warp each (ticket order = block order,
//              as the plan's look-back needs)
//   ANS        8 segments per item, one warp each
//   directory  one block per item (blocks with one tile skip it)
//   tiles      one tile per item
// An item only waits (bounded) on items earlier in the queue: the ANS and
// later items on all plans; a directory on its block's ANS segments; a tile
// on its block's ANS segments and directory.  CTAs that took those items are
// running, so every wait ends.
// ---------------------------------------------------------------------------
__device__ inline bool wait_geq(const uint32_t *p, uint32_t want) {
    if (*reinterpret_cast<const volatile uint32_t *>(p) >= want) { __threadfence(); return true; }
    const uint64_t t0 = globaltimer_ns();
    unsigned ns = 64;
    while (*reinterpret_cast<const volatile uint32_t *>(p) < want) {
        if (globaltimer_ns() - t0 > kWaitLimitNs) return false;
        __nanosleep(ns);
        if (ns < 2048) ns <<= 1;
    }
    __threadfence();
    return true;
}

union BatchSmem {
    DecSmem dec;
    struct {
        WarpRec R[kDecWarps];
        PlanScratch Q[kDecWarps];
        AnsSm T[kDecWarps];
    } w;
};

// plan / ANS items only overwrite the per-tile part of the merge's state
static_assert(offsetof(DecSmem, sel) >= sizeof(((BatchSmem *)0)->w), "batch scratch overlaps the selectors");
static_assert(offsetof(DecSmem, mbar) >= sizeof(((BatchSmem *)0)->w), "batch scratch overlaps the mbarrier");

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

// Items of a batch's queue once all plans are done (header written by the last plan).
__device__ inline uint32_t batch_items_total(const BatchQueue &q) {
    const uint32_t *hdr = reinterpret_cast<const uint32_t *>(q.ws);
    const uint32_t nplan = (uint32_t)((q.nblk + kDecWarps - 1) / kDecWarps);
    return nplan + (hdr[2] + kDecWarps - 1) / kDecWarps + (uint32_t)q.nblk + hdr[6];
}

enum : int { kItemDone = 0, kItemNone = 1, kItemStop = 2 };

// Runs item `item` of the queue with the whole CTA.  kItemDone: processed;
// kItemNone: past the end of the queue; kItemStop: a bounded wait expired in a
// way that leaves this CTA's shared memory unsafe to reuse (a bulk copy may
// still be in flight), so the CTA must stop.  Statuses of affected blocks are set.
__device__ inline int batch_item(const BatchQueue &q, uint32_t item, BatchSmem &B, const AnsTables &A,
                                 uint32_t &phase, int &last_b, bool &last_ok) {
    DecSmem &S = B.dec;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int nblk = q.nblk;
    uint32_t *hdr = reinterpret_cast<uint32_t *>(q.ws);
    const DecWs W = dec_ws(q.ws, nblk);
    const uint32_t nplan = (uint32_t)((nblk + kDecWarps - 1) / kDecWarps);
    if (item < nplan) {
        // ---- plans ----
        const int b = (int)(item * kDecWarps + warp);
        if (b < nblk) plan_block(b, q.comp, q.comp_off, nblk, q.ws, q.status, B.w.R[warp], B.w.Q[warp]);
        __syncthreads();
        if (t == 0) { __threadfence(); atomicAdd(&hdr[10], 1u); }
        return kItemDone;
    }
    // everything after the plans needs all plans
    int ok = 1;
    if (t == 0) ok = wait_geq(&hdr[10], nplan);
    if (__syncthreads_or(!ok)) {
        if (t == 0) for (int b = 0; b < nblk; b++) if (q.status[b] == PIVCO_OK) q.status[b] = PIVCO_ERR_TIMEOUT;
        __syncthreads();
        return kItemStop;
    }
    const uint32_t total_segs = hdr[2], total_tiles = hdr[6];
    const uint32_t nseg_items = (total_segs + kDecWarps - 1) / kDecWarps;
    uint32_t it = item - nplan;
    if (it < nseg_items) {
        // ---- ANS segments ----
        const uint32_t g = it * kDecWarps + warp;
        if (g < total_segs) {
            const int b = ans_item(g, q.comp, q.comp_off, nblk, q.ws, q.ws_bytes, q.status, A, B.w.R[warp],
                                   B.w.T[warp], last_b, last_ok);
            if (lane == 0) { __threadfence(); atomicAdd(&W.segs_done[b], 1u); }
        }
        __syncthreads();
        last_b = -1;   // the cached record may be overwritten by a later tile item
        return kItemDone;
    }
    it -= nseg_items;
    if (it < (uint32_t)nblk) {
        // ---- directory of block it ----
        const int b = (int)it;
        if (W.blk_ntile[b] > 1) {
            const uint32_t nsegs = (b + 1 < nblk ? W.blk_seg[b + 1] : total_segs) - W.blk_seg[b];
            int okw = 1;
            if (t == 0) okw = wait_geq(&W.segs_done[b], nsegs);
            if (__syncthreads_or(!okw)) {
                if (t == 0) q.status[b] = PIVCO_ERR_TIMEOUT;
            } else {
                dir_block(b, q.comp, q.comp_off, nblk, q.ws, q.ws_bytes, q.status, S);
            }
            __syncthreads();
            if (t == 0) { __threadfence(); atomicExch(&W.dir_done[b], 1u); }
        }
        return kItemDone;
    }
    it -= (uint32_t)nblk;
    if (it >= total_tiles) return kItemNone;
    // ---- tile it ----
    const int b = find_block(W.blk_tile, nblk, it);
    const uint32_t nsegs = (b + 1 < nblk ? W.blk_seg[b + 1] : total_segs) - W.blk_seg[b];
    int okw = 1;
    if (t == 0) {
        okw = wait_geq(&W.segs_done[b], nsegs);
        if (okw && W.blk_ntile[b] > 1) okw = wait_geq(&W.dir_done[b], 1u);
    }
    if (__syncthreads_or(!okw)) {
        if (t == 0) q.status[b] = PIVCO_ERR_TIMEOUT;
        __syncthreads();
        return kItemDone;
    }
    return tile_item(it, q.comp, q.comp_off, nblk, q.out, q.out_off, q.ws, q.ws_bytes, q.status, S, phase)
               ? kItemDone : kItemStop;
}

__global__ void __launch_bounds__(kDecThreads, 3) decode_batch_kernel(const uint8_t *__restrict__ comp,
                                                                      const uint64_t *__restrict__ comp_off, int nblk,
                                                                      uint8_t *__restrict__ out,
                                                                      const uint64_t *__restrict__ out_off,
                                                                      uint8_t *__restrict__ ws, uint64_t ws_bytes,
                                                                      int32_t *__restrict__ status,
                                                                      const __grid_constant__ AnsTables A) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    BatchSmem &B = *reinterpret_cast<BatchSmem *>(smem_raw);
    DecSmem &S = B.dec;
    const BatchQueue q{comp, comp_off, out, out_off, ws, ws_bytes, status, nblk};
    uint32_t *hdr = reinterpret_cast<uint32_t *>(ws);
    merge_cta_init(S);
    uint32_t phase = 0;
    int last_b = -1;
    bool last_ok = false;
    for (;;) {
        if (threadIdx.x == 0) S.item = atomicAdd(&hdr[9], 1u);
        __syncthreads();
        const uint32_t item = S.item;
        __syncthreads();
        if (batch_item(q, item, B, A, phase, last_b, last_ok) != kItemDone) return;
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

__global__ void __launch_bounds__(kDecThreads, 3) serve_loop_kernel(ServeCtl *__restrict__ ctl,
                                                                    const ServeDesc *__restrict__ ring,
                                                                    ServeFlags *flags, uint64_t idle_ns,
                                                                    uint64_t life_ns,
                                                                    const __grid_constant__ AnsTables A) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    BatchSmem &B = *reinterpret_cast<BatchSmem *>(smem_raw);
    __shared__ ServeDesc D;
    __shared__ uint32_t s_cmd, s_item, s_r;
    const int t = threadIdx.x;
    merge_cta_init(B.dec);
    uint32_t phase = 0;
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
        const int res = batch_item(q, item, B, A, phase, last_b, last_ok);
        if (res == kItemNone) {
            if (t == 0) atomicCAS(&ctl->cur, r, r + 1);
            __syncthreads();
            continue;
        }
        if (t == 0) {
            uint32_t *hdr = reinterpret_cast<uint32_t *>(q.ws);
            __threadfence();
            const uint32_t n = atomicAdd(&hdr[11], 1u) + 1;
            const uint32_t nplan = (uint32_t)((q.nblk + kDecWarps - 1) / kDecWarps);
            if (*reinterpret_cast<volatile uint32_t *>(&hdr[10]) >= nplan) {
                __threadfence();
                if (n == batch_items_total(q)) {
                    int32_t worst = PIVCO_OK;
                    for (int b = 0; b < q.nblk && worst == PIVCO_OK; b++)
                        worst = *reinterpret_cast<volatile int32_t *>(&q.status[b]);
                    flags->worst[r % kServeRing] = worst;
                    __threadfence_system();
                    st_release_sys_u32(&flags->done[r % kServeRing], r + 1);
                }
            }
        }
        if (res == kItemStop) return;   // its shared memory may still receive a bulk copy
        __syncthreads();
    }
}

// Host: an upper bound, from host copies of the records, of the workspace the
// decode of these blocks needs under tuning `tu` (never below what the plan
// computes for valid records): the scratch of every ANS-coded node exactly,
// and rank directories plus tile cursors for the most tiles the plan can
// choose (a level of a valid record holds at most n symbols).
size_t decode_ws_bound(const uint8_t *comp, const uint64_t *comp_off, int nblk, const DecTuning &tu) {
    uint64_t dir = 0, scratch = 0;
    const uint64_t t_fit = ((uint64_t)(kDLvlCap - 4 * 256) / 5 * 4) & ~(uint64_t)(kDUnit - 1);
    uint64_t t_min = tu.tile_max < t_fit ? tu.tile_max : t_fit;
    if (t_min < (uint64_t)kDUnit) t_min = kDUnit;
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
            if (m && m != kMarkRawSel) scratch += scratch_stride((nv + 7) / 8);
        }
        const uint64_t ntile = ((uint64_t)n + t_min - 1) / t_min;
        dir += (4 * ent + 4 * (ntile + 1) * V + 15) & ~(uint64_t)15;
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
    const int smem = (int)sizeof(DecSmem);
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
    const DecTuning &tu = current_tuning();
    dec_ws_init_kernel<<<min(1024, div_up(nblk, 256)), 256, 0, st>>>(ws, nblk, tu.dir_bits, tu.tile_max);
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
    cudaError_t e = cudaFuncSetAttribute(decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(DecSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(decode_dir_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(DecSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(decode_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BatchSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(serve_loop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BatchSmem));
    return e;
}
}  // namespace pv
