// Decode kernel: bottom-up merge through per-node rank directories (Sec. 3).
//
// Persistent CTAs; each decodes whole blocks.  A record that fits is copied
// into shared memory with one bulk (TMA 1D) copy while the CTA rebuilds the
// canonical tree from the code lengths; larger records and ANS-decoded
// bitmaps are read through L1/L2.
//
// A block is decoded in root chunks.  The root's symbols go straight to the
// output; only depths >= 1 need level buffers, so a chunk can be as long as
// the busiest level below the root allows (for skewed data a whole block).
// For a chunk, every internal node v needs a contiguous range of its bitmap
// starting at its cursor c_v; its length d_v is the number of the chunk's
// symbols whose code passes through v.  Top-down (demand pass) each node's
// range is popcounted per 128-bit unit; the exclusive per-unit popcounts are
// the node's rank directory for the chunk (rank1 of an element = unit base +
// popcount inside the unit), and the node's total is its right child's
// demand.  Bottom-up (merge pass, deepest level first) every node rebuilds
// its symbol sequence out_v[k] = bit ? R[rank1(k)] : L[k - rank1(k)] from its
// children's sequences or leaf constants (MVV / MCV / MVC / MCC of Table 8):
// each lane merges 4 symbols with one byte permute whose selector depends
// only on the lane's 4 bits.
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

struct DecSmem {
    uint8_t rec[kDRecSmem];          // record copy (bulk copy destination, 16-aligned)
    uint8_t buf[2][kDLvlBytes];      // level buffers (depth d uses buf[d & 1])
    uint32_t ubase[kDMaxUnits];      // unit popcount, then the unit's rank base within its node
    uint8_t umap[kDMaxUnits];        // unit -> node
    uint32_t sel[4][16];             // byte-permute selectors by (node kind, 4 bits)
    uint32_t cur[256];               // bits of node v consumed by earlier chunks
    uint32_t dem[256];               // bits of node v used by this chunk
    uint32_t span[256];              // span of node v in its level buffer
    uint32_t ustart[256];            // first unit of node v (chunk numbering)
    uint32_t nv[256];
    uint32_t src_off[256];           // bitmap start: record byte offset or scratch offset
    uint32_t alen[256];              // body bytes of node v
    uint32_t lvl_units[17];
    uint32_t lvl_tot[17];            // symbols through the nodes of each depth (whole block)
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
    int32_t overflow;                // chunk too long for the level buffers
    uint32_t chunk;                  // current chunk length
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

// 32 bits starting at bit `bit` of a 16-byte-aligned byte array of `limit`
// bytes (aligned words at or past `limit` read as 0)
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

__global__ void __launch_bounds__(kDecThreads, 3) decode_kernel(const uint8_t *__restrict__ comp,
                                                                const uint64_t *__restrict__ comp_off,
                                                                int nblk, uint8_t *__restrict__ out,
                                                                const uint64_t *__restrict__ out_off,
                                                                const uint8_t *__restrict__ ws, uint64_t ws_bytes,
                                                                int32_t *__restrict__ status) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    DecSmem &S = *reinterpret_cast<DecSmem *>(smem_raw);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) mbar_init(&S.mbar, 1);
    if (t < 64) {
        // selector of output byte j for 4 bits `nib`: a one takes the next
        // byte of the right window (bytes 4..7), a zero the next byte of the
        // left window (bytes 0..3); a leaf side always takes its constant
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
    uint32_t phase = 0;
    const uint32_t total_segs = reinterpret_cast<const uint32_t *>(ws)[2];
    const uint64_t *blk_scratch = reinterpret_cast<const uint64_t *>(ws + 64) + nblk;
    const uint64_t dstart = (decode_ws_fixed_bytes(nblk) + 16ull * total_segs + 255) & ~255ull;

    for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
        if (status[b] != PIVCO_OK) continue;   // the plan / ANS pass already failed this block
        const uint8_t *rec_g = comp + comp_off[b];
        const uint64_t avail = comp_off[b + 1] - comp_off[b];
        uint8_t *dst = out + out_off[b];
        const uint64_t ocap = out_off[b + 1] - out_off[b];
        const uint32_t rb = ld_le32(rec_g), n = ld_le32(rec_g + 4);
        const uint32_t V = (uint32_t)rec_g[8] | ((uint32_t)rec_g[9] << 8), kind = rec_g[10], aux = rec_g[11];
        if ((comp_off[b] & 15) || n != ocap || rb > avail) {   // the plan validated magic / size / layout
            if (t == 0) status[b] = n != ocap ? PIVCO_ERR_CAPACITY : PIVCO_ERR_CORRUPT;
            continue;
        }
        if (kind == 0) {
            if (t == 0 && (n != 0 || V != 0 || aux != 0 || rb != kHdr)) status[b] = PIVCO_ERR_CORRUPT;
            continue;
        }
        if (kind == 1) {
            if (n == 0 || V != 0 || rb != kHdr) { if (t == 0) status[b] = PIVCO_ERR_CORRUPT; continue; }
            for (uint32_t i = t; i < n; i += kDecThreads) dst[i] = (uint8_t)aux;
            continue;
        }
        if (aux != 0 || n == 0) { if (t == 0) status[b] = PIVCO_ERR_CORRUPT; continue; }
        // ---- record into shared memory (overlaps the tree construction) ----
        const bool in_smem = rb <= (uint32_t)kDRecSmem;
        if (in_smem && t == 0) {
            fence_proxy_async_smem();
            mbar_expect_tx(&S.mbar, rb);
            bulk_g2s(S.rec, rec_g, rb, &S.mbar);
        }
        if (t < 128) {
            const uint8_t x = rec_g[kLensOff + t];
            S.lens[2 * t] = x & 15;
            S.lens[2 * t + 1] = x >> 4;
        }
        if (t == 0) S.flag = 0;
        __syncthreads();
        build_tree_shape(S.lens, S.ts, S.codes, S.sorted, S.rank_scratch);
        const int bad_tree = !S.ts.ok || (uint32_t)S.ts.n_int != V;
        const int maxd = S.ts.max_len;
        if (!bad_tree) {
            if (t < 17) { S.first[t] = S.ts.first[t]; S.lvl_tot[t] = 0; }
            if (t < (int)V) {
                const int d = node_depth(S.ts, t);
                S.depth[t] = (uint8_t)d;
                S.child[t][0] = (int16_t)node_child(S.ts, S.sorted, t, d, 0);
                S.child[t][1] = (int16_t)node_child(S.ts, S.sorted, t, d, 1);
                S.nv[t] = ld_le32(rec_g + kNvOff + 4 * t);
                S.marker[t] = rec_g[kNvOff + 4 * V + t];
                S.cur[t] = 0;
            }
        }
        __syncthreads();
        // per-node checks, per-depth symbol totals, body offsets (raw region, then
        // the selected region) and scratch offsets of the ANS-decoded bitmaps
        int bad = 0;
        if (!bad_tree) {
            if (t < (int)V) {
                const uint32_t nvv = S.nv[t];
                if (nvv < 2) bad = 1;
                for (int c = 0; c < 2; c++) {
                    const int ch = S.child[t][c];
                    if (ch >= 0) {
                        if (S.nv[ch] > nvv) bad = 1;
                        atomicAdd(&S.lvl_tot[S.depth[ch]], S.nv[ch]);
                    }
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
                    return S.src_kind[v] == 2 ? ((((S.nv[v] + 7) / 8) + 15u) & ~15u) + 16u : 0u;
                }, [&](int v, uint32_t p) { if (S.src_kind[v] == 2) S.src_off[v] = p; });
                if (lane == 0) {
                    if (((base2 + sel_tot + 15u) & ~15u) != rb) bad = 1;
                    if (scr_tot && (dstart + blk_scratch[b] + scr_tot > ws_bytes ||
                                    decode_ws_fixed_bytes(nblk) + 16ull * total_segs > ws_bytes))
                        bad |= 2;
                }
            }
        }
        bad = __syncthreads_or(bad);
        if (t == 0 && !bad_tree) {
            uint64_t mx = 1;
            for (int d = 1; d < 16; d++) mx = S.lvl_tot[d] > mx ? S.lvl_tot[d] : mx;
            // the busiest level of a chunk of X symbols is about X * mx / n (a chunk
            // that overflows the level buffers is shortened and redone)
            uint64_t X = (uint64_t)(kDLvlCap - 4 * 256) * n / mx;
            X = X > (uint64_t)kDMaxRoot ? (uint64_t)kDMaxRoot : X;
            X = X < n ? (X & ~(uint64_t)(kDUnit - 1)) : n;
            S.chunk = X < (uint64_t)kDUnit ? (uint32_t)kDUnit : (uint32_t)X;
            S.flag = (bad & 1) ? 1 : (bad ? 2 : 0);
        }
        int timed_out = in_smem ? !mbar_wait(&S.mbar, phase) : 0;
        timed_out = __syncthreads_or(timed_out);
        if (timed_out) {
            // bounded wait expired: give the copy one more bounded wait, then stop this CTA
            mbar_wait(&S.mbar, phase);
            if (t == 0) for (int bb = b; bb < nblk; bb += gridDim.x) status[bb] = PIVCO_ERR_TIMEOUT;
            return;
        }
        if (in_smem) phase ^= 1;
        if (bad_tree || S.flag) {
            if (t == 0) status[b] = (!bad_tree && S.flag == 2) ? PIVCO_ERR_CAPACITY : PIVCO_ERR_CORRUPT;
            __syncthreads();
            continue;
        }
        NodeSrc src;
        src.rec_g = rec_g;
        src.rb = rb;
        src.scratch = ws + dstart + blk_scratch[b];
        src.scratch_lim = ws_bytes > dstart + blk_scratch[b] ? ws_bytes - dstart - blk_scratch[b] : 0;
        const bool out4 = (reinterpret_cast<uintptr_t>(dst) & 3) == 0;

        for (uint32_t P = 0; P < n;) {
            // ---------------- demand pass (top-down) ----------------
            const uint32_t cc = min(S.chunk, n - P);
            if (t == 0) { S.dem[0] = cc; S.lvl_units[0] = 0; S.overflow = 0; }
            __syncthreads();
            for (int d = 0; d < maxd; d++) {
                const int f0 = S.first[d], f1 = S.first[d + 1];
                if (warp == 0) {
                    // one scan of (span bytes, units) pairs over the depth's nodes
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
                // unit -> node map and unit popcounts
                for (uint32_t g = S.lvl_units[d] + t; g < S.lvl_units[d + 1]; g += kDecThreads) {
                    const int v = find_node_d(S.ustart, f0, f1, g);
                    S.umap[g] = (uint8_t)v;
                    const uint32_t k0 = (g - S.ustart[v]) * kDUnit, dv = S.dem[v], c = S.cur[v];
                    uint32_t pc = 0;
#pragma unroll
                    for (uint32_t q = 0; q < 4; q++) {
                        const int64_t e = (int64_t)k0 + 32 * q;
                        if (e < dv) pc += __popc(mask_valid(node_bits(S, src, v, c + (uint32_t)e), (int64_t)dv - e));
                    }
                    S.ubase[g] = pc;
                }
                __syncthreads();
                // rank directory: per-node exclusive scan of the unit popcounts; children's demands
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
                            S.dem[ch] = dc;
                            if ((uint64_t)S.cur[ch] + dc > S.nv[ch]) S.flag = 1;
                        }
                    }
                }
                __syncthreads();
                if (S.flag) break;
            }
            if (S.flag) break;
            if (S.overflow) {
                // the chunk would not fit the level buffers: halve it and redo the demand pass
                if (t == 0) S.chunk = max((uint32_t)kDUnit, (S.chunk / 4 * 3) & ~(uint32_t)(kDUnit - 1));
                __syncthreads();
                continue;
            }
            // ---------------- merge pass (bottom-up) ----------------
            for (int d = maxd - 1; d >= 0; d--) {
                const uint8_t *bin = S.buf[(d + 1) & 1];
                uint8_t *bout = S.buf[d & 1];
                const uint32_t g1 = S.lvl_units[d + 1];
                for (uint32_t g = S.lvl_units[d] + warp; g < g1; g += kDecWarps) {
                    const int v = S.umap[g];
                    const uint32_t k0 = (g - S.ustart[v]) * kDUnit, k = k0 + 4 * lane;
                    const uint32_t dv = S.dem[v], q = lane >> 3;
                    const int64_t e = (int64_t)k0 + 32 * q;
                    const uint32_t wq = e < dv ? mask_valid(node_bits(S, src, v, S.cur[v] + (uint32_t)e), (int64_t)dv - e) : 0u;
                    const uint32_t w0 = __shfl_sync(0xffffffffu, wq, 0), w1 = __shfl_sync(0xffffffffu, wq, 8),
                                   w2 = __shfl_sync(0xffffffffu, wq, 16);
                    if (k >= dv) continue;
                    const uint32_t r1 = S.ubase[g] + (q > 0 ? __popc(w0) : 0) + (q > 1 ? __popc(w1) : 0) +
                                        (q > 2 ? __popc(w2) : 0) + __popc(wq & ((1u << (4 * (lane & 7))) - 1u));
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
                __syncthreads();
            }
            for (uint32_t v = t; v < V; v += kDecThreads) S.cur[v] += S.dem[v];
            P += cc;
            __syncthreads();
        }
        // every node's bitmap must be consumed exactly; pad bits must be zero
        int bad_end = S.flag;
        for (uint32_t v = t; v < V && !bad_end; v += kDecThreads) {
            if (S.cur[v] != S.nv[v]) bad_end = 1;
            else if (S.nv[v] & 7) {
                const uint32_t last = node_bits(S, src, (int)v, S.nv[v] & ~7u) & 0xFFu;
                if (last >> (S.nv[v] & 7)) bad_end = 1;
            }
        }
        bad_end = __syncthreads_or(bad_end);
        if (t == 0 && bad_end) status[b] = PIVCO_ERR_CORRUPT;
    }
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
    const int smem = (int)sizeof(DecSmem);
    cudaError_t e = cudaFuncSetAttribute(decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, decode_kernel, kDecThreads, smem);
    if (occ < 1) occ = 1;
    const int grid = nblk < sms * occ ? nblk : sms * occ;
    decode_kernel<<<grid, kDecThreads, smem, st>>>(comp, comp_off, nblk, out, out_off, ws, ws_bytes, status);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pv
