// Encode-side statistics and code construction kernels:
//   histogram      -- per-block byte counts (Sec. 4: dominates end-to-end encode)
//   code_lengths   -- optimal length-limited lengths by package-merge (App. D, L = 11)
//   build_layout   -- canonical codes, breadth-first node table, n_v, ANS
//                     selection (Sec. 5.2) and the record layout (App. D)
#include "pivco_dev.cuh"

namespace pv {

// ---------------------------------------------------------------------------
// Histogram.  Grid (nblk, slices); each CTA counts one slice of one block.
// Per-warp shared histograms.  Skewed data (P(top) up to 0.95) would
// serialise on the most frequent byte's counter, so each warp samples its
// most frequent byte and counts it in 32 per-lane counters (bins 256 + lane,
// one bank each), summed into its bin at the end; every byte is one
// shared-memory add, with no branch.
// ---------------------------------------------------------------------------
constexpr int kHistThreads = 256;
constexpr int kHistWarps = kHistThreads / 32;
constexpr int kHistBins = 256 + 32;

__global__ void zero_u32_kernel(uint32_t *p, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = 0;
}

// counts byte v: the hot byte in the lane's own counter
__device__ inline void hist_add_byte(uint32_t v, uint32_t hot, uint32_t hot_bin, uint32_t *wh) {
    atomicAdd(&wh[v == hot ? hot_bin : v], 1u);
}
__device__ inline void hist_add_word(uint32_t w, uint32_t hot, uint32_t hot_bin, uint32_t *wh) {
#pragma unroll
    for (int k = 0; k < 4; k++) hist_add_byte(__byte_perm(w, 0u, 0x4440u + k), hot, hot_bin, wh);
}
__device__ inline void hist_add_vec(const uint4 &q, uint32_t hot, uint32_t hot_bin, uint32_t *wh) {
    hist_add_word(q.x, hot, hot_bin, wh);
    hist_add_word(q.y, hot, hot_bin, wh);
    hist_add_word(q.z, hot, hot_bin, wh);
    hist_add_word(q.w, hot, hot_bin, wh);
}

// The most frequent of 32 samples of in[lo, hi) (warp-uniform; 0 when empty)
__device__ inline uint32_t hist_hot_byte(const uint8_t *__restrict__ in, uint64_t lo, uint64_t hi) {
    const int lane = threadIdx.x & 31;
    if (hi <= lo) return 0;
    const uint64_t pos = lo + ((uint64_t)lane * 2654435761u) % (hi - lo);
    const uint32_t v = in[pos];
    const uint32_t peers = __match_any_sync(0xffffffffu, v);
    int best = __popc(peers), bl = lane;
    for (int o = 16; o; o >>= 1) {
        const int ob = __shfl_xor_sync(0xffffffffu, best, o), ol = __shfl_xor_sync(0xffffffffu, bl, o);
        if (ob > best || (ob == best && ol < bl)) { best = ob; bl = ol; }
    }
    return __shfl_sync(0xffffffffu, v, bl);
}

// Counts in[lo, hi) into the warp's histogram my (kHistBins, zeroed) with
// stride-`step` work sharing starting at `first` (lane or thread index):
// head bytes up to 16-byte alignment, 16-byte loads four in flight, the tail.
__device__ inline void hist_range(const uint8_t *__restrict__ in, uint64_t lo, uint64_t hi, uint32_t first,
                                  uint32_t step, uint32_t hot, uint32_t *my) {
    const uint32_t hot_bin = 256u + (threadIdx.x & 31);
    // (the 16-byte boundary of the address: `in` itself may be unaligned)
    uint64_t a = lo + ((16u - (uint32_t)(reinterpret_cast<uintptr_t>(in + lo) & 15u)) & 15u);
    if (a > hi) a = hi;
    for (uint64_t i = lo + first; i < a; i += step) hist_add_byte(in[i], hot, hot_bin, my);
    const uint64_t nvec = (hi - a) / 16;
    const uint4 *vp = reinterpret_cast<const uint4 *>(in + a);
    uint64_t i = first;
    for (; i + 3 * step < nvec; i += 4 * step) {
        uint4 q[4];
#pragma unroll
        for (int u = 0; u < 4; u++) q[u] = __ldg(vp + i + u * step);
#pragma unroll
        for (int u = 0; u < 4; u++) hist_add_vec(q[u], hot, hot_bin, my);
    }
    for (; i < nvec; i += step) hist_add_vec(__ldg(vp + i), hot, hot_bin, my);
    for (uint64_t j = a + nvec * 16 + first; j < hi; j += step) hist_add_byte(in[j], hot, hot_bin, my);
}

// Adds the warp's 32 hot-byte counters into the hot byte's bin (whole warp,
// after its counting)
__device__ inline void hist_fold_hot(uint32_t *my, uint32_t hot) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    const uint32_t c = __reduce_add_sync(0xffffffffu, my[256 + lane]);
    if (lane == 0) my[hot] += c;
    __syncwarp();
}

__global__ void __launch_bounds__(kHistThreads) histogram_kernel(const uint8_t *__restrict__ in,
                                                                 const uint64_t *__restrict__ blk_off,
                                                                 uint32_t *__restrict__ hist, int slices) {
    __shared__ uint32_t wh[kHistWarps][kHistBins];
    const int b = blockIdx.x, sl = blockIdx.y;
    const int t = threadIdx.x, warp = t >> 5;
    const uint64_t lo0 = blk_off[b], hi0 = blk_off[b + 1];
    const uint64_t n = hi0 - lo0;
    const uint64_t span = ((n + slices - 1) / slices + 15) & ~uint64_t(15);
    const uint64_t lo = lo0 + min(n, span * sl), hi = lo0 + min(n, span * (sl + 1));
    for (int i = t; i < kHistWarps * kHistBins; i += kHistThreads) (&wh[0][0])[i] = 0;
    const uint32_t hot = hist_hot_byte(in, lo, hi);
    __syncthreads();
    hist_range(in, lo, hi, (uint32_t)t, kHistThreads, hot, wh[warp]);
    hist_fold_hot(wh[warp], hot);
    __syncthreads();
    for (int s = t; s < 256; s += kHistThreads) {
        uint32_t sum = 0;
#pragma unroll
        for (int w = 0; w < kHistWarps; w++) sum += wh[w][s];
        if (slices == 1) hist[(size_t)b * 256 + s] = sum;
        else if (sum) atomicAdd(&hist[(size_t)b * 256 + s], sum);
    }
}

cudaError_t launch_histogram(const uint8_t *in, const uint64_t *blk_off, int nblk, uint32_t *hist, int slices,
                             cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    if (slices < 1) slices = 1;
    if (slices > 1) {
        zero_u32_kernel<<<min(1024, div_up((long long)nblk * 256, 256)), 256, 0, st>>>(hist, (size_t)nblk * 256);
        count_launches(1);
    }
    histogram_kernel<<<dim3(nblk, slices), kHistThreads, 0, st>>>(in, blk_off, hist, slices);
    count_launches(1);
    return cudaGetLastError();
}

// Chunked histogram: one CTA per block, warp w counting chunk w of it (the
// encoder's warp chunks) into its own shared histogram.  The chunk
// histograms are written as they are (zeros for chunks the block does not
// have), the block histogram is their sum: no global atomics.
// One block by one CTA (256 threads): wh is shared scratch; the block
// histogram also goes to h_sm (shared) when given.
__device__ inline void histogram_chunks_block(int b, const uint8_t *__restrict__ in,
                                              const uint64_t *__restrict__ blk_off, uint32_t *__restrict__ hist,
                                              uint32_t *__restrict__ chunk_hist, uint32_t (*wh)[kHistBins],
                                              uint32_t *h_sm) {
    static_assert(kHistWarps == kEncChunks, "one warp per encoder chunk");
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint64_t n = blk_off[b + 1] - blk_off[b];
    const uint32_t nw = enc_nchunks(n);
    const uint64_t lo = blk_off[b] + enc_chunk_start(n, warp, nw), hi = blk_off[b] + enc_chunk_start(n, warp + 1, nw);
    uint32_t *my = wh[warp];
    for (int i = lane; i < kHistBins; i += 32) my[i] = 0;
    const uint32_t hot = hist_hot_byte(in, lo, hi);
    __syncwarp();
    hist_range(in, lo, hi, (uint32_t)lane, 32u, hot, my);
    hist_fold_hot(my, hot);
    __syncthreads();
    for (int s = t; s < 256; s += kHistThreads) {
        uint32_t sum = 0;
#pragma unroll
        for (int w = 0; w < kHistWarps; w++) {
            chunk_hist[((size_t)b * kEncChunks + w) * 256 + s] = wh[w][s];
            sum += wh[w][s];
        }
        hist[(size_t)b * 256 + s] = sum;
        if (h_sm) h_sm[s] = sum;
    }
}

__global__ void __launch_bounds__(kHistThreads) histogram_chunks_kernel(const uint8_t *__restrict__ in,
                                                                        const uint64_t *__restrict__ blk_off,
                                                                        uint32_t *__restrict__ hist,
                                                                        uint32_t *__restrict__ chunk_hist) {
    __shared__ uint32_t wh[kHistWarps][kHistBins];
    histogram_chunks_block(blockIdx.x, in, blk_off, hist, chunk_hist, wh, nullptr);
}

cudaError_t launch_histogram_chunks(const uint8_t *in, const uint64_t *blk_off, int nblk, uint32_t *hist,
                                    uint32_t *chunk_hist, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    histogram_chunks_kernel<<<nblk, kHistThreads, 0, st>>>(in, blk_off, hist, chunk_hist);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Code lengths by package-merge, one CTA (256 threads) per block.
// Lists are built from the deepest level L up to level 1.  Level L is the
// leaves sorted by (count, symbol); level l merges the sorted leaves with the
// packages formed by pairing neighbours of level l+1 (an odd last item is
// dropped).  A leaf sorts before a package of equal weight, so a leaf's
// position is i + #packages lighter than it and a package's position is
// j + #leaves not heavier than it.  Selecting the first 2K-2 items of level 1
// and following packages down: at each level the selected items are a
// prefix of the list; its leaves are the lightest leaves, and each gains one
// bit of length; its packages select twice as many items one level deeper.
// ---------------------------------------------------------------------------
constexpr int kPmThreads = 256;

// # of a[0..256) below x, a sorted with its unused tail holding the type's
// maximum (above every x searched for): binary lifting over 255 places, then
// one compare for the last, with no bounds checks
template <typename W>
__device__ inline int count_less_w(const W *a, W x) {
    int pos = 0;
#pragma unroll
    for (int step = 128; step >= 1; step >>= 1) pos = a[pos + step - 1] < x ? pos + step : pos;
    return pos + (a[pos] < x ? 1 : 0);
}
// # of a[0..256) not above x (the same tail)
template <typename W>
__device__ inline int count_le_w(const W *a, W x) {
    int pos = 0;
#pragma unroll
    for (int step = 128; step >= 1; step >>= 1) pos = a[pos + step - 1] <= x ? pos + step : pos;
    return pos + (a[pos] <= x ? 1 : 0);
}

// Levels max_len - 1 .. 1 of package-merge: each level merges the sorted
// leaves with the packages of the level below; leafpos[l][i] is leaf i's
// place at level l.  W: the weight type (32 bits when no package can reach
// 2^32 - 1, which halves the shared-memory traffic of the searches).  leafw
// (256 places) holds the type's maximum past the K leaves; pw is given the
// same tail at every level, so the searches need no bounds.
template <typename W>
__device__ inline void pm_levels(const W *leafw, W *pw, W (*lw)[512], uint16_t (*leafpos)[256], int K, int max_len) {
    const int t = threadIdx.x;
    for (int i = t; i < K; i += kPmThreads) { lw[max_len & 1][i] = leafw[i]; leafpos[max_len][i] = (uint16_t)i; }
    int len_prev = K;
    __syncthreads();
    for (int lvl = max_len - 1; lvl >= 1; lvl--) {
        const W *prev = lw[(lvl + 1) & 1];
        W *cur = lw[lvl & 1];
        const int P = len_prev / 2;
        for (int j = t; j < 256; j += kPmThreads) pw[j] = j < P ? prev[2 * j] + prev[2 * j + 1] : ~W(0);
        __syncthreads();
        for (int i = t; i < K; i += kPmThreads) {
            const int pos = i + count_less_w(pw, leafw[i]);
            cur[pos] = leafw[i];
            leafpos[lvl][i] = (uint16_t)pos;
        }
        for (int j = t; j < P; j += kPmThreads) cur[j + count_le_w(leafw, pw[j])] = pw[j];
        len_prev = K + P;
        __syncthreads();
    }
}

struct ClSmem {
    uint64_t leafw[256];
    uint8_t leafsym[256];
    uint64_t lw[2][512];
    uint64_t pw[256];
    uint16_t leafpos[kMaxLen + 1][256];
    int32_t s_len[kMaxLen + 2];
};

// Code lengths of the histogram h (shared, 256) into lens (shared, 256) by
// one CTA of 256 threads; returns the status (every thread).
__device__ inline int code_lengths_block(const uint32_t *h, int max_len, ClSmem &C, uint8_t *lens) {
    uint64_t *leafw = C.leafw, *pw = C.pw;
    uint8_t *leafsym = C.leafsym;
    uint64_t (*lw)[512] = C.lw;
    uint16_t (*leafpos)[256] = C.leafpos;
    int32_t *s_len = C.s_len;
    const int t = threadIdx.x;
    lens[t] = 0;
    const int K = __syncthreads_count(h[t] != 0);
    if (K >= 2 && K <= (1 << max_len)) {
        // present symbols sorted by (count, symbol): bitonic sort of one key per
        // thread (absent symbols sort last); in-warp steps exchange by shuffle
        {
            uint64_t key = h[t] ? (((uint64_t)h[t] << 8) | (uint64_t)t) : ~0ull;
            for (int k = 2; k <= 256; k <<= 1) {
                for (int j = k >> 1; j > 0; j >>= 1) {
                    uint64_t other;
                    if (j >= 32) {
                        pw[t] = key;
                        __syncthreads();
                        other = pw[t ^ j];
                        __syncthreads();
                    } else {
                        other = __shfl_xor_sync(0xffffffffu, key, j);
                    }
                    const bool lower = (t & j) == 0, up = (t & k) == 0;
                    // the lower partner keeps the smaller key in an ascending run
                    key = (lower == up) ? (key < other ? key : other) : (key < other ? other : key);
                }
            }
            leafw[t] = t < K ? key >> 8 : ~0ull;   // (the searches' tail past the leaves)
            if (t < K) leafsym[t] = (uint8_t)(key & 0xFF);
        }
        __syncthreads();
        // an item of a level holds at most one copy of a leaf per level
        // below, so no weight exceeds max_len * K * (largest count); 32-bit
        // weights stay below 2^32 - 1, the searches' tail value
        if ((uint64_t)max_len * (uint64_t)K * leafw[K - 1] < (1ull << 32) - 1) {
            uint32_t *leafw32 = reinterpret_cast<uint32_t *>(pw), *pw32 = leafw32 + 256;
            uint32_t (*lw32)[512] = reinterpret_cast<uint32_t (*)[512]>(&lw[0][0]);
            const uint32_t w = t < K ? (uint32_t)leafw[t] : 0xFFFFFFFFu;
            __syncthreads();
            leafw32[t] = w;
            __syncthreads();
            pm_levels<uint32_t>(leafw32, pw32, lw32, leafpos, K, max_len);
        } else {
            pm_levels<uint64_t>(leafw, pw, lw, leafpos, K, max_len);
        }
        // selection, top-down (one warp): at each level the selected items are
        // the first m; count the leaves among them (their positions increase
        // with i) by testing blocks of 8 leaves, then within the boundary block
        if (t < 32) {
            int m = 2 * K - 2;
            for (int lvl = 1; lvl <= max_len; lvl++) {
                const int last = min(8 * t + 7, K - 1);
                const bool full = 8 * t < K && leafpos[lvl][last] < m;
                const int nb = __popc(__ballot_sync(0xffffffffu, full));
                const int i2 = 8 * nb + t;
                const bool below = t < 8 && i2 < K && leafpos[lvl][min(i2, 255)] < m;
                const int cnt = min(8 * nb, K) + __popc(__ballot_sync(0xffffffffu, below));
                if (t == 0) s_len[lvl] = cnt;
                m = 2 * (m - cnt);
            }
        }
        __syncthreads();
        if (t < K) {
            int l = 0;
            for (int lvl = 1; lvl <= max_len; lvl++) l += (t < s_len[lvl]);
            lens[leafsym[t]] = (uint8_t)l;
        }
    }
    __syncthreads();
    return (K > (1 << max_len)) ? PIVCO_ERR_INVALID_ARG : PIVCO_OK;
}

__global__ void __launch_bounds__(kPmThreads) code_lengths_kernel(const uint32_t *__restrict__ hist, int max_len,
                                                                  uint8_t *__restrict__ lens_out,
                                                                  int32_t *__restrict__ status) {
    __shared__ ClSmem C;
    __shared__ uint32_t h[256];
    __shared__ uint8_t lens[256];
    const int b = blockIdx.x, t = threadIdx.x;
    h[t] = hist[(size_t)b * 256 + t];
    __syncthreads();
    const int st = code_lengths_block(h, max_len, C, lens);
    lens_out[(size_t)b * 256 + t] = lens[t];
    if (t == 0 && status) status[b] = st;
}

cudaError_t launch_code_lengths(const uint32_t *hist, int nblk, int max_len, uint8_t *lens, int32_t *status,
                                cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    code_lengths_kernel<<<nblk, kPmThreads, 0, st>>>(hist, max_len, lens, status);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Layout: canonical codes, node table, n_v, ANS selection, record layout.
// One CTA (256 threads) per block.
// ---------------------------------------------------------------------------
struct SelectParams {
    pivco_params p;
    int32_t fseh_q16[50];
};

// Sec. 5.2: selected when ceil(n/8) >= min bytes, skew > num/den and
// (depth + fse_H) / (depth + 1) < ratio.  Table t = round(100 * skew) in
// 50..99; bit 7 flags a bitmap whose ones are the majority (XOR 0xFF).
__device__ inline uint8_t ans_select(uint64_t nv, uint64_t n1, int depth, const SelectParams &sp) {
    if (!sp.p.ans_enable || nv == 0) return 0;
    const uint64_t bytes = (nv + 7) / 8;
    if (bytes < (uint64_t)sp.p.ans_min_bytes) return 0;
    const uint64_t n0 = nv - n1, mx = n0 > n1 ? n0 : n1;
    if (mx * (uint64_t)sp.p.ans_skew_den <= (uint64_t)sp.p.ans_skew_num * nv) return 0;
    uint64_t tt = (200 * mx + nv) / (2 * nv);
    tt = tt < 50 ? 50 : (tt > 99 ? 99 : tt);
    const uint64_t lhs = ((uint64_t)depth * 65536u + (uint64_t)sp.fseh_q16[tt - 50]) * 100u;
    const uint64_t rhs = (uint64_t)sp.p.ans_ratio_pct * (uint64_t)(depth + 1) * 65536u;
    if (!(lhs < rhs)) return 0;
    uint8_t m = (uint8_t)(tt - 49);
    if (n1 > n0) m |= 0x80;
    return m;
}

constexpr int kLayThreads = 256;

struct LaySmem {
    BlockLayout L;
    uint8_t sorted[256];
    uint16_t codes[256];
    int32_t scratch[256];
    TreeShape ts;
    FlatTree F;
    unsigned long long s_part[kLayThreads / 32];
};

// Layout of block b from its histogram h and lengths lens (both shared, 256)
// by one CTA of 256 threads: written to layout[b], rec_bound[b], status[b].
__device__ inline void build_layout_block(int b, const uint32_t *h, const uint8_t *lens, const SelectParams &sp,
                                          LaySmem &Y, BlockLayout *__restrict__ layout,
                                          uint64_t *__restrict__ rec_bound, int32_t *__restrict__ status) {
    BlockLayout &L = Y.L;
    uint8_t *sorted = Y.sorted;
    uint16_t *codes = Y.codes;
    int32_t *scratch = Y.scratch;
    TreeShape &ts = Y.ts;
    const int t = threadIdx.x;
    // zero the shared layout
    for (int i = t; i < (int)(sizeof(BlockLayout) / 4); i += kLayThreads) reinterpret_cast<uint32_t *>(&L)[i] = 0;
    __syncthreads();
    const int K = __syncthreads_count(h[t] != 0);
    uint64_t n = 0;
    {
        // block total: warp sums, then the 8 partial sums (no same-address atomics)
        unsigned long long *s_part = Y.s_part;
        uint64_t x = h[t];
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((t & 31) == 0) s_part[t >> 5] = x;
        __syncthreads();
#pragma unroll
        for (int w = 0; w < kLayThreads / 32; w++) n += s_part[w];
    }
    int st = PIVCO_OK;
    if (t == 0) { L.n = (uint32_t)n; L.status = 0; }
    if (K <= 1) {
        if (t == 0) {
            L.kind = K == 0 ? 0 : 1;
            L.flat = sp.p.flat ? 1 : 0;
            L.rec_bound = kHdr;
            L.body0 = kHdr;
        }
        if (h[t]) L.csym = (uint8_t)t;
        __syncthreads();
    } else {
        build_tree_shape(lens, ts, codes, sorted, scratch);
        const bool flat = sp.p.flat != 0;
        FlatTree &F = Y.F;
        if (flat && t < 32) flat_tree_build(ts.cnt, ts.len_base, sorted, F);
        __syncthreads();
        if (!ts.ok || ts.K != K || n > 0xFFFFFFFFull || (flat && !F.ok)) {
            st = PIVCO_ERR_INVALID_ARG;
        } else {
            const int V = flat ? F.n_nodes : ts.n_int;
            const int maxd = flat ? F.maxd : ts.max_len;     // node levels
            const int32_t *fst = flat ? F.first : ts.first;
            if (t == 0) {
                L.kind = 2;
                L.flat = flat ? 1 : 0;
                L.n_int = (uint16_t)V;
                L.max_depth = (uint8_t)maxd;
                for (int d = 0; d <= 16; d++) L.depth_first[d] = (uint8_t)(d < maxd ? fst[d] : V);
                for (int d = 0; d <= 16; d++) L.tree_a[d] = (uint16_t)(flat ? F.a[d] : ts.a[d]);
            }
            if (flat) {
                // regrouped codes (symbol x of item i is (code_i << D) | x) and
                // code indices (its item's code-order offset + x), per symbol
                if (t < K) {
                    const int sy = sorted[t], l = lens[sy];
                    int i;
                    uint32_t x;
                    flat_sym(F, ts.cnt, l, t - ts.len_base[l], i, x);
                    codes[sy] = (uint16_t)((flat_item_code(F, i) << F.iD[i]) | x);
                    L.ci[sy] = (uint8_t)(F.ioff[i] + x);
                }
                __syncthreads();
            }
            L.code[t] = codes[t];
            L.len[t] = lens[t];
            bool okn = true;
            if (t < V) {
                int d = 0;
                uint32_t chv = 0;
                if (flat) {
                    okn = flat_node(F, sorted, t, d, chv);
                } else {
                    d = node_depth(ts, t);
                    chv = ((uint32_t)node_child(ts, sorted, t, d, 0) & 0xFFFFu) |
                          ((uint32_t)node_child(ts, sorted, t, d, 1) << 16);
                }
                L.depth[t] = (uint8_t)d;
                // (a canonical node's word holds its children as 16-bit ints: never flat)
                const uint32_t D = flat ? ch_flat_d(chv) : 0u;
                if (D == 1 || D > 8) okn = false;
                L.fd[t] = (uint8_t)D;
                L.fbase[t] = D ? (uint8_t)(chv & 0xFFu) : 0;
                for (int c = 0; c < 2; c++) {
                    const uint32_t x = D ? 0u : (chv >> (16 * c)) & 0xFFFFu;
                    L.child[t][c] = flat ? (int16_t)((x & 0x8000u) ? -(int)(x & 0xFFu) - 1 : (int)x)
                                         : (int16_t)(chv >> (16 * c));
                }
            }
            if (__syncthreads_or(!okn)) {
                st = PIVCO_ERR_INVALID_ARG;
            } else {
                if (flat) {
                    // a flat node's count from prefix sums of the block's
                    // counts in code order (its symbols are consecutive there)
                    uint32_t *hc = reinterpret_cast<uint32_t *>(scratch);   // 256 counts, then warp sums
                    hc[t] = 0;
                    __syncthreads();
                    if (lens[t]) hc[L.ci[t]] = h[t];
                    __syncthreads();
                    uint32_t x = hc[t], inc = x;
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                        if ((t & 31) >= o) inc += y;
                    }
                    __shared__ uint32_t wsum[kLayThreads / 32];
                    if ((t & 31) == 31) wsum[t >> 5] = inc;
                    __syncthreads();
                    for (int w2 = 0; w2 < (t >> 5); w2++) inc += wsum[w2];
                    __syncthreads();
                    hc[t] = inc - x;            // exclusive prefix: counts of code indices < t
                    __syncthreads();
                    if (t < V && L.fd[t]) {
                        const uint32_t D = L.fd[t], lo = L.ci[sorted[L.fbase[t]]], hi = lo + (1u << D) - 1u;
                        L.nlo[t] = (uint8_t)lo;
                        L.nhi1[t] = (uint8_t)hi;
                        L.nv[t] = (hi + 1 < 256 ? hc[hi + 1] : (uint32_t)n) - hc[lo];
                    }
                } else if (t < K) {
                    L.ci[sorted[t]] = (uint8_t)t;
                }
                __syncthreads();
                // n_v bottom-up, one depth at a time: a node's count is its
                // children's (a flat node's, its symbols'); its leaves (a
                // contiguous run of the code order) start at its left child's
                // and end at its right child's
                for (int d = maxd - 1; d >= 0; d--) {
                    const int v = fst[d] + t;
                    if (v < fst[d + 1] && v < V) {
                        if (!L.fd[v]) {   // (a flat node's count and range are set)
                            uint32_t c = 0;
                            for (int k = 0; k < 2; k++) {
                                const int ch = L.child[v][k];
                                c += ch >= 0 ? L.nv[ch] : h[-ch - 1];
                            }
                            L.nv[v] = c;
                            const int c0 = L.child[v][0], c1 = L.child[v][1];
                            L.nlo[v] = c0 >= 0 ? L.nlo[c0] : L.ci[-c0 - 1];
                            L.nhi1[v] = c1 >= 0 ? L.nhi1[c1] : L.ci[-c1 - 1];
                        }
                    }
                    __syncthreads();
                }
                if (t < V && !L.fd[t]) {
                    const int c = L.child[t][1];
                    const uint64_t n1 = c >= 0 ? L.nv[c] : h[-c - 1];
                    L.sel[t] = ans_select(L.nv[t], n1, L.depth[t], sp);
                }
                // a big block: some level (depth >= 1) of the whole block
                // does not fit an encoder level buffer (spans of whole
                // 16-byte units), so the chunked encoder splits it
                if (t >= 1 && t < maxd) {
                    uint64_t lvl = 0;
                    for (int v = fst[t]; v < fst[t + 1]; v++) lvl += ((uint64_t)L.nv[v] + 7u) & ~7ull;
                    if (lvl > (uint64_t)kEBuf && enc_nchunks(n) >= 2) L.big = 1;
                }
                __syncthreads();
            if (t < 32) {
                // bodies: the raw (unselected) nodes first, then the selected ones, node order
                const int lane = t;
                uint32_t nsel = 0, raw_tot = 0;
                for (int base = 0; base < V; base += 32) {
                    const int v = base + lane;
                    const bool in = v < V;
                    nsel += __popc(__ballot_sync(0xffffffffu, in && L.sel[v]));
                    raw_tot += __reduce_add_sync(0xffffffffu, (in && !L.sel[v]) ? (uint32_t)(((uint64_t)L.nv[v] * max(1u, (uint32_t)L.fd[v]) + 7) / 8) : 0u);
                }
                const uint32_t off0 = ((kNvOff + 5u * V + 3u) & ~3u) + 4u * nsel;
                uint32_t c_raw = off0, c_sel = off0 + raw_tot;
                for (int base = 0; base < V; base += 32) {
                    const int v = base + lane;
                    const bool in = v < V, sel = in && L.sel[v];
                    const uint32_t by = in ? (uint32_t)(((uint64_t)L.nv[v] * max(1u, (uint32_t)L.fd[v]) + 7) / 8) : 0u;
                    uint32_t xr = (in && !sel) ? by : 0u, xs = sel ? by : 0u;
                    uint32_t ir = xr, is = xs;
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t yr = __shfl_up_sync(0xffffffffu, ir, o), ys = __shfl_up_sync(0xffffffffu, is, o);
                        if (lane >= o) { ir += yr; is += ys; }
                    }
                    if (in) L.body_off[v] = sel ? c_sel + is - xs : c_raw + ir - xr;
                    c_raw += __shfl_sync(0xffffffffu, ir, 31);
                    c_sel += __shfl_sync(0xffffffffu, is, 31);
                }
                if (lane == 0) {
                    L.body0 = off0;
                    L.n_sel = (uint8_t)nsel;
                    L.body_end = c_sel;
                    L.rec_bound = (c_sel + 15u) & ~15u;
                }
            }
            }
        }
    }
    if (t == 0) L.status = (uint8_t)st;
    __syncthreads();
    if (st != PIVCO_OK && t == 0) { L.kind = 0; L.rec_bound = kHdr; }
    __syncthreads();
    uint32_t *dst = reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(layout) + (size_t)b * kLayoutBytes);
    for (int i = t; i < (int)(sizeof(BlockLayout) / 4); i += kLayThreads) dst[i] = reinterpret_cast<uint32_t *>(&L)[i];
    if (t == 0) {
        rec_bound[b] = L.rec_bound;
        if (status) status[b] = st;
    }
}

__global__ void __launch_bounds__(kLayThreads) build_layout_kernel(const uint32_t *__restrict__ hist,
                                                                   const uint8_t *__restrict__ lens_in,
                                                                   const __grid_constant__ SelectParams sp,
                                                                   BlockLayout *__restrict__ layout,
                                                                   uint64_t *__restrict__ rec_bound,
                                                                   int32_t *__restrict__ status) {
    __shared__ LaySmem Y;
    __shared__ uint32_t h[256];
    __shared__ uint8_t lens[256];
    const int b = blockIdx.x, t = threadIdx.x;
    h[t] = hist[(size_t)b * 256 + t];
    lens[t] = lens_in[(size_t)b * 256 + t];
    build_layout_block(b, h, lens, sp, Y, layout, rec_bound, status);
}

// The encoder's planning in one launch, one CTA per block: chunk histograms,
// code lengths, layout.  The block's statistics stay in shared memory from
// one step to the next, and blocks in different steps share the SMs.
struct PlanSmem {
    uint32_t h[256];
    uint8_t lens[256];
    union {
        uint32_t wh[kHistWarps][kHistBins];
        ClSmem cl;
        LaySmem lay;
    } u;
};

__global__ void __launch_bounds__(kHistThreads) block_plan_kernel(const uint8_t *__restrict__ in,
                                                                  const uint64_t *__restrict__ blk_off, int max_len,
                                                                  const __grid_constant__ SelectParams sp,
                                                                  uint32_t *__restrict__ hist,
                                                                  uint32_t *__restrict__ chunk_hist,
                                                                  uint8_t *__restrict__ lens_out,
                                                                  BlockLayout *__restrict__ layout,
                                                                  uint64_t *__restrict__ rec_bound,
                                                                  int32_t *__restrict__ status) {
    static_assert(kHistThreads == kPmThreads && kPmThreads == kLayThreads, "one CTA shape for the three steps");
    __shared__ PlanSmem P;
    const int b = blockIdx.x, t = threadIdx.x;
    histogram_chunks_block(b, in, blk_off, hist, chunk_hist, P.u.wh, P.h);
    __syncthreads();
    code_lengths_block(P.h, max_len, P.u.cl, P.lens);   // (its status is the layout's too)
    lens_out[(size_t)b * 256 + t] = P.lens[t];
    __syncthreads();
    build_layout_block(b, P.h, P.lens, sp, P.u.lay, layout, rec_bound, status);
}

cudaError_t launch_block_plan(const uint8_t *in, const uint64_t *blk_off, int nblk, const pivco_params &p,
                              uint32_t *hist, uint32_t *chunk_hist, uint8_t *lens, BlockLayout *layout,
                              uint64_t *rec_bound, int32_t *status, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    SelectParams sp;
    sp.p = p;
    const AnsTables &T = host_ans_tables();
    for (int i = 0; i < 50; i++) sp.fseh_q16[i] = T.fseh_q16[i];
    block_plan_kernel<<<nblk, kHistThreads, 0, st>>>(in, blk_off, p.max_len, sp, hist, chunk_hist, lens, layout,
                                                     rec_bound, status);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_build_layout(const uint32_t *hist, const uint8_t *lens, int nblk, const pivco_params &p,
                                BlockLayout *layout, uint64_t *rec_bound, int32_t *status, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    SelectParams sp;
    sp.p = p;
    const AnsTables &T = host_ans_tables();
    for (int i = 0; i < 50; i++) sp.fseh_q16[i] = T.fseh_q16[i];
    build_layout_kernel<<<nblk, kLayThreads, 0, st>>>(hist, lens, sp, layout, rec_bound, status);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pv
