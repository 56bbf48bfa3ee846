// Host side of the C ABI (include/pivco.h): argument checks, the library's
// static ANS tables, and kernel launches.  No call here allocates device memory.
#include <cmath>
#include <cstring>
#include <atomic>
#include <mutex>

#include "pivco_dev.cuh"

namespace pv {

// ---------------------------------------------------------------------------
// Static ANS tables (Sec. 5.2): for skew t = 50..99 %, bytes of i.i.d. bits
// with P(bit = 0) = t / 100.  One byte with k one-bits has probability
// t^(8-k) (100-t)^k / 100^8; its frequency out of 2^15 is that times 2^15,
// rounded down, at least 1; byte 0x00 takes the remaining slack so the
// frequencies sum to 2^15 exactly.
// ---------------------------------------------------------------------------
static AnsTables g_tab;
static std::once_flag g_tab_once;

static void build_tables() {
    static const uint32_t C8[9] = {1, 8, 28, 56, 70, 56, 28, 8, 1};
    const uint64_t D = 305175781250ull;   // 100^8 / 2^15
    for (int t = 50; t <= 99; t++) {
        const int i = t - 50;
        uint64_t w[9];
        int64_t q[9], tot = 0;
        for (int k = 0; k <= 8; k++) {
            uint64_t x = 1;
            for (int j = 0; j < 8 - k; j++) x *= (uint64_t)t;
            for (int j = 0; j < k; j++) x *= (uint64_t)(100 - t);
            w[k] = x;
            q[k] = (int64_t)(x / D);
            if (q[k] < 1) q[k] = 1;
            tot += (int64_t)C8[k] * q[k];
        }
        q[0] += (int64_t)kAnsM - tot;
        uint32_t start = 0;
        long double h = 0.0L;
        for (int k = 0; k <= 8; k++) {
            g_tab.q[i][k] = (uint16_t)q[k];
            g_tab.start[i][k] = (uint16_t)start;
            start += C8[k] * (uint32_t)q[k];
            g_tab.magic[i][k] = q[k] >= 2 ? (uint32_t)((((uint64_t)1 << 32) + (uint64_t)q[k] - 1) / (uint64_t)q[k]) : 0u;
            const long double p = (long double)w[k] / 1e16L;
            h += (long double)C8[k] * p * log2l((long double)kAnsM / (long double)q[k]);
        }
        g_tab.start[i][9] = (uint16_t)(start & 0xFFFF);   // 2^15
        g_tab.fseh_q16[i] = (int32_t)floorl(h / 8.0L * 65536.0L + 0.5L);
    }
    int n = 0;
    for (int k = 0; k <= 8; k++) {
        g_tab.class_base[k] = (uint8_t)n;
        int r = 0;
        for (int b = 0; b < 256; b++)
            if (__builtin_popcount(b) == k) { g_tab.class_member[n++] = (uint8_t)b; g_tab.rank_in_class[b] = (uint8_t)r++; }
    }
    g_tab.class_base[9] = 0;   // 256 does not fit; unused
}

static std::atomic<uint64_t> g_launches{0};
void count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

const AnsTables &host_ans_tables() {
    std::call_once(g_tab_once, build_tables);
    return g_tab;
}

}  // namespace pv

using namespace pv;

static inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }
static inline pivco_status ok_or_cuda(cudaError_t e) { return e == cudaSuccess ? PIVCO_OK : PIVCO_ERR_CUDA; }

extern "C" {

const char *pivco_version(void) { return "pivco-gb300 1.0 (format PVC1, sm_103a)"; }

int32_t pivco_layout_bytes(void) { return kLayoutBytes; }

pivco_status pivco_histogram(const uint8_t *in, const uint64_t *blk_off, int32_t nblk, uint32_t *hist, void *stream) {
    if (nblk < 0 || (nblk > 0 && (!blk_off || !hist))) return PIVCO_ERR_INVALID_ARG;
    if (nblk == 0) return PIVCO_OK;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int slices = (4 * sms + nblk - 1) / nblk;
    if (slices > 256) slices = 256;
    if (slices < 1) slices = 1;
    return ok_or_cuda(launch_histogram(in, blk_off, nblk, hist, slices, S(stream)));
}

pivco_status pivco_code_lengths(const uint32_t *hist, int32_t nblk, int32_t max_len, uint8_t *lens, int32_t *status,
                                void *stream) {
    if (nblk < 0 || max_len < 1 || max_len > (int32_t)kMaxLen || (nblk > 0 && (!hist || !lens))) return PIVCO_ERR_INVALID_ARG;
    return ok_or_cuda(launch_code_lengths(hist, nblk, max_len, lens, status, S(stream)));
}

pivco_status pivco_build_layout(const uint32_t *hist, const uint8_t *lens, int32_t nblk, const pivco_params *params,
                                void *layout, uint64_t *rec_bound, int32_t *status, void *stream) {
    if (nblk < 0 || !params || (nblk > 0 && (!hist || !lens || !layout || !rec_bound || !status))) return PIVCO_ERR_INVALID_ARG;
    const pivco_params &p = *params;
    if (p.max_len < 1 || p.max_len > (int32_t)kMaxLen || p.ans_min_bytes < 0 || p.ans_skew_den <= 0 ||
        p.ans_skew_num < 0 || p.ans_ratio_pct < 0)
        return PIVCO_ERR_INVALID_ARG;
    return ok_or_cuda(launch_build_layout(hist, lens, nblk, p, reinterpret_cast<BlockLayout *>(layout), rec_bound, status,
                                          S(stream)));
}

size_t pivco_scan_workspace_size(int32_t n) { return scan_ws_bytes(n); }

pivco_status pivco_exclusive_scan(const uint64_t *in, int32_t n, uint64_t *out, void *ws, size_t ws_bytes,
                                  int32_t *status_out, void *stream) {
    if (n < 0 || !out || !ws || ws_bytes < scan_ws_bytes(n) || (n > 0 && !in)) return PIVCO_ERR_INVALID_ARG;
    return ok_or_cuda(launch_scan(in, n, out, ws, status_out, S(stream)));
}

pivco_status pivco_encode_blocks(const uint8_t *in, const uint64_t *blk_off, int32_t nblk, const void *layout,
                                 uint8_t *out, const uint64_t *out_off, uint64_t *rec_bytes, int32_t *status,
                                 void *stream) {
    if (nblk < 0 || (nblk > 0 && (!blk_off || !layout || !out || !out_off || !rec_bytes || !status)))
        return PIVCO_ERR_INVALID_ARG;
    return ok_or_cuda(launch_encode(in, blk_off, nblk, reinterpret_cast<const BlockLayout *>(layout), out, out_off,
                                    rec_bytes, status, S(stream)));
}

pivco_status pivco_ans_encode_blocks(const void *layout, int32_t nblk, uint8_t *out, const uint64_t *out_off,
                                     uint64_t *rec_bytes, void *ws, size_t ws_bytes, int32_t *status, void *stream) {
    if (nblk < 0 || (nblk > 0 && (!layout || !out || !out_off || !rec_bytes || !ws || !status))) return PIVCO_ERR_INVALID_ARG;
    return ok_or_cuda(launch_ans_encode_blocks(reinterpret_cast<const BlockLayout *>(layout), nblk, out, out_off,
                                               rec_bytes, reinterpret_cast<uint8_t *>(ws), ws_bytes, status,
                                               S(stream)));
}

size_t pivco_decode_plan_bytes(int32_t nblk) { return nblk < 0 ? 0 : decode_ws_fixed_bytes(nblk); }

pivco_status pivco_decode_workspace_size(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk, void *ws,
                                         size_t ws_bytes, int32_t *status, size_t *bytes, void *stream) {
    if (nblk < 0 || !bytes || (nblk > 0 && (!comp || !comp_off || !ws || !status))) return PIVCO_ERR_INVALID_ARG;
    if (nblk == 0) { *bytes = 0; return PIVCO_OK; }
    if (ws_bytes < decode_ws_fixed_bytes(nblk)) return PIVCO_ERR_CAPACITY;
    cudaError_t e = launch_decode_plan(comp, comp_off, nblk, reinterpret_cast<uint8_t *>(ws), ws_bytes, status, S(stream));
    if (e != cudaSuccess) return PIVCO_ERR_CUDA;
    return ok_or_cuda(read_decode_ws_need(reinterpret_cast<const uint8_t *>(ws), nblk, bytes, S(stream)));
}

pivco_status pivco_decode_blocks(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk, uint8_t *out,
                                 const uint64_t *out_off, void *ws, size_t ws_bytes, int32_t *status, void *stream) {
    if (nblk < 0 || (nblk > 0 && (!comp || !comp_off || !out_off || !ws || !status))) return PIVCO_ERR_INVALID_ARG;
    if (nblk == 0) return PIVCO_OK;
    if (ws_bytes < decode_ws_fixed_bytes(nblk)) return PIVCO_ERR_CAPACITY;
    return ok_or_cuda(launch_decode(comp, comp_off, nblk, out, out_off, reinterpret_cast<uint8_t *>(ws), ws_bytes,
                                    status, S(stream)));
}

pivco_status pivco_decode_plan(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk, void *ws, size_t ws_bytes,
                               int32_t *status, void *stream) {
    if (nblk < 0 || (nblk > 0 && (!comp || !comp_off || !ws || !status))) return PIVCO_ERR_INVALID_ARG;
    if (nblk == 0) return PIVCO_OK;
    if (ws_bytes < decode_ws_fixed_bytes(nblk)) return PIVCO_ERR_CAPACITY;
    return ok_or_cuda(launch_decode_plan(comp, comp_off, nblk, reinterpret_cast<uint8_t *>(ws), ws_bytes, status,
                                         S(stream)));
}

pivco_status pivco_decode_ans(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk, void *ws, size_t ws_bytes,
                              int32_t *status, void *stream) {
    if (nblk < 0 || (nblk > 0 && (!comp || !comp_off || !ws || !status))) return PIVCO_ERR_INVALID_ARG;
    if (nblk == 0) return PIVCO_OK;
    if (ws_bytes < decode_ws_fixed_bytes(nblk)) return PIVCO_ERR_CAPACITY;
    return ok_or_cuda(launch_ans_decode_planned(comp, comp_off, nblk, reinterpret_cast<uint8_t *>(ws), ws_bytes,
                                                status, S(stream)));
}

pivco_status pivco_decode_merge(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk, uint8_t *out,
                                const uint64_t *out_off, void *ws, size_t ws_bytes, int32_t *status, void *stream) {
    if (nblk < 0 || (nblk > 0 && (!comp || !comp_off || !out_off || !ws || !status))) return PIVCO_ERR_INVALID_ARG;
    if (nblk == 0) return PIVCO_OK;
    if (ws_bytes < decode_ws_fixed_bytes(nblk)) return PIVCO_ERR_CAPACITY;
    return ok_or_cuda(launch_decode_merge(comp, comp_off, nblk, out, out_off, reinterpret_cast<uint8_t *>(ws),
                                          ws_bytes, status, S(stream)));
}

uint64_t pivco_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

pivco_status pivco_ans_tables(int32_t *fse_h_q16, uint32_t *class_freq) {
    const AnsTables &T = host_ans_tables();
    for (int i = 0; i < 50; i++) {
        if (fse_h_q16) fse_h_q16[i] = T.fseh_q16[i];
        if (class_freq)
            for (int k = 0; k < 9; k++) class_freq[9 * i + k] = T.q[i][k];
    }
    return PIVCO_OK;
}

pivco_status pivco_ans_encode(const uint8_t *bitmaps, const uint64_t *bm_off, const uint8_t *table, int32_t nbm,
                              uint8_t *bodies, const uint64_t *body_off, uint64_t *body_bytes, int32_t *status,
                              void *stream) {
    if (nbm < 0 || (nbm > 0 && (!bitmaps || !bm_off || !table || !bodies || !body_off || !body_bytes || !status)))
        return PIVCO_ERR_INVALID_ARG;
    return ok_or_cuda(launch_ans_encode(bitmaps, bm_off, table, nbm, bodies, body_off, body_bytes, status, S(stream)));
}

pivco_status pivco_ans_decode(const uint8_t *bodies, const uint64_t *body_off, const uint8_t *table, int32_t nbm,
                              uint8_t *bitmaps, const uint64_t *bm_off, int32_t *status, void *stream) {
    if (nbm < 0 || (nbm > 0 && (!bitmaps || !bm_off || !table || !bodies || !body_off || !status)))
        return PIVCO_ERR_INVALID_ARG;
    return ok_or_cuda(launch_ans_decode(bodies, body_off, table, nbm, bitmaps, bm_off, status, S(stream)));
}

}  // extern "C"
