// Host side of the C ABI (include/pivco.h): argument checks, the library's
// static ANS tables, and kernel launches.  No call here allocates device memory.
#include <cmath>
#include <cstring>
#include <atomic>
#include <mutex>
#include <vector>

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

// launch tuning of the decode (process-wide; set by pivco_set_tuning / the autotuner)
static DecTuning g_tuning = {1u << 20, 128, 0};
static std::mutex g_tuning_mu;
DecTuning current_tuning() {
    std::lock_guard<std::mutex> lk(g_tuning_mu);
    return g_tuning;
}
void set_tuning(const DecTuning &t) {
    std::lock_guard<std::mutex> lk(g_tuning_mu);
    g_tuning = t;
}
void count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

static std::atomic<uint64_t> g_wait_limit{kWaitLimitNs};
uint64_t wait_limit_ns() { return g_wait_limit.load(std::memory_order_relaxed); }

const AnsTables &host_ans_tables() {
    std::call_once(g_tab_once, build_tables);
    return g_tab;
}

}  // namespace pv

using namespace pv;

static inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Library-owned decode workspace for pivco_decode_blocks_static: one array
// per device, part of this module (no allocation call ever makes it).  Its
// address is looked up once per device, with that device current.
static constexpr size_t kStaticWsBytes = 16u << 20;
static __device__ __align__(256) uint8_t g_static_ws[kStaticWsBytes];
static constexpr int kMaxDevices = 64;
static uint8_t *g_static_ws_ptr[kMaxDevices];
static std::mutex g_static_ws_mu;

// cudaErrorStreamCaptureUnsupported when the address is not known yet and
// `st` is capturing (the lookup may load the module, which a capture forbids)
static cudaError_t static_ws_address(uint8_t **ptr, cudaStream_t st) {
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    if (d < 0 || d >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_static_ws_mu);
    if (!g_static_ws_ptr[d]) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(st, &cs);
        if (e != cudaSuccess) return e;
        if (cs != cudaStreamCaptureStatusNone) return cudaErrorStreamCaptureUnsupported;
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_ws);
        if (e != cudaSuccess) return e;
        g_static_ws_ptr[d] = reinterpret_cast<uint8_t *>(p);
    }
    *ptr = g_static_ws_ptr[d];
    return cudaSuccess;
}

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

// the layout buffer is read with 16-byte loads
static bool layout_aligned(const void *layout) { return !(reinterpret_cast<uintptr_t>(layout) & 15); }

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
        p.ans_skew_num < 0 || p.ans_ratio_pct < 0 || (p.flat != 0 && p.flat != 1))
        return PIVCO_ERR_INVALID_ARG;
    if (nblk > 0 && !layout_aligned(layout)) return PIVCO_ERR_INVALID_ARG;
    return ok_or_cuda(launch_build_layout(hist, lens, nblk, p, reinterpret_cast<BlockLayout *>(layout), rec_bound, status,
                                          S(stream)));
}

pivco_status pivco_plan_blocks(const uint8_t *in, const uint64_t *blk_off, int32_t nblk, const pivco_params *params,
                               uint32_t *hist, uint32_t *chunk_hist, uint8_t *lens, void *layout, uint64_t *rec_bound,
                               int32_t *status, void *stream) {
    if (nblk < 0 || !params ||
        (nblk > 0 && (!blk_off || !hist || !chunk_hist || !lens || !layout || !rec_bound || !status)))
        return PIVCO_ERR_INVALID_ARG;
    const pivco_params &p = *params;
    if (p.max_len < 1 || p.max_len > (int32_t)kMaxLen || p.ans_min_bytes < 0 || p.ans_skew_den <= 0 ||
        p.ans_skew_num < 0 || p.ans_ratio_pct < 0 || (p.flat != 0 && p.flat != 1))
        return PIVCO_ERR_INVALID_ARG;
    if (nblk > 0 && !layout_aligned(layout)) return PIVCO_ERR_INVALID_ARG;
    return ok_or_cuda(launch_block_plan(in, blk_off, nblk, p, hist, chunk_hist, lens,
                                        reinterpret_cast<BlockLayout *>(layout), rec_bound, status, S(stream)));
}

size_t pivco_scan_workspace_size(int32_t n) { return scan_ws_bytes(n); }

pivco_status pivco_exclusive_scan(const uint64_t *in, int32_t n, uint64_t *out, void *ws, size_t ws_bytes,
                                  int32_t *status_out, void *stream) {
    if (n < 0 || !out || !ws || ws_bytes < scan_ws_bytes(n) || (n > 0 && !in)) return PIVCO_ERR_INVALID_ARG;
    return ok_or_cuda(launch_scan(in, n, out, ws, status_out, S(stream)));
}

pivco_status pivco_encode_blocks(const uint8_t *in, const uint64_t *blk_off, int32_t nblk, void *layout,
                                 uint8_t *out, const uint64_t *out_off, uint64_t *rec_bytes, int32_t *status,
                                 void *stream) {
    if (nblk < 0 || (nblk > 0 && (!blk_off || !layout || !out || !out_off || !rec_bytes || !status)))
        return PIVCO_ERR_INVALID_ARG;
    if (nblk > 0 && !layout_aligned(layout)) return PIVCO_ERR_INVALID_ARG;
    return ok_or_cuda(launch_encode(in, blk_off, nblk, reinterpret_cast<BlockLayout *>(layout), nullptr, out,
                                    out_off, rec_bytes, status, S(stream)));
}

pivco_status pivco_histogram_chunks(const uint8_t *in, const uint64_t *blk_off, int32_t nblk, uint32_t *hist,
                                    uint32_t *chunk_hist, void *stream) {
    if (nblk < 0 || (nblk > 0 && (!blk_off || !hist || !chunk_hist))) return PIVCO_ERR_INVALID_ARG;
    if (nblk == 0) return PIVCO_OK;
    return ok_or_cuda(launch_histogram_chunks(in, blk_off, nblk, hist, chunk_hist, S(stream)));
}

pivco_status pivco_encode_blocks_chunked(const uint8_t *in, const uint64_t *blk_off, int32_t nblk, void *layout,
                                         const uint32_t *chunk_hist, uint8_t *out, const uint64_t *out_off,
                                         uint64_t *rec_bytes, int32_t *status, void *stream) {
    if (nblk < 0 || (nblk > 0 && (!blk_off || !layout || !chunk_hist || !out || !out_off || !rec_bytes || !status)))
        return PIVCO_ERR_INVALID_ARG;
    if (nblk > 0 && !layout_aligned(layout)) return PIVCO_ERR_INVALID_ARG;
    return ok_or_cuda(launch_encode(in, blk_off, nblk, reinterpret_cast<BlockLayout *>(layout), chunk_hist, out,
                                    out_off, rec_bytes, status, S(stream)));
}

pivco_status pivco_ans_encode_blocks(const void *layout, int32_t nblk, uint8_t *out, const uint64_t *out_off,
                                     uint64_t *rec_bytes, void *ws, size_t ws_bytes, int32_t *status, void *stream) {
    if (nblk < 0 || (nblk > 0 && (!layout || !out || !out_off || !rec_bytes || !ws || !status))) return PIVCO_ERR_INVALID_ARG;
    if (nblk > 0 && !layout_aligned(layout)) return PIVCO_ERR_INVALID_ARG;
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

pivco_status pivco_decode_blocks_static(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk, uint8_t *out,
                                        const uint64_t *out_off, int32_t *status, void *stream) {
    static_assert(kStaticWsBytes == PIVCO_DECODE_STATIC_WS_BYTES, "header and library disagree on the size");
    if (nblk < 0 || (nblk > 0 && (!comp || !comp_off || !out_off || !status))) return PIVCO_ERR_INVALID_ARG;
    if (nblk == 0) return PIVCO_OK;
    if (decode_ws_fixed_bytes(nblk) > kStaticWsBytes) return PIVCO_ERR_CAPACITY;
    uint8_t *ws = nullptr;
    const cudaError_t e = static_ws_address(&ws, S(stream));
    if (e == cudaErrorStreamCaptureUnsupported) return PIVCO_ERR_INVALID_ARG;
    if (e != cudaSuccess) return PIVCO_ERR_CUDA;
    // the plan step's first launch zeroes the header, look-back states and
    // counters; scratch and directories need no clearing
    return ok_or_cuda(launch_decode(comp, comp_off, nblk, out, out_off, ws, kStaticWsBytes, status, S(stream)));
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

pivco_status pivco_access_workspace_size(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk, void *ws,
                                         size_t ws_bytes, int32_t *status, size_t *bytes, void *stream) {
    if (nblk < 0 || !bytes || (nblk > 0 && (!comp || !comp_off || !ws || !status))) return PIVCO_ERR_INVALID_ARG;
    if (nblk == 0) { *bytes = 0; return PIVCO_OK; }
    if (ws_bytes < decode_ws_fixed_bytes(nblk)) return PIVCO_ERR_CAPACITY;
    cudaError_t e = launch_decode_plan(comp, comp_off, nblk, reinterpret_cast<uint8_t *>(ws), ws_bytes, status, S(stream),
                                       true);
    if (e != cudaSuccess) return PIVCO_ERR_CUDA;
    return ok_or_cuda(read_decode_ws_need(reinterpret_cast<const uint8_t *>(ws), nblk, bytes, S(stream)));
}

pivco_status pivco_access_prepare(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk, void *ws,
                                  size_t ws_bytes, int32_t *status, void *stream) {
    if (nblk < 0 || (nblk > 0 && (!comp || !comp_off || !ws || !status))) return PIVCO_ERR_INVALID_ARG;
    if (nblk == 0) return PIVCO_OK;
    if (ws_bytes < decode_ws_fixed_bytes(nblk)) return PIVCO_ERR_CAPACITY;
    return ok_or_cuda(launch_access_prepare(comp, comp_off, nblk, reinterpret_cast<uint8_t *>(ws), ws_bytes, status,
                                            S(stream)));
}

pivco_status pivco_access(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk, const uint32_t *qblk,
                          const uint32_t *qpos, int32_t nq, uint8_t *sym, int32_t *qstatus, const void *ws,
                          size_t ws_bytes, const int32_t *status, void *stream) {
    if (nblk < 0 || nq < 0 || (nq > 0 && (!comp || !comp_off || !qblk || !qpos || !sym || !ws || !status)))
        return PIVCO_ERR_INVALID_ARG;
    if (nq == 0) return PIVCO_OK;
    if (ws_bytes < decode_ws_fixed_bytes(nblk)) return PIVCO_ERR_CAPACITY;
    return ok_or_cuda(launch_access(comp, comp_off, nblk, qblk, qpos, nq, sym, qstatus,
                                    reinterpret_cast<const uint8_t *>(ws), ws_bytes, status, S(stream)));
}

pivco_status pivco_golomb_plan(const uint8_t *in, const uint64_t *blk_off, int32_t nblk, uint64_t *rec_size,
                               int32_t *status, void *stream) {
    if (nblk < 0 || (nblk > 0 && (!blk_off || !rec_size || !status))) return PIVCO_ERR_INVALID_ARG;
    return ok_or_cuda(launch_golomb_plan(in, blk_off, nblk, rec_size, status, S(stream)));
}

pivco_status pivco_golomb_encode(const uint8_t *in, const uint64_t *blk_off, int32_t nblk, uint8_t *out,
                                 const uint64_t *out_off, uint64_t *rec_bytes, int32_t *status, void *stream) {
    if (nblk < 0 || (nblk > 0 && (!blk_off || !out || !out_off || !rec_bytes || !status))) return PIVCO_ERR_INVALID_ARG;
    return ok_or_cuda(launch_golomb_encode(in, blk_off, nblk, out, out_off, rec_bytes, status, S(stream)));
}

pivco_status pivco_golomb_decode(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk, uint8_t *out,
                                 const uint64_t *out_off, int32_t *status, void *stream) {
    if (nblk < 0 || (nblk > 0 && (!comp || !comp_off || !out_off || !status))) return PIVCO_ERR_INVALID_ARG;
    return ok_or_cuda(launch_golomb_decode(comp, comp_off, nblk, out, out_off, status, S(stream)));
}

uint64_t pivco_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

pivco_status pivco_set_wait_limit(uint64_t ns) {
    g_wait_limit.store(ns, std::memory_order_relaxed);
    return PIVCO_OK;
}

uint64_t pivco_get_wait_limit(void) { return wait_limit_ns(); }

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

// ---------------------------------------------------------------------------
// Batching: persistent work-queue decode, tuning, graph capture, autotuner
// ---------------------------------------------------------------------------
pivco_status pivco_decode_batched(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk, uint8_t *out,
                                  const uint64_t *out_off, void *ws, size_t ws_bytes, int32_t *status, void *stream) {
    if (nblk < 0 || (nblk > 0 && (!comp || !comp_off || !out_off || !ws || !status))) return PIVCO_ERR_INVALID_ARG;
    if (nblk == 0) return PIVCO_OK;
    if (ws_bytes < decode_ws_fixed_bytes(nblk)) return PIVCO_ERR_CAPACITY;
    return ok_or_cuda(launch_decode_batch(comp, comp_off, nblk, out, out_off, reinterpret_cast<uint8_t *>(ws), ws_bytes,
                                          status, S(stream)));
}

pivco_status pivco_get_tuning(pivco_tuning *t) {
    if (!t) return PIVCO_ERR_INVALID_ARG;
    const DecTuning c = current_tuning();
    t->tile_max = (int32_t)c.tile_max;
    t->dir_bits = (int32_t)c.dir_bits;
    t->ctas_per_sm = (int32_t)c.ctas_per_sm;
    t->reserved = 0;
    return PIVCO_OK;
}

pivco_status pivco_set_tuning(const pivco_tuning *t) {
    if (!t || t->tile_max < 128 || t->tile_max > (1 << 20) || (t->tile_max & 127) || t->dir_bits < 32 ||
        t->dir_bits > 256 || (t->dir_bits & 31) || t->ctas_per_sm < 0 || t->ctas_per_sm > 32)
        return PIVCO_ERR_INVALID_ARG;
    set_tuning(DecTuning{(uint32_t)t->tile_max, (uint32_t)t->dir_bits, (uint32_t)t->ctas_per_sm});
    return PIVCO_OK;
}

struct pivco_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

pivco_status pivco_graph_begin(void *stream) {
    if (!stream) return PIVCO_ERR_INVALID_ARG;   // the legacy stream cannot be captured
    // kernel attributes and the ANS tables are set up outside the capture
    host_ans_tables();
    if (prepare_decode_kernels() != cudaSuccess || prepare_encode_kernels() != cudaSuccess ||
        prepare_ans_kernels() != cudaSuccess || prepare_golomb_kernels() != cudaSuccess)
        return PIVCO_ERR_CUDA;
    return ok_or_cuda(cudaStreamBeginCapture(S(stream), cudaStreamCaptureModeThreadLocal));
}

pivco_status pivco_graph_end(void *stream, pivco_graph **out) {
    if (!stream || !out) return PIVCO_ERR_INVALID_ARG;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(S(stream), &g);
    if (e != cudaSuccess) return PIVCO_ERR_CUDA;
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return PIVCO_ERR_CUDA;
    }
    pivco_graph *h = new pivco_graph{g, x};
    *out = h;
    return PIVCO_OK;
}

pivco_status pivco_graph_launch(pivco_graph *g, void *stream) {
    if (!g) return PIVCO_ERR_INVALID_ARG;
    return ok_or_cuda(cudaGraphLaunch(g->exec, S(stream)));
}

pivco_status pivco_graph_destroy(pivco_graph *g) {
    if (!g) return PIVCO_OK;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return PIVCO_OK;
}

pivco_status pivco_autotune_decode(const uint8_t *comp, const uint64_t *comp_off, int32_t nblk, uint8_t *out,
                                   const uint64_t *out_off, void *ws, size_t ws_bytes, int32_t *status, int32_t reps,
                                   void *stream, pivco_tuning *best, float *best_ms) {
    if (nblk <= 0 || !comp || !comp_off || !out_off || !ws || !status || !best || reps < 1) return PIVCO_ERR_INVALID_ARG;
    static const uint32_t tiles[] = {16384, 65536, 1u << 20};
    static const uint32_t dirs[] = {64, 128, 256};
    static const uint32_t ctas[] = {0, 2};
    const DecTuning saved = current_tuning();
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PIVCO_ERR_CUDA;
    float bms = 1e30f;
    DecTuning bt = saved;
    std::vector<int32_t> st_host((size_t)nblk);
    pivco_status rc = PIVCO_OK;
    for (uint32_t tm : tiles)
        for (uint32_t db : dirs)
            for (uint32_t cs : ctas) {
                if (rc != PIVCO_OK) break;   // a CUDA error ends the whole search
                set_tuning(DecTuning{tm, db, cs});
                // the workspace this tuning needs (tile cursors and directories grow as
                // tiles shrink): a candidate that does not fit is skipped, not timed
                cudaError_t e = launch_decode_plan(comp, comp_off, nblk, reinterpret_cast<uint8_t *>(ws), ws_bytes,
                                                   status, S(stream));
                size_t need = 0;
                e = e == cudaSuccess ? read_decode_ws_need(reinterpret_cast<const uint8_t *>(ws), nblk, &need,
                                                           S(stream)) : e;
                if (e != cudaSuccess) { rc = PIVCO_ERR_CUDA; break; }
                if (need > ws_bytes) continue;
                // one warm launch, then the timed ones
                e = launch_decode_batch(comp, comp_off, nblk, out, out_off, reinterpret_cast<uint8_t *>(ws), ws_bytes,
                                        status, S(stream));
                e = e == cudaSuccess ? cudaEventRecord(e0, S(stream)) : e;
                for (int r = 0; r < reps && e == cudaSuccess; r++)
                    e = launch_decode_batch(comp, comp_off, nblk, out, out_off, reinterpret_cast<uint8_t *>(ws), ws_bytes,
                                            status, S(stream));
                e = e == cudaSuccess ? cudaEventRecord(e1, S(stream)) : e;
                e = e == cudaSuccess ? cudaEventSynchronize(e1) : e;
                float ms = 0;
                e = e == cudaSuccess ? cudaEventElapsedTime(&ms, e0, e1) : e;
                e = e == cudaSuccess ? cudaMemcpyAsync(st_host.data(), status, sizeof(int32_t) * (size_t)nblk,
                                                       cudaMemcpyDeviceToHost, S(stream)) : e;
                e = e == cudaSuccess ? cudaStreamSynchronize(S(stream)) : e;
                if (e != cudaSuccess) { rc = PIVCO_ERR_CUDA; break; }
                bool clean = true;
                for (int32_t x : st_host) clean = clean && x == PIVCO_OK;
                if (!clean) continue;     // corrupt input or a failed tuning: never chosen
                ms /= (float)reps;
                if (ms < bms) { bms = ms; bt = DecTuning{tm, db, cs}; }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == PIVCO_OK && bms >= 1e30f) rc = PIVCO_ERR_CAPACITY;
    set_tuning(rc == PIVCO_OK ? bt : saved);
    if (rc == PIVCO_OK) {
        best->tile_max = (int32_t)bt.tile_max;
        best->dir_bits = (int32_t)bt.dir_bits;
        best->ctas_per_sm = (int32_t)bt.ctas_per_sm;
        best->reserved = 0;
        if (best_ms) *best_ms = bms;
    }
    return rc;
}

}  // extern "C"
