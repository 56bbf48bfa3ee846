// Host-buffer codec (host side): compress and decompress batches that live in
// host memory, with the host<->device copies overlapped with the kernels.
// The blocks are cut into segments of about equal raw size; segment s is
// copied in on one stream while earlier segments are coded on two compute
// streams (alternating, so that one segment's kernels fill the other's
// tail) and copied out on a fourth.  Every segment has its own
// device buffers, sized once at creation (compressed bytes: the record bound
// of every block), so a call allocates nothing unless a compressed input is
// larger than the codec's own output could be.
#include <algorithm>
#include <cstring>
#include <vector>

#include "pivco_dev.cuh"

namespace pv {
namespace {

constexpr size_t kAl = 256;
inline size_t al(size_t x) { return (x + kAl - 1) & ~(kAl - 1); }

// the largest record a block of n symbols can have: the fixed tables
// (header, lengths, n_v and markers of 255 nodes, alen words) and at most
// max_len bits per symbol spread over 255 bodies, rounded to 16
inline uint64_t rec_cap(uint64_t n) { return 2 * n + 2720; }

struct Seg {
    int b0 = 0, nb = 0;
    uint64_t r0 = 0, rn = 0;            // raw byte range
    uint64_t *boff = nullptr;           // nb + 1 block offsets, relative to r0
    uint32_t *hist = nullptr, *chunk = nullptr;
    uint8_t *lens = nullptr, *layout = nullptr;
    uint64_t *bound = nullptr, *off = nullptr, *rec_bytes = nullptr, *coff = nullptr;
    int32_t *status = nullptr, *dstatus = nullptr;
    uint8_t *scan_ws = nullptr, *comp = nullptr, *ans_ws = nullptr, *dws = nullptr;
    uint64_t comp_cap = 0;
    size_t ans_ws_bytes = 0, dws_bytes = 0;
    void *block = nullptr;              // the fixed buffers above, one allocation
};

}  // namespace
}  // namespace pv

struct pivco_host_codec {
    int nblk = 0, nseg = 0, dev = 0;
    pivco_params prm{};
    std::vector<uint64_t> blk_off;
    std::vector<pv::Seg> seg;
    cudaStream_t cmps[2] = {nullptr, nullptr}, h2d = nullptr, d2h = nullptr;
    std::vector<cudaEvent_t> ev_in, ev_sz, ev_done;
    uint8_t *d_in = nullptr, *d_out = nullptr;
    uint64_t *h_off = nullptr;          // pinned: per segment nb + 1 offsets
    uint64_t *h_coff = nullptr;         // pinned: relative compressed offsets
    int32_t *h_status = nullptr;        // pinned: nblk
    uint64_t comp_capacity = 0;
};

namespace {

using pv::Seg;
using pv::al;

cudaError_t free_all(pivco_host_codec *c) {
    for (Seg &s : c->seg) {
        cudaFree(s.block);
        cudaFree(s.comp);
        cudaFree(s.ans_ws);
        cudaFree(s.dws);
    }
    cudaFree(c->d_in);
    cudaFree(c->d_out);
    cudaFreeHost(c->h_off);
    cudaFreeHost(c->h_coff);
    cudaFreeHost(c->h_status);
    for (auto e : c->ev_in) cudaEventDestroy(e);
    for (auto e : c->ev_sz) cudaEventDestroy(e);
    for (auto e : c->ev_done) cudaEventDestroy(e);
    for (auto st : c->cmps)
        if (st) cudaStreamDestroy(st);
    if (c->h2d) cudaStreamDestroy(c->h2d);
    if (c->d2h) cudaStreamDestroy(c->d2h);
    return cudaGetLastError();
}

pivco_status wait_all(pivco_host_codec *c, cudaError_t e) {
    const cudaError_t e1 = cudaStreamSynchronize(c->h2d), e2 = cudaStreamSynchronize(c->cmps[0]),
                      e4 = cudaStreamSynchronize(c->cmps[1]), e3 = cudaStreamSynchronize(c->d2h);
    if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : (e4 != cudaSuccess ? e4 : e3));
    return e == cudaSuccess ? PIVCO_OK : PIVCO_ERR_CUDA;
}

#define HC_TRY(x)                              \
    do {                                       \
        const cudaError_t e_ = (x);            \
        if (e_ != cudaSuccess) return wait_all(c, e_); \
    } while (0)

}  // namespace

extern "C" {

pivco_status pivco_host_codec_create(const uint64_t *blk_off, int32_t nblk, const pivco_params *params,
                                     int32_t segments, pivco_host_codec **codec) {
    if (!codec || !params || nblk < 0 || (nblk > 0 && !blk_off) || segments < 1) return PIVCO_ERR_INVALID_ARG;
    const pivco_params &p = *params;
    if (p.max_len < 1 || p.max_len > (int32_t)pv::kMaxLen || p.ans_min_bytes < 0 || p.ans_skew_den <= 0 ||
        p.ans_skew_num < 0 || p.ans_ratio_pct < 0 || (p.flat != 0 && p.flat != 1))
        return PIVCO_ERR_INVALID_ARG;
    if (nblk > 0 && blk_off[0] != 0) return PIVCO_ERR_INVALID_ARG;
    for (int b = 0; b < nblk; b++)
        if (blk_off[b + 1] < blk_off[b] || blk_off[b + 1] - blk_off[b] > 0xFFFFFFFFull) return PIVCO_ERR_INVALID_ARG;
    *codec = nullptr;
    auto *c = new pivco_host_codec();
    c->nblk = nblk;
    c->prm = p;
    c->blk_off.assign(blk_off, blk_off + nblk + 1);
    cudaGetDevice(&c->dev);
    // segments of about equal raw size (at least one block each)
    const int nseg = nblk == 0 ? 0 : (segments < nblk ? segments : nblk);
    const uint64_t total = nblk ? blk_off[nblk] : 0;
    c->nseg = nseg;
    c->seg.resize(nseg);
    int b = 0;
    for (int s = 0; s < nseg; s++) {
        Seg &g = c->seg[s];
        g.b0 = b;
        const uint64_t want = total / nseg * (uint64_t)(s + 1);
        int e = b + 1;
        const int max_e = nblk - (nseg - 1 - s);   // leave a block for each later segment
        while (e < max_e && blk_off[e] < want) e++;
        if (s == nseg - 1) e = nblk;
        g.nb = e - b;
        g.r0 = blk_off[b];
        g.rn = blk_off[e] - blk_off[b];
        b = e;
    }
    cudaError_t err = cudaSuccess;
    auto ok = [&](cudaError_t e) { if (e != cudaSuccess && err == cudaSuccess) err = e; return err == cudaSuccess; };
    ok(cudaStreamCreateWithFlags(&c->cmps[0], cudaStreamNonBlocking));
    ok(cudaStreamCreateWithFlags(&c->cmps[1], cudaStreamNonBlocking));
    ok(cudaStreamCreateWithFlags(&c->h2d, cudaStreamNonBlocking));
    ok(cudaStreamCreateWithFlags(&c->d2h, cudaStreamNonBlocking));
    c->ev_in.assign(nseg, nullptr);
    c->ev_sz.assign(nseg, nullptr);
    c->ev_done.assign(nseg, nullptr);
    for (int s = 0; s < nseg && err == cudaSuccess; s++) {
        ok(cudaEventCreateWithFlags(&c->ev_in[s], cudaEventDisableTiming));
        ok(cudaEventCreateWithFlags(&c->ev_sz[s], cudaEventDisableTiming));
        ok(cudaEventCreateWithFlags(&c->ev_done[s], cudaEventDisableTiming));
    }
    if (err == cudaSuccess && total) {
        ok(cudaMalloc(&c->d_in, total));
        ok(cudaMalloc(&c->d_out, total));
    }
    if (err == cudaSuccess) {
        ok(cudaHostAlloc(&c->h_off, 8 * ((size_t)nblk + nseg + 1), cudaHostAllocDefault));
        ok(cudaHostAlloc(&c->h_coff, 8 * ((size_t)nblk + nseg + 1), cudaHostAllocDefault));
        ok(cudaHostAlloc(&c->h_status, 4 * ((size_t)nblk + 1), cudaHostAllocDefault));
    }
    std::vector<uint64_t> rel;
    for (int s = 0; s < nseg && err == cudaSuccess; s++) {
        Seg &g = c->seg[s];
        const size_t nb = (size_t)g.nb;
        // one allocation for the fixed per-block buffers
        size_t o = 0;
        const size_t o_boff = o; o += al(8 * (nb + 1));
        const size_t o_hist = o; o += al(4 * 256 * nb);
        const size_t o_chunk = o; o += al(4 * 256 * pv::kEncChunks * nb);
        const size_t o_lens = o; o += al(256 * nb);
        const size_t o_layout = o; o += al((size_t)pv::kLayoutBytes * nb);
        const size_t o_bound = o; o += al(8 * nb);
        const size_t o_off = o; o += al(8 * (nb + 1));
        const size_t o_rb = o; o += al(8 * nb);
        const size_t o_coff = o; o += al(8 * (nb + 1));
        const size_t o_st = o; o += al(4 * nb);
        const size_t o_dst = o; o += al(4 * nb);
        const size_t o_scan = o; o += al(pv::scan_ws_bytes((int)nb));
        if (!ok(cudaMalloc(&g.block, o))) break;
        uint8_t *base = reinterpret_cast<uint8_t *>(g.block);
        g.boff = reinterpret_cast<uint64_t *>(base + o_boff);
        g.hist = reinterpret_cast<uint32_t *>(base + o_hist);
        g.chunk = reinterpret_cast<uint32_t *>(base + o_chunk);
        g.lens = base + o_lens;
        g.layout = base + o_layout;
        g.bound = reinterpret_cast<uint64_t *>(base + o_bound);
        g.off = reinterpret_cast<uint64_t *>(base + o_off);
        g.rec_bytes = reinterpret_cast<uint64_t *>(base + o_rb);
        g.coff = reinterpret_cast<uint64_t *>(base + o_coff);
        g.status = reinterpret_cast<int32_t *>(base + o_st);
        g.dstatus = reinterpret_cast<int32_t *>(base + o_dst);
        g.scan_ws = base + o_scan;
        g.comp_cap = 0;
        for (int k = 0; k < g.nb; k++) g.comp_cap += pv::rec_cap(blk_off[g.b0 + k + 1] - blk_off[g.b0 + k]);
        c->comp_capacity += g.comp_cap;
        if (!ok(cudaMalloc(&g.comp, g.comp_cap ? g.comp_cap : 16))) break;
        if (p.ans_enable) {
            g.ans_ws_bytes = g.comp_cap + 256 * nb;
            if (!ok(cudaMalloc(&g.ans_ws, g.ans_ws_bytes))) break;
        }
        rel.resize(nb + 1);
        for (size_t k = 0; k <= nb; k++) rel[k] = blk_off[g.b0 + k] - g.r0;
        ok(cudaMemcpy(g.boff, rel.data(), 8 * (nb + 1), cudaMemcpyHostToDevice));
    }
    if (err == cudaSuccess) err = pv::prepare_encode_kernels();
    if (err == cudaSuccess) err = pv::prepare_decode_kernels();
    if (err == cudaSuccess && p.ans_enable) err = pv::prepare_ans_kernels();
    if (err != cudaSuccess) {
        free_all(c);
        delete c;
        return PIVCO_ERR_CUDA;
    }
    *codec = c;
    return PIVCO_OK;
}

pivco_status pivco_host_codec_destroy(pivco_host_codec *c) {
    if (!c) return PIVCO_ERR_INVALID_ARG;
    cudaSetDevice(c->dev);
    cudaStreamSynchronize(c->h2d);
    cudaStreamSynchronize(c->cmps[0]);
    cudaStreamSynchronize(c->cmps[1]);
    cudaStreamSynchronize(c->d2h);
    const cudaError_t e = free_all(c);
    delete c;
    return e == cudaSuccess ? PIVCO_OK : PIVCO_ERR_CUDA;
}

uint64_t pivco_host_codec_comp_capacity(const pivco_host_codec *c) { return c ? c->comp_capacity : 0; }

pivco_status pivco_host_compress(pivco_host_codec *c, const uint8_t *in, uint8_t *comp, uint64_t comp_cap,
                                 uint64_t *comp_off, int32_t *status) {
    if (!c || !comp_off || (c->nblk > 0 && (!status || (c->blk_off[c->nblk] && !in) || !comp)))
        return PIVCO_ERR_INVALID_ARG;
    cudaSetDevice(c->dev);
    comp_off[0] = 0;
    if (c->nblk == 0) return PIVCO_OK;
    // everything that needs no host decision: copies in, then plan, place and code each segment
    size_t ho = 0;
    for (int s = 0; s < c->nseg; s++) {
        Seg &g = c->seg[s];
        cudaStream_t cmp = c->cmps[s & 1];
        if (g.rn) HC_TRY(cudaMemcpyAsync(c->d_in + g.r0, in + g.r0, g.rn, cudaMemcpyHostToDevice, c->h2d));
        HC_TRY(cudaEventRecord(c->ev_in[s], c->h2d));
        HC_TRY(cudaStreamWaitEvent(cmp, c->ev_in[s], 0));
        const uint8_t *src = c->d_in + g.r0;
        HC_TRY(pv::launch_block_plan(src, g.boff, g.nb, c->prm, g.hist, g.chunk, g.lens,
                                     reinterpret_cast<pv::BlockLayout *>(g.layout), g.bound, g.status, cmp));
        HC_TRY(pv::launch_scan(g.bound, g.nb, g.off, g.scan_ws, g.status, cmp));
        HC_TRY(pv::launch_encode(src, g.boff, g.nb, reinterpret_cast<pv::BlockLayout *>(g.layout), g.chunk,
                                 g.comp, g.off, g.rec_bytes, g.status, cmp));
        if (c->prm.ans_enable)
            HC_TRY(pv::launch_ans_encode_blocks(reinterpret_cast<const pv::BlockLayout *>(g.layout), g.nb, g.comp,
                                                g.off, g.rec_bytes, g.ans_ws, g.ans_ws_bytes, g.status, cmp));
        HC_TRY(cudaMemcpyAsync(c->h_off + ho, g.off, 8 * ((size_t)g.nb + 1), cudaMemcpyDeviceToHost, cmp));
        HC_TRY(cudaMemcpyAsync(c->h_status + g.b0, g.status, 4 * (size_t)g.nb, cudaMemcpyDeviceToHost, cmp));
        HC_TRY(cudaEventRecord(c->ev_sz[s], cmp));
        ho += (size_t)g.nb + 1;
    }
    // each segment's records go out as soon as their size is known
    uint64_t base = 0;
    bool room = true;
    ho = 0;
    for (int s = 0; s < c->nseg; s++) {
        Seg &g = c->seg[s];
        HC_TRY(cudaEventSynchronize(c->ev_sz[s]));
        const uint64_t *o = c->h_off + ho;
        const uint64_t size = o[g.nb];
        if (size > g.comp_cap || base + size > comp_cap) room = false;
        if (room) {
            HC_TRY(cudaStreamWaitEvent(c->d2h, c->ev_sz[s], 0));
            if (size) HC_TRY(cudaMemcpyAsync(comp + base, g.comp, size, cudaMemcpyDeviceToHost, c->d2h));
        }
        for (int k = 0; k < g.nb; k++) comp_off[g.b0 + k] = base + o[k];
        base += size;
        ho += (size_t)g.nb + 1;
    }
    comp_off[c->nblk] = base;
    const pivco_status st = wait_all(c, cudaSuccess);
    if (st != PIVCO_OK) return st;
    memcpy(status, c->h_status, 4 * (size_t)c->nblk);
    return room ? PIVCO_OK : PIVCO_ERR_CAPACITY;
}

pivco_status pivco_host_decompress(pivco_host_codec *c, const uint8_t *comp, const uint64_t *comp_off, uint8_t *out,
                                   int32_t *status) {
    if (!c || !comp_off || (c->nblk > 0 && (!status || (c->blk_off[c->nblk] && !out))))
        return PIVCO_ERR_INVALID_ARG;
    cudaSetDevice(c->dev);
    if (c->nblk == 0) return PIVCO_OK;
    for (int b = 0; b < c->nblk; b++)
        if (comp_off[b + 1] < comp_off[b]) return PIVCO_ERR_INVALID_ARG;
    if (comp_off[c->nblk] > comp_off[0] && !comp) return PIVCO_ERR_INVALID_ARG;
    const pv::DecTuning tu = pv::current_tuning();
    // sizes from the host records first (relative offsets, workspace bounds, room for the records)
    size_t ho = 0;
    for (int s = 0; s < c->nseg; s++) {
        Seg &g = c->seg[s];
        const uint64_t c0 = comp_off[g.b0], cn = comp_off[g.b0 + g.nb] - c0;
        uint64_t *rel = c->h_coff + ho;
        for (int k = 0; k <= g.nb; k++) rel[k] = comp_off[g.b0 + k] - c0;
        // from the block sizes alone (reading every record's node table on
        // the host would cost more than the copies)
        const size_t need = std::max(pv::decode_ws_size_bound(c->blk_off.data() + g.b0, g.nb, tu),
                                     pv::decode_ws_fixed_bytes(g.nb));
        // (every stream is idle between calls)
        if (cn > g.comp_cap) {
            cudaFree(g.comp);
            g.comp = nullptr;
            HC_TRY(cudaMalloc(&g.comp, cn));
            g.comp_cap = cn;
        }
        if (need > g.dws_bytes) {
            cudaFree(g.dws);
            g.dws = nullptr;
            g.dws_bytes = 0;
            HC_TRY(cudaMalloc(&g.dws, need));
            g.dws_bytes = need;
        }
        ho += (size_t)g.nb + 1;
    }
    ho = 0;
    for (int s = 0; s < c->nseg; s++) {
        Seg &g = c->seg[s];
        const uint64_t c0 = comp_off[g.b0], cn = comp_off[g.b0 + g.nb] - c0;
        cudaStream_t cmp = c->cmps[s & 1];
        HC_TRY(cudaMemcpyAsync(g.coff, c->h_coff + ho, 8 * ((size_t)g.nb + 1), cudaMemcpyHostToDevice, c->h2d));
        if (cn) HC_TRY(cudaMemcpyAsync(g.comp, comp + c0, cn, cudaMemcpyHostToDevice, c->h2d));
        HC_TRY(cudaEventRecord(c->ev_in[s], c->h2d));
        HC_TRY(cudaStreamWaitEvent(cmp, c->ev_in[s], 0));
        HC_TRY(pv::launch_decode_batch(g.comp, g.coff, g.nb, c->d_out + g.r0, g.boff, g.dws, g.dws_bytes, g.dstatus,
                                       cmp));
        HC_TRY(cudaMemcpyAsync(c->h_status + g.b0, g.dstatus, 4 * (size_t)g.nb, cudaMemcpyDeviceToHost, cmp));
        HC_TRY(cudaEventRecord(c->ev_done[s], cmp));
        HC_TRY(cudaStreamWaitEvent(c->d2h, c->ev_done[s], 0));
        if (g.rn) HC_TRY(cudaMemcpyAsync(out + g.r0, c->d_out + g.r0, g.rn, cudaMemcpyDeviceToHost, c->d2h));
        ho += (size_t)g.nb + 1;
    }
    const pivco_status st = wait_all(c, cudaSuccess);
    if (st != PIVCO_OK) return st;
    memcpy(status, c->h_status, 4 * (size_t)c->nblk);
    return PIVCO_OK;
}

}  // extern "C"
