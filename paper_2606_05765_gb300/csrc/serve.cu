// Serving runtime (host side): admission by device-memory budget, the
// request ring, launches of the device-resident loop (serve_loop_kernel),
// result copies and retirement.  One scheduler thread owns every CUDA call
// of a server; pivco_server_submit / poll / drain only exchange requests with
// it under a mutex.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "pivco_dev.cuh"

namespace pv {
namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }
inline double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with coalescing; offsets are kAlign-aligned.
class Arena {
public:
    void reset(size_t size) { free_.clear(); if (size) free_[0] = size; }
    bool alloc(size_t n, size_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
        if (it != free_.begin()) {
            auto pv_ = std::prev(it);
            if (pv_->first + pv_->second == it->first) { pv_->second += it->second; free_.erase(it); }
        }
    }
private:
    std::map<size_t, size_t> free_;
};

enum ReqState : int32_t { kUnknown = 0, kPending = 1, kRunning = 2, kDone = 3 };

struct Request {
    uint64_t seq = 0;
    const uint8_t *comp_h = nullptr;
    uint8_t *out_h = nullptr;
    std::vector<uint64_t> comp_off, out_off;   // host copies (comp_off rebased to 0)
    int32_t nblk = 0;
    size_t comp_bytes = 0, raw_bytes = 0, ws_bytes = 0, need = 0, arena_off = 0;
    std::atomic<int> stage{0}; // 0 pending, 1 copying in, 2 published, 3 copying out, 4 finished
    bool retired = false;
    int32_t status = PIVCO_OK;
    double t_submit = 0, t_done = 0;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<uint8_t> hdr;  // workspace header image (64 bytes)
};

struct Launch {
    uint64_t gen;
    cudaEvent_t ev;
    uint32_t *snap;            // pinned: ctl->cur when the launch ended
};

}  // namespace
}  // namespace pv

struct pivco_server {
    int device = 0;
    uint8_t *arena = nullptr;      // caller's device memory
    size_t arena_bytes = 0, budget = 0, used = 0;
    pv::Arena alloc;
    pv::ServeCtl *ctl = nullptr;   // inside the arena
    pv::ServeDesc *ring_d = nullptr;
    pv::ServeDesc *ring_h = nullptr;   // pinned staging of ring entries
    pv::ServeFlags *flags = nullptr;   // pinned, mapped
    pv::ServeFlags *flags_d = nullptr;
    uint32_t *snaps = nullptr;         // pinned launch snapshots
    uint8_t *zeros = nullptr;          // pinned zero page for workspace headers and states
    size_t zeros_bytes = 0;
    cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
    uint64_t idle_ns = 200000, life_ns = 4000000;

    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<pv::Request>> pending;            // submitted, not admitted
    std::map<uint64_t, std::shared_ptr<pv::Request>> live;       // admitted, not retired
    std::map<uint64_t, std::shared_ptr<pv::Request>> finished;   // results ready (kept for poll)
    uint64_t next_id = 0;      // ids handed out by submit (== seq: admission is in order)
    std::thread th;
    std::atomic<bool> quit{false};
    std::atomic<int> fatal{PIVCO_OK};
    uint64_t admit_next = 0;   // requests below this were admitted (admission is in id order)

    // scheduler-thread state
    uint64_t published = 0, next_seq = 0, gen = 0;
    uint64_t cur_done = 0;                 // ctl->cur seen at the end of the latest finished launch
    std::deque<pv::Launch> launches;       // in stream order
    std::vector<cudaEvent_t> ev_pool;
    std::vector<bool> slot_busy;

    cudaEvent_t get_event() {
        if (!ev_pool.empty()) { cudaEvent_t e = ev_pool.back(); ev_pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        return e;
    }
    void put_event(cudaEvent_t e) { if (e) ev_pool.push_back(e); }

    std::vector<uint8_t *> old_zeros;   // outgrown zero pages (copies may still read them)
    bool ensure_zeros(size_t n) {
        if (n <= zeros_bytes) return true;
        if (zeros) old_zeros.push_back(zeros);
        zeros = nullptr;
        zeros_bytes = 0;
        size_t sz = std::max(n, (size_t)1 << 20);
        if (cudaHostAlloc((void **)&zeros, sz, cudaHostAllocDefault) != cudaSuccess) return false;
        memset(zeros, 0, sz);
        zeros_bytes = sz;
        return true;
    }

    // admission: the oldest submitted requests while they fit the budget and the arena
    bool admit() {
        bool progress = false;
        for (;;) {
            std::shared_ptr<pv::Request> r;
            {
                std::lock_guard<std::mutex> lk(mu);
                if (pending.empty()) break;
                r = pending.front();
                if (used + r->need > budget) break;
                const uint32_t slot = (uint32_t)(r->seq % pv::kServeRing);
                if (slot_busy[slot]) break;
                size_t off = 0;
                if (!alloc.alloc(r->need, &off)) break;
                r->arena_off = off;
                used += r->need;
                slot_busy[slot] = true;
                pending.pop_front();
                admit_next = r->seq + 1;
                live[r->seq] = r;
                r->stage = 1;
            }
            // device layout of the request: records, offsets, statuses, workspace, output
            uint8_t *base = arena + r->arena_off;
            const size_t n1 = (size_t)r->nblk + 1;
            uint8_t *d_comp = base;
            uint64_t *d_coff = reinterpret_cast<uint64_t *>(base + pv::align_up(r->comp_bytes));
            uint64_t *d_ooff = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(d_coff) + pv::align_up(8 * n1));
            int32_t *d_st = reinterpret_cast<int32_t *>(reinterpret_cast<uint8_t *>(d_ooff) + pv::align_up(8 * n1));
            uint8_t *d_ws = reinterpret_cast<uint8_t *>(d_st) + pv::align_up(4 * (size_t)r->nblk);
            uint8_t *d_out = d_ws + r->ws_bytes;
            const size_t fixed = pv::decode_ws_fixed_bytes(r->nblk);
            cudaError_t e = ensure_zeros(fixed) ? cudaSuccess : cudaErrorMemoryAllocation;
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_ws, zeros, fixed, cudaMemcpyHostToDevice, s_in);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_ws, r->hdr.data(), r->hdr.size(), cudaMemcpyHostToDevice, s_in);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_st, zeros, 4 * (size_t)r->nblk, cudaMemcpyHostToDevice, s_in);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_comp, r->comp_h, r->comp_bytes, cudaMemcpyHostToDevice, s_in);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_coff, r->comp_off.data(), 8 * n1, cudaMemcpyHostToDevice, s_in);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_ooff, r->out_off.data(), 8 * n1, cudaMemcpyHostToDevice, s_in);
            const uint32_t slot = (uint32_t)(r->seq % pv::kServeRing);
            pv::ServeDesc &dsc = ring_h[slot];
            dsc.comp = d_comp;
            dsc.comp_off = d_coff;
            dsc.out = d_out;
            dsc.out_off = d_ooff;
            dsc.ws = d_ws;
            dsc.ws_bytes = r->ws_bytes;
            dsc.status = d_st;
            dsc.nblk = r->nblk;
            dsc.seq = (uint32_t)r->seq;
            if (e == cudaSuccess) e = cudaMemcpyAsync(ring_d + slot, &dsc, sizeof(dsc), cudaMemcpyHostToDevice, s_in);
            r->ev_in = get_event();
            if (e == cudaSuccess) e = r->ev_in ? cudaEventRecord(r->ev_in, s_in) : cudaErrorMemoryAllocation;
            if (e != cudaSuccess) { fatal = PIVCO_ERR_CUDA; return false; }
            progress = true;
        }
        return progress;
    }

    // publish, in sequence order, the requests whose inputs have landed
    bool publish() {
        bool progress = false;
        for (;;) {
            std::shared_ptr<pv::Request> r;
            {
                std::lock_guard<std::mutex> lk(mu);
                auto it = live.find(published);
                if (it == live.end() || it->second->stage != 1) break;
                r = it->second;
            }
            const cudaError_t q = cudaEventQuery(r->ev_in);
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess) { fatal = PIVCO_ERR_CUDA; return false; }
            put_event(r->ev_in);
            r->ev_in = nullptr;
            r->stage = 2;
            published++;
            std::atomic_thread_fence(std::memory_order_release);
            __atomic_store_n(&flags->tail, (uint32_t)published, __ATOMIC_RELEASE);
            progress = true;
        }
        return progress;
    }

    // keep one loop launch queued behind the running one while work is published
    bool launch_loop() {
        bool progress = false;
        while (!launches.empty()) {
            const cudaError_t q = cudaEventQuery(launches.front().ev);
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess) { fatal = PIVCO_ERR_CUDA; return false; }
            cur_done = std::max<uint64_t>(cur_done, *reinterpret_cast<volatile uint32_t *>(launches.front().snap));
            put_event(launches.front().ev);
            launches.pop_front();
            progress = true;
        }
        bool work = false;
        {
            std::lock_guard<std::mutex> lk(mu);
            // published requests to decode, and finished ones the device has not yet moved past
            for (auto &kv : live)
                if (kv.second->stage == 2 || (kv.second->stage == 4 && cur_done <= kv.first)) { work = true; break; }
        }
        if (work && launches.size() < 2) {
            pv::Launch L;
            L.gen = gen++;
            L.snap = snaps + (L.gen % 64);
            L.ev = get_event();
            cudaError_t e = L.ev ? pv::launch_serve_loop(ctl, ring_d, flags_d, idle_ns, life_ns, s_run)
                                 : cudaErrorMemoryAllocation;
            if (e == cudaSuccess) e = cudaMemcpyAsync(L.snap, &ctl->cur, 4, cudaMemcpyDeviceToHost, s_run);
            if (e == cudaSuccess) e = cudaEventRecord(L.ev, s_run);
            if (e != cudaSuccess) { fatal = PIVCO_ERR_CUDA; return false; }
            launches.push_back(L);
            progress = true;
        }
        return progress;
    }

    // decoded requests: copy results out; finished copies: hand to poll; retire memory
    bool complete() {
        bool progress = false;
        std::vector<std::shared_ptr<pv::Request>> rs;
        {
            std::lock_guard<std::mutex> lk(mu);
            for (auto &kv : live) rs.push_back(kv.second);
        }
        for (auto &r : rs) {
            const uint32_t slot = (uint32_t)(r->seq % pv::kServeRing);
            if (r->stage == 2 && r->nblk == 0) {   // nothing to decode: the device only steps over it
                r->t_done = pv::now_ms();
                {
                    std::lock_guard<std::mutex> lk(mu);
                    r->stage = 4;
                    finished[r->seq] = r;
                }
                cv.notify_all();
                progress = true;
            }
            if (r->stage == 2 &&
                __atomic_load_n(&flags->done[slot], __ATOMIC_ACQUIRE) == (uint32_t)(r->seq + 1)) {
                r->status = *reinterpret_cast<volatile int32_t *>(&flags->worst[slot]);
                const pv::ServeDesc &dsc = ring_h[slot];
                cudaError_t e = r->raw_bytes ? cudaMemcpyAsync(r->out_h, dsc.out, r->raw_bytes,
                                                               cudaMemcpyDeviceToHost, s_out) : cudaSuccess;
                r->ev_out = get_event();
                if (e == cudaSuccess) e = r->ev_out ? cudaEventRecord(r->ev_out, s_out) : cudaErrorMemoryAllocation;
                if (e != cudaSuccess) { fatal = PIVCO_ERR_CUDA; return false; }
                r->stage = 3;
                progress = true;
            }
            if (r->stage == 3) {
                const cudaError_t q = cudaEventQuery(r->ev_out);
                if (q == cudaErrorNotReady) continue;
                if (q != cudaSuccess) { fatal = PIVCO_ERR_CUDA; return false; }
                put_event(r->ev_out);
                r->ev_out = nullptr;
                r->t_done = pv::now_ms();
                {
                    std::lock_guard<std::mutex> lk(mu);
                    r->stage = 4;
                    finished[r->seq] = r;
                }
                cv.notify_all();
                progress = true;
            }
            // retire: no CTA of any later launch can reach a request below cur_done
            if (r->stage == 4 && !r->retired && cur_done > r->seq) {
                std::lock_guard<std::mutex> lk(mu);
                alloc.release(r->arena_off, r->need);
                used -= r->need;
                slot_busy[r->seq % pv::kServeRing] = false;
                r->retired = true;
                live.erase(r->seq);
                progress = true;
            }
        }
        return progress;
    }

    void run() {
        cudaSetDevice(device);
        while (!quit.load()) {
            bool p = admit();
            p |= publish();
            p |= launch_loop();
            p |= complete();
            if (fatal.load() != PIVCO_OK) {
                std::lock_guard<std::mutex> lk(mu);
                cv.notify_all();
                break;
            }
            if (!p) std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
};

extern "C" {

pivco_status pivco_server_create(void *arena, size_t arena_bytes, const pivco_server_config *cfg,
                                 pivco_server **out) {
    if (!arena || !out || (reinterpret_cast<uintptr_t>(arena) & 255)) return PIVCO_ERR_INVALID_ARG;
    const size_t reserved = pv::align_up(sizeof(pv::ServeCtl)) + pv::align_up(sizeof(pv::ServeDesc) * pv::kServeRing);
    if (arena_bytes <= reserved) return PIVCO_ERR_CAPACITY;
    std::unique_ptr<pivco_server> s(new pivco_server());
    if (cudaGetDevice(&s->device) != cudaSuccess) return PIVCO_ERR_CUDA;
    s->arena = reinterpret_cast<uint8_t *>(arena);
    s->ctl = reinterpret_cast<pv::ServeCtl *>(s->arena);
    s->ring_d = reinterpret_cast<pv::ServeDesc *>(s->arena + pv::align_up(sizeof(pv::ServeCtl)));
    s->arena_bytes = arena_bytes - reserved;
    s->arena = s->arena + reserved;
    s->budget = cfg && cfg->budget_bytes ? std::min<size_t>(cfg->budget_bytes, s->arena_bytes) : s->arena_bytes;
    if (cfg && cfg->idle_us > 0) s->idle_ns = 1000ull * (uint64_t)cfg->idle_us;
    if (cfg && cfg->epoch_us > 0) s->life_ns = 1000ull * (uint64_t)cfg->epoch_us;
    s->alloc.reset(s->arena_bytes);
    s->slot_busy.assign(pv::kServeRing, false);
    cudaError_t e = cudaHostAlloc((void **)&s->flags, sizeof(pv::ServeFlags), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        memset(s->flags, 0, sizeof(pv::ServeFlags));
        e = cudaHostGetDevicePointer((void **)&s->flags_d, s->flags, 0);
    }
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->ring_h, sizeof(pv::ServeDesc) * pv::kServeRing, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->snaps, 64 * sizeof(uint32_t), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_run, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_out, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = pv::prepare_decode_kernels();
    if (e == cudaSuccess) e = cudaMemsetAsync(s->ctl, 0, reserved, s->s_in);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->s_in);
    if (e != cudaSuccess) {
        pivco_server *raw = s.release();
        raw->quit = true;
        pivco_server_destroy(raw);
        return PIVCO_ERR_CUDA;
    }
    memset(s->snaps, 0, 64 * sizeof(uint32_t));
    pivco_server *raw = s.release();
    raw->th = std::thread([raw] { raw->run(); });
    *out = raw;
    return PIVCO_OK;
}

pivco_status pivco_server_submit(pivco_server *s, const uint8_t *comp, const uint64_t *comp_off, int32_t nblk,
                                 const uint64_t *out_off, uint8_t *out, uint64_t *id) {
    if (!s || !comp_off || !out_off || !id || nblk < 0) return PIVCO_ERR_INVALID_ARG;
    if (s->fatal.load() != PIVCO_OK) return (pivco_status)s->fatal.load();
    auto r = std::make_shared<pv::Request>();
    r->nblk = nblk;
    r->comp_off.resize((size_t)nblk + 1);
    r->out_off.resize((size_t)nblk + 1);
    for (int32_t b = 0; b <= nblk; b++) {
        r->comp_off[b] = comp_off[b] - comp_off[0];
        r->out_off[b] = out_off[b] - out_off[0];
        if (b && (comp_off[b] < comp_off[b - 1] || out_off[b] < out_off[b - 1])) return PIVCO_ERR_INVALID_ARG;
    }
    r->comp_bytes = r->comp_off[nblk];
    r->raw_bytes = r->out_off[nblk];
    if ((r->comp_bytes && !comp) || (r->raw_bytes && !out) || (comp_off[0] & 15)) return PIVCO_ERR_INVALID_ARG;
    r->comp_h = comp + comp_off[0];
    r->out_h = out + out_off[0];
    const pv::DecTuning tu = pv::current_tuning();
    // the workspace header and counters exist even for an empty request (the loop steps over it)
    r->ws_bytes = pv::align_up(std::max(nblk ? pv::decode_ws_bound(r->comp_h, r->comp_off.data(), nblk, tu) : (size_t)0,
                                        pv::decode_ws_fixed_bytes(nblk)));
    const size_t n1 = (size_t)nblk + 1;
    r->need = pv::align_up(r->comp_bytes) + 2 * pv::align_up(8 * n1) + pv::align_up(4 * (size_t)nblk) + r->ws_bytes +
              pv::align_up(r->raw_bytes);
    if (r->need > s->budget) return PIVCO_ERR_CAPACITY;
    r->hdr.assign(64, 0);
    memcpy(r->hdr.data() + 28, &tu.dir_bits, 4);
    memcpy(r->hdr.data() + 32, &tu.tile_max, 4);
    const uint64_t lim = pv::wait_limit_ns();
    memcpy(r->hdr.data() + 56, &lim, 8);
    r->t_submit = pv::now_ms();
    std::lock_guard<std::mutex> lk(s->mu);
    r->seq = s->next_id++;
    *id = r->seq;
    s->pending.push_back(r);
    return PIVCO_OK;
}

pivco_status pivco_server_poll(pivco_server *s, uint64_t id, int32_t *state, int32_t *status, double *latency_ms) {
    if (!s || !state) return PIVCO_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto f = s->finished.find(id);
    if (f != s->finished.end()) {
        *state = pv::kDone;
        if (status) *status = f->second->status;
        if (latency_ms) *latency_ms = f->second->t_done - f->second->t_submit;
        return PIVCO_OK;
    }
    if (status) *status = PIVCO_OK;
    if (latency_ms) *latency_ms = 0;
    *state = id >= s->next_id ? pv::kUnknown
             : id >= s->admit_next ? pv::kPending
             : s->live.count(id) ? pv::kRunning : pv::kUnknown;
    return (pivco_status)s->fatal.load();
}

pivco_status pivco_server_drain(pivco_server *s, int32_t timeout_ms) {
    if (!s) return PIVCO_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto until = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    for (;;) {
        if (s->fatal.load() != PIVCO_OK) return (pivco_status)s->fatal.load();
        bool all = s->pending.empty();
        for (auto &kv : s->live) if (kv.second->stage != 4) { all = false; break; }
        if (all) return PIVCO_OK;
        if (s->cv.wait_until(lk, until) == std::cv_status::timeout) {
            bool all2 = s->pending.empty();
            for (auto &kv : s->live) if (kv.second->stage != 4) { all2 = false; break; }
            return all2 ? PIVCO_OK : PIVCO_ERR_TIMEOUT;
        }
    }
}

pivco_status pivco_server_forget(pivco_server *s, uint64_t id) {
    if (!s) return PIVCO_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    s->finished.erase(id);
    return PIVCO_OK;
}

pivco_status pivco_server_destroy(pivco_server *s) {
    if (!s) return PIVCO_ERR_INVALID_ARG;
    if (s->flags) __atomic_store_n(&s->flags->stop, 1u, __ATOMIC_RELEASE);
    s->quit = true;
    if (s->th.joinable()) s->th.join();
    cudaSetDevice(s->device);
    pivco_status rc = PIVCO_OK;
    if (s->s_run && cudaStreamSynchronize(s->s_run) != cudaSuccess) rc = PIVCO_ERR_CUDA;
    if (s->s_in) cudaStreamSynchronize(s->s_in);
    if (s->s_out) cudaStreamSynchronize(s->s_out);
    for (auto &L : s->launches) cudaEventDestroy(L.ev);
    for (auto &kv : s->live) {
        if (kv.second->ev_in) cudaEventDestroy(kv.second->ev_in);
        if (kv.second->ev_out) cudaEventDestroy(kv.second->ev_out);
    }
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    if (s->s_in) cudaStreamDestroy(s->s_in);
    if (s->s_run) cudaStreamDestroy(s->s_run);
    if (s->s_out) cudaStreamDestroy(s->s_out);
    if (s->flags) cudaFreeHost(s->flags);
    if (s->ring_h) cudaFreeHost(s->ring_h);
    if (s->snaps) cudaFreeHost(s->snaps);
    if (s->zeros) cudaFreeHost(s->zeros);
    for (uint8_t *z : s->old_zeros) cudaFreeHost(z);
    delete s;
    return rc;
}

}  // extern "C"
