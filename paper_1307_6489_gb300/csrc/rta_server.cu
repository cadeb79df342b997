// The serving engine: a stream of telescope bundles processed with continuous
// batching under an HBM budget (the RTA processes the event builder's output
// as it arrives, Sec. 4.2, within the 30 s alert latency of Sec. 2.1).
//
// One scheduler thread owns the device side. Submitted bundles wait in a FIFO;
// the head is admitted as soon as a slot (a CUDA stream) is free and the
// budget arena has room for its buffers, so a bundle that arrives while others
// are on the GPU starts as soon as memory and a slot free up, and the copies
// and kernels of different bundles overlap on the device. Per bundle, on its
// slot stream: host-to-device copies, the fused image kernel, then the learned
// reconstruction (one kernel with no model workspace, so the learned stages of
// concurrent bundles overlap as well) or the geometric intersection, the
// sky-map fill on the map stream, and the copy of the event list back to the
// caller's host buffer. Completion is detected by polling a CUDA event; the
// bundle's arena range is freed only then. Timing events on the slot stream
// split each bundle's time into queue wait, copies in, device work and copy out.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rta.h"
#include "rta_launch.cuh"

namespace {

int vfail(int code, const char* fmt, ...) {
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    rta::set_last_error(msg);
    return code;
}

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

constexpr size_t kAlign = 256;
size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// First-fit sub-allocator over one device range (the HBM budget).
struct Arena {
    char* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;   // offset -> length
    void reset() {
        free_.clear();
        if (size) free_[0] = size;
    }
    bool alloc(size_t n, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, o = it->first;
                free_.erase(it);
                if (rest) free_[o + n] = rest;
                return true;
            }
        return false;
    }
    void release(size_t off, size_t n) {
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Layout {   // byte offsets of one bundle's buffers inside its arena range
    size_t wave, wave_off, img_tel, evt_off, hillas, events, stereo, total;
};

Layout layout_of(const rta_bundle_t& b, bool need_stereo) {
    Layout L;
    size_t o = 0;
    L.wave = o; o = up(o + size_t(b.n_wave) * 2);
    L.wave_off = o; o = up(o + size_t(b.n_img) * 8);
    L.img_tel = o; o = up(o + size_t(b.n_img) * 4);
    L.evt_off = o; o = up(o + size_t(b.n_evt + 1) * 4);
    L.hillas = o; o = up(o + size_t(b.n_img) * sizeof(rta_hillas_t));
    L.events = o; o = up(o + size_t(b.n_evt) * sizeof(rta_event_t));
    L.stereo = o; if (need_stereo) o = up(o + size_t(b.n_evt) * sizeof(rta_stereo_t));
    L.total = o;
    return L;
}

enum { REQ_PENDING = 0, REQ_RUNNING = 1, REQ_DONE = 2, REQ_FAILED = 3 };

struct Req {
    uint64_t ticket = 0;
    rta_bundle_t b{};
    Layout L{};
    size_t off = 0;
    int slot = -1;
    int state = REQ_PENDING;
    int rc = RTA_OK;
    int64_t done_ns = 0;
    rta_bundle_times_t times{};
};

struct Slot {
    cudaStream_t s = nullptr;
    cudaEvent_t e_ev = nullptr, e_map = nullptr, e_done = nullptr;
    cudaEvent_t t_in = nullptr, t_copied = nullptr, t_computed = nullptr, t_out = nullptr;   // timing
    uint64_t ticket = 0;
    bool busy = false;
    // pinned staging of the bundle's tables (in) and event list (out): copies from
    // and to pageable memory would block the scheduler thread (and with it every
    // other slot) until this slot's stream reached them
    char* h_stage = nullptr;
};

}  // namespace

struct rta_stream {
    rta_ctx* ctx = nullptr;
    rta_model* model = nullptr;
    int device = 0;
    int window_mode = 0, start = 0, W = 0, core_nb = 0;
    float t_hi = 0.f, t_lo = 0.f, fallback_deg = 0.5f;
    int64_t max_img = 0, max_evt = 0;
    Arena arena;
    std::vector<Slot> slots;
    cudaStream_t s_map = nullptr;
    unsigned int* d_slabs = nullptr;   // RTA_SKY_SLABS x 256 x 256
    unsigned int* d_slabs_min = nullptr;   // RTA_SKY_MIN_SLABS x 256 x 256
    unsigned int* d_map = nullptr;
    int64_t slab_sec[RTA_SKY_SLABS];
    int64_t slab_min[RTA_SKY_MIN_SLABS];
    // transient-search work buffers (grown on demand)
    unsigned int *d_won = nullptr, *d_woff = nullptr, *d_pre_on = nullptr, *d_pre_off = nullptr, *d_nal = nullptr;
    int* d_hw = nullptr;
    rta_alert_t* d_alerts = nullptr;
    size_t alerts_cap = 0;
    double* d_sig = nullptr;
    int64_t *d_son = nullptr, *d_soff = nullptr;
    // requests
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Req> reqs;
    uint64_t next_ticket = 1;
    int running = 0;
    bool stop = false;
    std::thread worker;
    int64_t n_done = 0, bytes_done = 0;
};

namespace {

int64_t floor_div(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Count events into the one-second slab of arrival_ns and the one-minute slab of
// its second, on the map stream, recycling a slab when a newer second (minute)
// claims it; events of a second (minute) that has left its ring are not counted.
// Caller holds S->mu.
cudaError_t fill_slabs(rta_stream* S, const rta_event_t* d_ev, int64_t n_evt, int64_t arrival_ns) {
    const int64_t sec = arrival_ns / 1000000000ll;
    const int slab = int(((sec % RTA_SKY_SLABS) + RTA_SKY_SLABS) % RTA_SKY_SLABS);
    const int64_t mnt = floor_div(sec, 60);
    const int mslab = int(((mnt % RTA_SKY_MIN_SLABS) + RTA_SKY_MIN_SLABS) % RTA_SKY_MIN_SLABS);
    const size_t map_bytes = sizeof(unsigned int) * RTA_SKY_N * RTA_SKY_N;
    unsigned int* p_sec = S->d_slabs + size_t(slab) * RTA_SKY_N * RTA_SKY_N;
    unsigned int* p_min = S->d_slabs_min + size_t(mslab) * RTA_SKY_N * RTA_SKY_N;
    cudaError_t e = cudaSuccess;
    if (S->slab_sec[slab] < sec) {
        e = cudaMemsetAsync(p_sec, 0, map_bytes, S->s_map);
        S->slab_sec[slab] = sec;
    }
    if (e == cudaSuccess && S->slab_min[mslab] < mnt) {
        e = cudaMemsetAsync(p_min, 0, map_bytes, S->s_map);
        S->slab_min[mslab] = mnt;
    }
    if (e != cudaSuccess || n_evt <= 0) return e;
    unsigned int* a = S->slab_sec[slab] == sec ? p_sec : nullptr;
    unsigned int* b = S->slab_min[mslab] == mnt ? p_min : nullptr;
    if (!a && !b) return cudaSuccess;
    return rta::launch_skymap_fill(d_ev, n_evt, a, b, S->s_map);
}

int dispatch(rta_stream* S, Req& r, Slot& sl) {
    const rta_bundle_t& b = r.b;
    char* base = S->arena.base + r.off;
    uint16_t* d_wave = reinterpret_cast<uint16_t*>(base + r.L.wave);
    int64_t* d_off = reinterpret_cast<int64_t*>(base + r.L.wave_off);
    int32_t* d_tel = reinterpret_cast<int32_t*>(base + r.L.img_tel);
    int32_t* d_evt = reinterpret_cast<int32_t*>(base + r.L.evt_off);
    rta_hillas_t* d_h = reinterpret_cast<rta_hillas_t*>(base + r.L.hillas);
    rta_event_t* d_ev = reinterpret_cast<rta_event_t*>(base + r.L.events);
    rta_stereo_t* d_st = reinterpret_cast<rta_stereo_t*>(base + r.L.stereo);
    cudaStream_t s = sl.s;
    r.times.admit_ns = now_ns();
    r.times.slot = int(&sl - &S->slots[0]);
#define D_TRY(call)                                                                                 \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return vfail(RTA_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)
    // the tables through the slot's pinned staging (the slot's previous bundle, the
    // last user of it, has completed), in the order of the device layout
    const size_t tb_off = size_t(b.n_img) * 8, tb_tel = size_t(b.n_img) * 4, tb_evt = size_t(b.n_evt + 1) * 4;
    std::memcpy(sl.h_stage, b.h_wave_off, tb_off);
    std::memcpy(sl.h_stage + tb_off, b.h_img_tel, tb_tel);
    std::memcpy(sl.h_stage + tb_off + tb_tel, b.h_evt_off, tb_evt);
    D_TRY(cudaEventRecord(sl.t_in, s));
    D_TRY(cudaMemcpyAsync(d_wave, b.h_wave, size_t(b.n_wave) * 2, cudaMemcpyHostToDevice, s));
    D_TRY(cudaMemcpyAsync(d_off, sl.h_stage, tb_off, cudaMemcpyHostToDevice, s));
    D_TRY(cudaMemcpyAsync(d_tel, sl.h_stage + tb_off, tb_tel, cudaMemcpyHostToDevice, s));
    D_TRY(cudaMemcpyAsync(d_evt, sl.h_stage + tb_off + tb_tel, tb_evt, cudaMemcpyHostToDevice, s));
    D_TRY(cudaEventRecord(sl.t_copied, s));
    int rc = rta_image_chain(S->ctx, d_wave, b.n_wave, d_off, d_tel, b.n_img, S->window_mode, S->start, S->W,
                             S->t_hi, S->t_lo, S->core_nb, d_h, s);
    if (rc) return rc;
    if (S->model) {
        rc = rta_surrogate_infer(S->model, d_h, d_tel, b.n_img, d_evt, b.n_evt, S->fallback_deg, d_ev, s);
        if (rc) return rc;
    } else {
        rc = rta_stereo(S->ctx, d_h, d_tel, b.n_img, d_evt, b.n_evt, d_st, s);
        if (rc) return rc;
        D_TRY(rta::launch_stereo_to_events(d_st, b.n_evt, d_ev, s));
    }
    D_TRY(cudaEventRecord(sl.t_computed, s));
    // sky map: the one-second and one-minute slabs of the bundle's arrival
    D_TRY(cudaEventRecord(sl.e_ev, s));
    D_TRY(cudaStreamWaitEvent(S->s_map, sl.e_ev, 0));
    D_TRY(fill_slabs(S, d_ev, b.n_evt, b.arrival_ns));
    D_TRY(cudaEventRecord(sl.e_map, S->s_map));
    D_TRY(cudaStreamWaitEvent(s, sl.e_map, 0));
    D_TRY(cudaMemcpyAsync(sl.h_stage, d_ev, size_t(b.n_evt) * sizeof(rta_event_t), cudaMemcpyDeviceToHost, s));
    D_TRY(cudaEventRecord(sl.t_out, s));
    D_TRY(cudaEventRecord(sl.e_done, s));
#undef D_TRY
    return RTA_OK;
}

void worker_loop(rta_stream* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lock(S->mu);
    while (!S->stop) {
        bool progress = false;
        // completions
        for (auto& sl : S->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.e_done);
            if (q == cudaErrorNotReady) continue;
            Req& r = S->reqs[sl.ticket];
            if (q == cudaSuccess) {     // the event list, from the slot's staging; the bundle's times
                std::memcpy(r.b.h_events, sl.h_stage, size_t(r.b.n_evt) * sizeof(rta_event_t));
                cudaEventElapsedTime(&r.times.h2d_ms, sl.t_in, sl.t_copied);
                cudaEventElapsedTime(&r.times.compute_ms, sl.t_copied, sl.t_computed);
                cudaEventElapsedTime(&r.times.d2h_ms, sl.t_computed, sl.t_out);
            }
            r.done_ns = now_ns();
            r.times.done_ns = r.done_ns;
            r.state = q == cudaSuccess ? REQ_DONE : REQ_FAILED;
            if (q != cudaSuccess) r.rc = RTA_E_CUDA;
            S->arena.release(r.off, r.L.total);
            sl.busy = false;
            --S->running;
            ++S->n_done;
            S->bytes_done += r.b.n_wave * 2;
            progress = true;
        }
        // admissions, in arrival order
        while (!S->pending.empty()) {
            auto fs = std::find_if(S->slots.begin(), S->slots.end(), [](const Slot& x) { return !x.busy; });
            if (fs == S->slots.end()) break;
            Req& r = S->reqs[S->pending.front()];
            size_t off;
            if (!S->arena.alloc(r.L.total, &off)) break;   // wait for memory to free up
            S->pending.pop_front();
            r.off = off;
            r.slot = int(fs - S->slots.begin());
            r.state = REQ_RUNNING;
            fs->busy = true;
            fs->ticket = r.ticket;
            ++S->running;
            const int rc = dispatch(S, r, *fs);
            if (rc) {   // nothing more is enqueued for it; let what was enqueued finish
                cudaStreamSynchronize(fs->s);
                cudaStreamSynchronize(S->s_map);
                S->arena.release(r.off, r.L.total);
                fs->busy = false;
                --S->running;
                r.state = REQ_FAILED;
                r.rc = rc;
                r.done_ns = now_ns();
            }
            progress = true;
        }
        if (progress) S->done_cv.notify_all();
        if (S->running > 0) {
            lock.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lock.lock();
        } else if (!progress) {
            S->cv.wait_for(lock, std::chrono::milliseconds(5));
        }
    }
}

void release_all(rta_stream* S) {
    for (auto& sl : S->slots) {
        if (sl.s) cudaStreamDestroy(sl.s);
        if (sl.h_stage) cudaFreeHost(sl.h_stage);
        cudaEvent_t ev[] = {sl.e_ev, sl.e_map, sl.e_done, sl.t_in, sl.t_copied, sl.t_computed, sl.t_out};
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
    }
    if (S->s_map) cudaStreamDestroy(S->s_map);
    cudaFree(S->arena.base);
    cudaFree(S->d_slabs);
    cudaFree(S->d_slabs_min);
    {
        void* w[] = {S->d_won, S->d_woff, S->d_pre_on, S->d_pre_off, S->d_nal, S->d_hw, S->d_alerts, S->d_sig,
                     S->d_son, S->d_soff};
        for (void* q : w) cudaFree(q);
    }
    cudaFree(S->d_map);
}

}  // namespace

extern "C" {

int rta_stream_create(rta_ctx* ctx, rta_model* model, size_t hbm_budget_bytes, int max_inflight, int64_t max_img,
                      int64_t max_evt, int window_mode, int start, int W, float t_hi, float t_lo,
                      int core_needs_neighbour, float fallback_deg, rta_stream** out) {
    if (!ctx || !out) return vfail(RTA_E_INVALID, "NULL argument");
    if (max_inflight < 1 || max_inflight > 16) return vfail(RTA_E_INVALID, "max_inflight %d outside 1..16", max_inflight);
    if (max_img < 1 || max_evt < 1 || max_img > (int64_t(1) << 30) || max_evt > (int64_t(1) << 30))
        return vfail(RTA_E_INVALID, "bad bundle capacity");
    if (hbm_budget_bytes < (size_t(1) << 20)) return vfail(RTA_E_INVALID, "HBM budget below 1 MiB");
    if (model && !(fallback_deg > 0.f)) return vfail(RTA_E_INVALID, "fallback bound must be > 0");
    int dev = 0;
    int rc = rta::surrogate_ctx_tables(ctx, nullptr, nullptr, nullptr, &dev);
    if (rc) return rc;
    cudaSetDevice(dev);
    rta_stream* S = new rta_stream();
    S->ctx = ctx;
    S->model = model;
    S->device = dev;
    S->window_mode = window_mode;
    S->start = start;
    S->W = W;
    S->core_nb = core_needs_neighbour;
    S->t_hi = t_hi;
    S->t_lo = t_lo;
    S->fallback_deg = fallback_deg;
    S->max_img = max_img;
    S->max_evt = max_evt;
    for (auto& x : S->slab_sec) x = -1;
    for (auto& x : S->slab_min) x = INT64_MIN;
    bool ok = cudaMalloc(&S->arena.base, hbm_budget_bytes) == cudaSuccess &&
              cudaMalloc(&S->d_slabs, sizeof(unsigned int) * RTA_SKY_SLABS * RTA_SKY_N * RTA_SKY_N) == cudaSuccess &&
              cudaMalloc(&S->d_slabs_min, sizeof(unsigned int) * RTA_SKY_MIN_SLABS * RTA_SKY_N * RTA_SKY_N) ==
                  cudaSuccess &&
              cudaMalloc(&S->d_map, sizeof(unsigned int) * RTA_SKY_N * RTA_SKY_N) == cudaSuccess &&
              cudaStreamCreateWithFlags(&S->s_map, cudaStreamNonBlocking) == cudaSuccess;
    S->slots.resize(max_inflight);
    // staging per slot: the tables in, or the event list out, of the largest bundle
    const size_t stage_bytes = std::max(size_t(max_img) * 12 + size_t(max_evt + 1) * 4,
                                        size_t(max_evt) * sizeof(rta_event_t));
    for (auto& sl : S->slots) {
        ok = ok && cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) == cudaSuccess;
        ok = ok && cudaHostAlloc(reinterpret_cast<void**>(&sl.h_stage), stage_bytes, cudaHostAllocDefault) == cudaSuccess;
        cudaEvent_t* ev[] = {&sl.e_ev, &sl.e_map, &sl.e_done};
        for (auto e : ev) ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
        cudaEvent_t* tv[] = {&sl.t_in, &sl.t_copied, &sl.t_computed, &sl.t_out};
        for (auto e : tv) ok = ok && cudaEventCreate(e) == cudaSuccess;
    }
    if (!ok) {
        release_all(S);
        delete S;
        return vfail(RTA_E_NOMEM, "stream resources: allocation failed (budget %zu bytes)", hbm_budget_bytes);
    }
    S->arena.size = hbm_budget_bytes;
    S->arena.reset();
    cudaMemset(S->d_slabs, 0, sizeof(unsigned int) * RTA_SKY_SLABS * RTA_SKY_N * RTA_SKY_N);
    cudaMemset(S->d_slabs_min, 0, sizeof(unsigned int) * RTA_SKY_MIN_SLABS * RTA_SKY_N * RTA_SKY_N);
    cudaDeviceSynchronize();
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return RTA_OK;
}

int rta_stream_submit(rta_stream* S, const rta_bundle_t* b, uint64_t* ticket) {
    if (!S || !b || !ticket) return vfail(RTA_E_INVALID, "NULL argument");
    if (b->n_img < 0 || b->n_evt < 1 || b->n_img > S->max_img || b->n_evt > S->max_evt || b->n_wave < 0)
        return vfail(RTA_E_INVALID, "bundle size outside the stream's capacity");
    if (!b->h_wave || !b->h_wave_off || !b->h_img_tel || !b->h_evt_off || !b->h_events)
        return vfail(RTA_E_INVALID, "NULL host buffer");
    if (b->h_evt_off[0] != 0 || b->h_evt_off[b->n_evt] != b->n_img)
        return vfail(RTA_E_INVALID, "evt_off must run from 0 to n_img");
    Req r;
    r.b = *b;
    r.times.arrival_ns = b->arrival_ns;
    r.times.submit_ns = now_ns();
    r.L = layout_of(*b, S->model == nullptr);
    if (r.L.total > S->arena.size) return vfail(RTA_E_NOMEM, "bundle needs %zu bytes, budget is %zu", r.L.total, S->arena.size);
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->pending.size() >= 4096) return vfail(RTA_E_BUSY, "submission queue full");
    r.ticket = S->next_ticket++;
    *ticket = r.ticket;
    S->reqs.emplace(r.ticket, r);
    S->pending.push_back(r.ticket);
    S->cv.notify_all();
    return RTA_OK;
}

int rta_stream_poll(rta_stream* S, uint64_t ticket, int64_t* done_ns) {
    return rta_stream_poll_times(S, ticket, done_ns, nullptr);
}

int rta_stream_poll_times(rta_stream* S, uint64_t ticket, int64_t* done_ns, rta_bundle_times_t* times) {
    if (!S) return vfail(RTA_E_INVALID, "NULL stream");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return vfail(RTA_E_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    const Req& r = it->second;
    if (r.state == REQ_PENDING || r.state == REQ_RUNNING) return RTA_E_BUSY;
    if (done_ns) *done_ns = r.done_ns;
    if (times) *times = r.times;
    const int rc = r.state == REQ_DONE ? RTA_OK : r.rc;
    S->reqs.erase(it);
    if (rc) return vfail(rc, "bundle %llu failed", (unsigned long long)ticket);
    return RTA_OK;
}

int rta_stream_drain(rta_stream* S, int timeout_ms) {
    if (!S) return vfail(RTA_E_INVALID, "NULL stream");
    std::unique_lock<std::mutex> lock(S->mu);
    const bool ok = S->done_cv.wait_for(lock, std::chrono::milliseconds(timeout_ms),
                                        [S] { return S->pending.empty() && S->running == 0; });
    return ok ? RTA_OK : vfail(RTA_E_TIMEOUT, "drain timed out");
}

int rta_skymap_read(rta_stream* S, int64_t now, uint32_t* h_map) {
    if (!S || !h_map) return vfail(RTA_E_INVALID, "NULL argument");
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lock(S->mu);
    const int64_t sec = now / 1000000000ll;
    unsigned long long use = 0;
    for (int k = 0; k < RTA_SKY_SLABS; ++k)
        if (S->slab_sec[k] > sec - RTA_SKY_SLABS && S->slab_sec[k] <= sec) use |= 1ull << k;
    cudaError_t e = rta::launch_skymap_sum(S->d_slabs, use, S->d_map, S->s_map);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_map, S->d_map, sizeof(uint32_t) * RTA_SKY_N * RTA_SKY_N, cudaMemcpyDeviceToHost, S->s_map);
    lock.unlock();
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->s_map);
    if (e != cudaSuccess) return vfail(RTA_E_CUDA, "sky map read: %s", cudaGetErrorString(e));
    return RTA_OK;
}

int rta_stream_add_events(rta_stream* S, const rta_event_t* d_events, int64_t n_evt, int64_t arrival_ns,
                          void* stream) {
    if (!S || (n_evt > 0 && !d_events) || n_evt < 0) return vfail(RTA_E_INVALID, "bad argument");
    cudaSetDevice(S->device);
    std::lock_guard<std::mutex> lock(S->mu);
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(S->s_map, ev, 0);
    if (e == cudaSuccess) e = fill_slabs(S, d_events, n_evt, arrival_ns);
    // the caller's stream must not reuse d_events before the fill has read it
    if (e == cudaSuccess) e = cudaEventRecord(ev, S->s_map);
    if (e == cudaSuccess) e = cudaStreamWaitEvent((cudaStream_t)stream, ev, 0);
    if (ev) cudaEventDestroy(ev);
    if (e != cudaSuccess) return vfail(RTA_E_CUDA, "sky map fill: %s", cudaGetErrorString(e));
    return RTA_OK;
}

int rta_stream_destroy(rta_stream* S) {
    if (!S) return RTA_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->device);
    cudaDeviceSynchronize();
    release_all(S);
    delete S;
    return RTA_OK;
}

}  // extern "C"

// ======================================================================= transient search
namespace {

bool window_ok(const rta_window_t& w) {
    if (w.on_s < 1 || w.off_s < 1) return false;
    if (int64_t(w.on_s) + w.off_s <= RTA_SKY_SLABS) return true;
    return w.on_s % 60 == 0 && w.off_s % 60 == 0 && int64_t(w.on_s) + w.off_s <= 60 * RTA_SKY_MIN_SLABS;
}

// Half-widths of the rows of the disk x^2 + y^2 <= R^2: hw[dy + R] = largest w
// with w^2 + dy^2 <= R^2.
std::vector<int> disk_half_widths(int R) {
    std::vector<int> hw(size_t(2 * R + 1));
    for (int dy = -R; dy <= R; ++dy) {
        int w = 0;
        while ((w + 1) * (w + 1) + dy * dy <= R * R) ++w;
        hw[size_t(dy + R)] = w;
    }
    return hw;
}

// Ring and slab masks of one window at time now_ns (caller holds S->mu).
void window_masks(const rta_stream* S, int64_t now_ns, const rta_window_t& w, const unsigned int** slabs,
                  int* n_slabs, unsigned long long* use_on, unsigned long long* use_off) {
    const int64_t now_s = now_ns / 1000000000ll;
    *use_on = *use_off = 0;
    if (int64_t(w.on_s) + w.off_s <= RTA_SKY_SLABS) {
        *slabs = S->d_slabs;
        *n_slabs = RTA_SKY_SLABS;
        for (int k = 0; k < RTA_SKY_SLABS; ++k) {
            const int64_t t = S->slab_sec[k];
            if (t > now_s - w.on_s && t <= now_s) *use_on |= 1ull << k;
            if (t > now_s - w.on_s - w.off_s && t <= now_s - w.on_s) *use_off |= 1ull << k;
        }
    } else {
        const int64_t now_m = floor_div(now_s, 60), on = w.on_s / 60, off = w.off_s / 60;
        *slabs = S->d_slabs_min;
        *n_slabs = RTA_SKY_MIN_SLABS;
        for (int k = 0; k < RTA_SKY_MIN_SLABS; ++k) {
            const int64_t t = S->slab_min[k];
            if (t > now_m - on && t <= now_m) *use_on |= 1ull << k;
            if (t > now_m - on - off && t <= now_m - on) *use_off |= 1ull << k;
        }
    }
}

cudaError_t ensure_work(rta_stream* S, size_t alerts_cap, bool maps) {
    const size_t nb = size_t(RTA_SKY_N) * RTA_SKY_N, np = size_t(RTA_SKY_N) * (RTA_SKY_N + 1);
    cudaError_t e = cudaSuccess;
    if (!S->d_won) {
        if ((e = cudaMalloc(&S->d_won, nb * 4)) != cudaSuccess || (e = cudaMalloc(&S->d_woff, nb * 4)) != cudaSuccess ||
            (e = cudaMalloc(&S->d_pre_on, np * 4)) != cudaSuccess ||
            (e = cudaMalloc(&S->d_pre_off, np * 4)) != cudaSuccess ||
            (e = cudaMalloc(&S->d_nal, sizeof(unsigned int))) != cudaSuccess ||
            (e = cudaMalloc(&S->d_hw, sizeof(int) * (2 * RTA_MAX_DISK_RADIUS + 1))) != cudaSuccess)
            return e;
    }
    if (alerts_cap > S->alerts_cap) {
        cudaFree(S->d_alerts);
        S->d_alerts = nullptr;
        S->alerts_cap = 0;
        if ((e = cudaMalloc(&S->d_alerts, sizeof(rta_alert_t) * alerts_cap)) != cudaSuccess) return e;
        S->alerts_cap = alerts_cap;
    }
    if (maps && !S->d_sig) {
        if ((e = cudaMalloc(&S->d_sig, nb * 8)) != cudaSuccess || (e = cudaMalloc(&S->d_son, nb * 8)) != cudaSuccess ||
            (e = cudaMalloc(&S->d_soff, nb * 8)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

// Enqueue the search of one window on the map stream (caller holds S->mu).
cudaError_t enqueue_window(rta_stream* S, int64_t now_ns, const rta_window_t& w, int index, int R, double s_min,
                           bool alerts, bool maps) {
    rta::TransientArgs t = {};
    window_masks(S, now_ns, w, &t.slabs, &t.n_slabs, &t.use_on, &t.use_off);
    t.on = S->d_won;
    t.off = S->d_woff;
    t.pre_on = S->d_pre_on;
    t.pre_off = S->d_pre_off;
    t.hw = S->d_hw;
    t.R = R;
    t.alpha = double(w.on_s) / double(w.off_s);
    t.s_min = s_min;
    t.window = index;
    t.alerts = alerts ? S->d_alerts : nullptr;
    t.n_alerts = S->d_nal;
    t.cap = unsigned(S->alerts_cap);
    t.sig = maps ? S->d_sig : nullptr;
    t.d_on = maps ? S->d_son : nullptr;
    t.d_off = maps ? S->d_soff : nullptr;
    return rta::launch_transient(t, S->s_map);
}

}  // namespace

extern "C" {

int rta_transient_search(rta_stream* S, int64_t now_ns, const rta_window_t* windows, int n_windows, int radius_bins,
                         double s_min, rta_alert_t* h_alerts, int max_alerts, int* n_alerts) {
    if (!S || !n_alerts || n_windows < 0 || (n_windows > 0 && !windows) || max_alerts < 0 ||
        (max_alerts > 0 && !h_alerts))
        return vfail(RTA_E_INVALID, "bad argument");
    if (radius_bins < 0 || radius_bins > RTA_MAX_DISK_RADIUS)
        return vfail(RTA_E_INVALID, "radius %d outside 0..%d", radius_bins, RTA_MAX_DISK_RADIUS);
    for (int i = 0; i < n_windows; ++i)
        if (!window_ok(windows[i]))
            return vfail(RTA_E_INVALID, "window %d (%d s on, %d s off) does not fit the slab rings", i, windows[i].on_s,
                         windows[i].off_s);
    *n_alerts = 0;
    if (n_windows == 0) return RTA_OK;
    cudaSetDevice(S->device);
    const std::vector<int> hw = disk_half_widths(radius_bins);
    unsigned int n_dev = 0;
    std::unique_lock<std::mutex> lock(S->mu);
    cudaError_t e = ensure_work(S, size_t(n_windows) * RTA_SKY_N * RTA_SKY_N, false);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->d_hw, hw.data(), sizeof(int) * hw.size(), cudaMemcpyHostToDevice, S->s_map);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->d_nal, 0, sizeof(unsigned int), S->s_map);
    for (int i = 0; i < n_windows && e == cudaSuccess; ++i)
        e = enqueue_window(S, now_ns, windows[i], i, radius_bins, s_min, true, false);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&n_dev, S->d_nal, sizeof(unsigned int), cudaMemcpyDeviceToHost, S->s_map);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->s_map);
    std::vector<rta_alert_t> all(std::min<size_t>(n_dev, S->alerts_cap));
    if (e == cudaSuccess && !all.empty())
        e = cudaMemcpy(all.data(), S->d_alerts, sizeof(rta_alert_t) * all.size(), cudaMemcpyDeviceToHost);
    lock.unlock();
    if (e != cudaSuccess) return vfail(RTA_E_CUDA, "transient search: %s", cudaGetErrorString(e));
    std::sort(all.begin(), all.end(), [](const rta_alert_t& a, const rta_alert_t& b) {
        if (a.window != b.window) return a.window < b.window;
        if (a.iy != b.iy) return a.iy < b.iy;
        return a.ix < b.ix;
    });
    *n_alerts = int(all.size());
    const size_t n_out = std::min<size_t>(all.size(), size_t(max_alerts));
    if (n_out) memcpy(h_alerts, all.data(), sizeof(rta_alert_t) * n_out);
    return RTA_OK;
}

int rta_significance_map(rta_stream* S, int64_t now_ns, rta_window_t window, int radius_bins, double* h_sig,
                         int64_t* h_on, int64_t* h_off) {
    if (!S || !h_sig) return vfail(RTA_E_INVALID, "bad argument");
    if (radius_bins < 0 || radius_bins > RTA_MAX_DISK_RADIUS)
        return vfail(RTA_E_INVALID, "radius %d outside 0..%d", radius_bins, RTA_MAX_DISK_RADIUS);
    if (!window_ok(window))
        return vfail(RTA_E_INVALID, "window (%d s on, %d s off) does not fit the slab rings", window.on_s, window.off_s);
    cudaSetDevice(S->device);
    const std::vector<int> hw = disk_half_widths(radius_bins);
    const size_t nb = size_t(RTA_SKY_N) * RTA_SKY_N;
    std::unique_lock<std::mutex> lock(S->mu);
    cudaError_t e = ensure_work(S, 0, true);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->d_hw, hw.data(), sizeof(int) * hw.size(), cudaMemcpyHostToDevice, S->s_map);
    if (e == cudaSuccess) e = enqueue_window(S, now_ns, window, 0, radius_bins, 0.0, false, true);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_sig, S->d_sig, nb * 8, cudaMemcpyDeviceToHost, S->s_map);
    if (e == cudaSuccess && h_on) e = cudaMemcpyAsync(h_on, S->d_son, nb * 8, cudaMemcpyDeviceToHost, S->s_map);
    if (e == cudaSuccess && h_off) e = cudaMemcpyAsync(h_off, S->d_soff, nb * 8, cudaMemcpyDeviceToHost, S->s_map);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->s_map);
    lock.unlock();
    if (e != cudaSuccess) return vfail(RTA_E_CUDA, "significance map: %s", cudaGetErrorString(e));
    return RTA_OK;
}

}  // extern "C"
