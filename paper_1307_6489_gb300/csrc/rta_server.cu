// The serving engine: a stream of telescope bundles processed with continuous
// batching under an HBM budget (the RTA processes the event builder's output
// as it arrives, Sec. 4.2, within the 30 s alert latency of Sec. 2.1), with
// the queue of bundles ready for reconstruction held in device memory.
//
// Admission (host): submitted bundles wait in arrival order until one of the
// copy slots is free and the budget arena has room for their waveforms and
// tables; the slot's stream then copies them in and, stream-ordered after the
// copies, a one-thread kernel publishes the bundle's descriptor into a ring in
// device memory (claim an index, write the descriptor, then its ready flag).
//
// Reconstruction (device-resident loop): passes on one compute stream, each
// of which takes at run time, on the device, every bundle published and not yet
// taken (in claim order, up to the batch capacity), gathers their image and
// event tables into one batch (image offsets rebased to the arena, event
// offsets to the batch), runs the fused image kernel and the learned (or the
// geometric) reconstruction once over the whole batch, writes each bundle's
// event rows straight into its slot's mapped host staging, and counts the
// events into the sky-map slabs of their bundles' arrival seconds (slab
// ownership is kept on the device). Bundles that arrive while a pass runs are
// taken by the next one, so copies of new bundles overlap the reconstruction
// of earlier ones and several bundles share one launch of each kernel. The
// host only launches passes while published bundles are outstanding and
// reads, after each pass, which tickets it took.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stddef.h>
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
    size_t wave, wave_off, img_tel, evt_off, total;
};

Layout layout_of(const rta_bundle_t& b) {
    Layout L;
    size_t o = 0;
    L.wave = o; o = up(o + size_t(b.n_wave) * 2);
    L.wave_off = o; o = up(o + size_t(b.n_img) * 8);
    L.img_tel = o; o = up(o + size_t(b.n_img) * 4);
    L.evt_off = o; o = up(o + size_t(b.n_evt + 1) * 4);
    L.total = o;
    return L;
}

// ------------------------------------------------------------------ device-side queue
constexpr int RING = 32;           // published descriptors; never more in flight than copy slots (<= 16)

struct BundleDesc {                // a bundle whose waveforms and tables are in the arena
    unsigned long long ticket;
    int64_t wave_base;             // its waveforms, in samples from the arena base
    const int64_t* wave_off;       // its tables in the arena
    const int32_t* img_tel;
    const int32_t* evt_off;
    int64_t n_img, n_evt, arrival_ns;
    rta_event_t* out;              // device view of its slot's mapped host staging
};
static_assert(sizeof(BundleDesc) % 8 == 0, "copied as 8-byte words");
struct RingSlot {
    BundleDesc d;
    int ready;                     // 1 from publication until taken
    int pad;
};
struct QueueCtl {
    unsigned long long claimed;    // descriptors claimed by publishers
    unsigned long long head;       // descriptors taken by passes
};
struct BatchEntry {                // a bundle in a pass: its descriptor and its first image and event
    BundleDesc d;
    int64_t img_base, evt_base;
};
struct BatchHead {                 // n_img and n_evt first: the kernels read them as device counts
    int64_t n_img, n_evt;
    int n;
    int pad;
    unsigned long long reset_sec, reset_min;   // sky-map slabs the pass's bundles claimed
};
struct SkyOwn {                    // the second (minute) each sky-map slab holds
    int64_t sec[RTA_SKY_SLABS];
    int64_t mnt[RTA_SKY_MIN_SLABS];
};

__host__ __device__ int64_t floor_div(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__host__ __device__ int mod_ring(int64_t a, int n) { return int(((a % n) + n) % n); }

// Publish one bundle (one thread, on its slot's stream after its copies).
__global__ void k_publish(RingSlot* ring, QueueCtl* ctl, BundleDesc d) {
    const unsigned long long i = atomicAdd(&ctl->claimed, 1ull);
    RingSlot* r = ring + (i % RING);
    r->d = d;
    __threadfence();
    atomicExch(&r->ready, 1);
}

// Slab ownership for the bundles batch[0..n), in order: a bundle of a newer
// second (minute) claims its slab, which is then cleared; one of an older one
// leaves it alone and its events are not counted there.
__device__ void claim_slabs(const BatchEntry* batch, int n, SkyOwn* own, BatchHead* head) {
    unsigned long long rs = 0, rm = 0;
    for (int k = 0; k < n; ++k) {
        const int64_t sec = floor_div(batch[k].d.arrival_ns, 1000000000ll), mnt = floor_div(sec, 60);
        const int s = mod_ring(sec, RTA_SKY_SLABS), m = mod_ring(mnt, RTA_SKY_MIN_SLABS);
        if (own->sec[s] < sec) {
            own->sec[s] = sec;
            rs |= 1ull << s;
        }
        if (own->mnt[m] < mnt) {
            own->mnt[m] = mnt;
            rm |= 1ull << m;
        }
    }
    head->reset_sec = rs;
    head->reset_min = rm;
}

// Take, in claim order, the published bundles that fit the batch capacity (the
// first always does: every bundle fits the capacity); one thread.
__global__ void k_take(RingSlot* ring, QueueCtl* ctl, int64_t cap_img, int64_t cap_evt, BatchEntry* batch,
                       BatchHead* head, SkyOwn* own) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned long long h = ctl->head;
    int n = 0;
    int64_t ni = 0, ne = 0;
    while (n < RING) {
        RingSlot* r = ring + ((h + n) % RING);
        if (atomicAdd(&r->ready, 0) == 0) break;      // claimed in order: the next one is not published yet
        __threadfence();
        BundleDesc d;
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&r->d);
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(&d);
        for (int w = 0; w < int(sizeof(BundleDesc) / 8); ++w) dst[w] = __ldcg(src + w);   // past L1: another
                                                                                       // kernel wrote it
        if (n > 0 && (ni + d.n_img > cap_img || ne + d.n_evt > cap_evt)) break;
        batch[n].d = d;
        batch[n].img_base = ni;
        batch[n].evt_base = ne;
        ni += d.n_img;
        ne += d.n_evt;
        atomicExch(&r->ready, 0);
        ++n;
    }
    ctl->head = h + n;
    head->n = n;
    head->n_img = ni;
    head->n_evt = ne;
    claim_slabs(batch, n, own, head);
}

// Slab ownership of one list of events with one arrival time (events added from
// outside the loop); one thread.
__global__ void k_claim_one(BatchEntry e, BatchEntry* batch, BatchHead* head, SkyOwn* own) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    batch[0] = e;
    head->n = 1;
    head->n_img = 0;
    head->n_evt = e.d.n_evt;
    claim_slabs(batch, 1, own, head);
}

// Clear the slabs the pass claimed: blockIdx.y = slab (the one-second ring, then
// the one-minute ring), blockIdx.x = a 4096-word chunk of it.
__global__ void k_slab_reset(const BatchHead* head, unsigned int* slabs, unsigned int* slabs_min) {
    const int k = blockIdx.y;
    const bool sec = k < RTA_SKY_SLABS;
    const unsigned long long mask = sec ? head->reset_sec : head->reset_min;
    const int s = sec ? k : k - RTA_SKY_SLABS;
    if (!((mask >> s) & 1ull)) return;
    unsigned int* p = (sec ? slabs : slabs_min) + size_t(s) * RTA_SKY_N * RTA_SKY_N + size_t(blockIdx.x) * 4096;
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) p[i] = 0u;
}

// The pass's bundle holding item i, items counted by img_base or evt_base.
__device__ __forceinline__ int bundle_of(const BatchEntry* batch, int n, int64_t i, bool by_event) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((by_event ? batch[mid].evt_base : batch[mid].img_base) <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The batch's tables: image offsets rebased to the arena, telescopes, event
// offsets rebased to the batch (an offset outside its bundle becomes -1, which
// the kernels report as malformed).
__global__ void k_gather(const BatchEntry* batch, const BatchHead* head, int64_t* off_m, int32_t* tel_m,
                         int32_t* evt_m) {
    const int n = head->n;
    const int64_t ni = head->n_img, ne = head->n_evt;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < ni; i += stride) {
        const BatchEntry& b = batch[bundle_of(batch, n, i, false)];
        const int64_t k = i - b.img_base;
        off_m[i] = b.d.wave_base + b.d.wave_off[k];
        tel_m[i] = b.d.img_tel[k];
    }
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e <= ne; e += stride) {
        if (e == ne) {
            evt_m[e] = int32_t(ni);
            continue;
        }
        const BatchEntry& b = batch[bundle_of(batch, n, e, true)];
        const int32_t v = b.d.evt_off[e - b.evt_base];
        evt_m[e] = (v < 0 || v > b.d.n_img) ? -1 : int32_t(b.img_base + v);
    }
}

// Each bundle's event rows into its slot's mapped host staging (geometric mode:
// formed from the stereo rows first, and kept in ev for the sky map too).
__global__ void k_batch_out(rta_event_t* ev, const rta_stereo_t* st, const BatchEntry* batch, const BatchHead* head) {
    const int n = head->n;
    const int64_t ne = head->n_evt;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < ne; e += int64_t(gridDim.x) * blockDim.x) {
        rta_event_t r;
        if (st) {
            r = rta::stereo_event_row(st[e]);
            ev[e] = r;
        } else {
            r = ev[e];
        }
        const BatchEntry& b = batch[bundle_of(batch, n, e, true)];
        b.d.out[e - b.evt_base] = r;
    }
}

// Sky-map counts of the batch's events, each in the slabs of its bundle's
// arrival second and minute when the slab still holds them.
__global__ void k_sky_fill(const rta_event_t* ev, const BatchEntry* batch, const BatchHead* head, const SkyOwn* own,
                           unsigned int* slabs, unsigned int* slabs_min) {
    const int n = head->n;
    const int64_t ne = head->n_evt;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < ne; e += int64_t(gridDim.x) * blockDim.x) {
        const rta_event_t r = ev[e];
        if (r.flags & RTA_EF_NO_DIRECTION) continue;
        const int ix = rta::sky_bin(r.dir_x), iy = rta::sky_bin(r.dir_y);
        if (ix < 0 || iy < 0) continue;
        const BatchEntry& b = batch[bundle_of(batch, n, e, true)];
        const int64_t sec = floor_div(b.d.arrival_ns, 1000000000ll), mnt = floor_div(sec, 60);
        const int s = mod_ring(sec, RTA_SKY_SLABS), m = mod_ring(mnt, RTA_SKY_MIN_SLABS);
        const size_t bin = size_t(iy) * RTA_SKY_N + ix;
        if (own->sec[s] == sec) atomicAdd(slabs + size_t(s) * RTA_SKY_N * RTA_SKY_N + bin, 1u);
        if (own->mnt[m] == mnt) atomicAdd(slabs_min + size_t(m) * RTA_SKY_N * RTA_SKY_N + bin, 1u);
    }
}

enum { REQ_PENDING = 0, REQ_COPYING = 1, REQ_PUBLISHED = 2, REQ_DONE = 3, REQ_FAILED = 4 };

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

struct Slot {                      // a copy slot: its stream, staging and the bundle it carries
    cudaStream_t s = nullptr;
    cudaEvent_t e_pub = nullptr;   // the bundle is published
    cudaEvent_t t_in = nullptr, t_copied = nullptr;   // timing
    uint64_t ticket = 0;
    bool busy = false;
    // pinned, mapped staging: the bundle's tables on the way in (copies from pageable
    // memory would block the scheduler thread until the slot's stream reached them),
    // its event rows, written by the device, on the way out
    char* h_stage = nullptr;
    rta_event_t* d_stage = nullptr;   // device view of h_stage
};

struct Pass {                      // a reconstruction pass in flight on the compute stream
    cudaEvent_t t_begin = nullptr, t_computed = nullptr, t_end = nullptr;
    char* h_tab = nullptr;         // pinned: the pass's BatchHead and BatchEntry table, copied back
};

}  // namespace

struct rta_stream {
    rta_ctx* ctx = nullptr;
    rta_model* model = nullptr;
    int device = 0;
    int window_mode = 0, start = 0, W = 0, core_nb = 0;
    float t_hi = 0.f, t_lo = 0.f, fallback_deg = 0.5f;
    int64_t max_img = 0, max_evt = 0, cap_img = 0, cap_evt = 0;
    Arena arena;
    std::vector<Slot> slots;
    cudaStream_t s_cmp = nullptr;  // the reconstruction passes, the sky map and its searches
    // device-side queue and the batch of the current pass
    RingSlot* d_ring = nullptr;
    QueueCtl* d_ctl = nullptr;
    BatchEntry* d_batch = nullptr;
    BatchHead* d_head = nullptr;
    int64_t* d_off_m = nullptr;
    int32_t* d_tel_m = nullptr;
    int32_t* d_evt_m = nullptr;
    rta_hillas_t* d_hil = nullptr;
    rta_event_t* d_ev = nullptr;
    rta_stereo_t* d_st = nullptr;
    std::vector<Pass> pass_pool;
    std::deque<int> passes;        // passes in flight, oldest first (indices into pass_pool)
    bool need_pass = false;
    // sky map
    SkyOwn* d_own = nullptr;
    SkyOwn own{};                  // host copy, read before a map or a search is formed
    unsigned int* d_slabs = nullptr;       // RTA_SKY_SLABS x 256 x 256
    unsigned int* d_slabs_min = nullptr;   // RTA_SKY_MIN_SLABS x 256 x 256
    unsigned int* d_map = nullptr;
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

constexpr size_t TAB_BYTES = sizeof(BatchHead) + sizeof(BatchEntry) * RING;

// The slabs' owners on the host, after every pass enqueued so far (caller holds S->mu).
cudaError_t read_own(rta_stream* S) {
    cudaError_t e = cudaMemcpyAsync(&S->own, S->d_own, sizeof(SkyOwn), cudaMemcpyDeviceToHost, S->s_cmp);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->s_cmp);
    return e;
}

#define D_TRY(call)                                                                                 \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return vfail(RTA_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

// Admit one bundle: copies in on the slot's stream, then its publication (*pub: its
// publication may be on the stream, so a failure after it must empty the device queue).
int dispatch(rta_stream* S, Req& r, Slot& sl, bool* pub) {
    *pub = false;
    const rta_bundle_t& b = r.b;
    char* base = S->arena.base + r.off;
    uint16_t* d_wave = reinterpret_cast<uint16_t*>(base + r.L.wave);
    int64_t* d_off = reinterpret_cast<int64_t*>(base + r.L.wave_off);
    int32_t* d_tel = reinterpret_cast<int32_t*>(base + r.L.img_tel);
    int32_t* d_evt = reinterpret_cast<int32_t*>(base + r.L.evt_off);
    cudaStream_t s = sl.s;
    r.times.admit_ns = now_ns();
    r.times.slot = int(&sl - &S->slots[0]);
    // the tables through the slot's pinned staging (free: its previous bundle is done)
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
    BundleDesc d = {};
    d.ticket = r.ticket;
    d.wave_base = int64_t((r.off + r.L.wave) / 2);
    d.wave_off = d_off;
    d.img_tel = d_tel;
    d.evt_off = d_evt;
    d.n_img = b.n_img;
    d.n_evt = b.n_evt;
    d.arrival_ns = b.arrival_ns;
    d.out = sl.d_stage;
    *pub = true;
    k_publish<<<1, 1, 0, s>>>(S->d_ring, S->d_ctl, d);
    D_TRY(cudaGetLastError());
    D_TRY(cudaEventRecord(sl.e_pub, s));
    return RTA_OK;
}

// One reconstruction pass on the compute stream over whatever is published when it runs.
int launch_pass(rta_stream* S, Pass& p) {
    cudaStream_t s = S->s_cmp;
    D_TRY(cudaEventRecord(p.t_begin, s));
    k_take<<<1, 32, 0, s>>>(S->d_ring, S->d_ctl, S->cap_img, S->cap_evt, S->d_batch, S->d_head, S->d_own);
    D_TRY(cudaGetLastError());
    k_slab_reset<<<dim3(RTA_SKY_N * RTA_SKY_N / 4096, RTA_SKY_SLABS + RTA_SKY_MIN_SLABS), 256, 0, s>>>(
        S->d_head, S->d_slabs, S->d_slabs_min);
    D_TRY(cudaGetLastError());
    const int g_img = int(std::min<int64_t>((S->cap_img + 255) / 256, 2048));
    k_gather<<<g_img, 256, 0, s>>>(S->d_batch, S->d_head, S->d_off_m, S->d_tel_m, S->d_evt_m);
    D_TRY(cudaGetLastError());
    const int64_t* d_ni = reinterpret_cast<const int64_t*>(reinterpret_cast<const char*>(S->d_head) +
                                                          offsetof(BatchHead, n_img));
    const int64_t* d_ne = reinterpret_cast<const int64_t*>(reinterpret_cast<const char*>(S->d_head) +
                                                          offsetof(BatchHead, n_evt));
    int rc = rta::serve_image_chain(S->ctx, reinterpret_cast<const uint16_t*>(S->arena.base),
                                    int64_t(S->arena.size / 2), S->d_off_m, S->d_tel_m, d_ni, S->cap_img,
                                    S->window_mode, S->start, S->W, S->t_hi, S->t_lo, S->core_nb, S->d_hil, s);
    if (rc) return rc;
    if (S->model)
        rc = rta::serve_infer(S->model, S->d_hil, S->d_tel_m, S->cap_img, S->d_evt_m, S->cap_evt, d_ni, d_ne,
                              S->fallback_deg, S->d_ev, s);
    else
        rc = rta::serve_stereo(S->ctx, S->d_hil, S->d_tel_m, S->cap_img, S->d_evt_m, S->cap_evt, d_ni, d_ne, S->d_st, s);
    if (rc) return rc;
    D_TRY(cudaEventRecord(p.t_computed, s));
    const int g_evt = int(std::min<int64_t>((S->cap_evt + 255) / 256, 2048));
    k_batch_out<<<g_evt, 256, 0, s>>>(S->d_ev, S->model ? nullptr : S->d_st, S->d_batch, S->d_head);
    D_TRY(cudaGetLastError());
    k_sky_fill<<<g_evt, 256, 0, s>>>(S->d_ev, S->d_batch, S->d_head, S->d_own, S->d_slabs, S->d_slabs_min);
    D_TRY(cudaGetLastError());
    D_TRY(cudaMemcpyAsync(p.h_tab, S->d_head, sizeof(BatchHead), cudaMemcpyDeviceToHost, s));
    D_TRY(cudaMemcpyAsync(p.h_tab + sizeof(BatchHead), S->d_batch, sizeof(BatchEntry) * RING, cudaMemcpyDeviceToHost, s));
    D_TRY(cudaEventRecord(p.t_end, s));
    return RTA_OK;
}

// A pass has completed: every bundle it took is done (caller holds S->mu).
void finish_pass(rta_stream* S, Pass& p) {
    const BatchHead* hd = reinterpret_cast<const BatchHead*>(p.h_tab);
    const BatchEntry* tab = reinterpret_cast<const BatchEntry*>(p.h_tab + sizeof(BatchHead));
    float dev_ms = 0.f, out_ms = 0.f;
    cudaEventElapsedTime(&dev_ms, p.t_begin, p.t_computed);
    cudaEventElapsedTime(&out_ms, p.t_computed, p.t_end);
    const int64_t t_done = now_ns();
    for (int k = 0; k < hd->n && k < RING; ++k) {
        auto it = S->reqs.find(tab[k].d.ticket);
        if (it == S->reqs.end()) continue;
        Req& r = it->second;
        if (r.state != REQ_COPYING && r.state != REQ_PUBLISHED) continue;   // failed meanwhile: released
        Slot& sl = S->slots[r.slot];
        // the event rows, written into the slot's staging by the pass
        std::memcpy(r.b.h_events, sl.h_stage, size_t(r.b.n_evt) * sizeof(rta_event_t));
        cudaEventElapsedTime(&r.times.h2d_ms, sl.t_in, sl.t_copied);
        float wait_ms = 0.f;
        cudaEventElapsedTime(&wait_ms, sl.t_copied, p.t_begin);
        r.times.ready_wait_ms = std::max(0.f, wait_ms);
        r.times.compute_ms = dev_ms;
        r.times.d2h_ms = out_ms;
        r.times.batch_bundles = hd->n;
        r.done_ns = t_done;
        r.times.done_ns = t_done;
        r.state = REQ_DONE;
        S->arena.release(r.off, r.L.total);
        sl.busy = false;
        --S->running;
        ++S->n_done;
        S->bytes_done += r.b.n_wave * 2;
    }
}

// Every admitted bundle fails (a pass or a publication could not be enqueued, or a
// CUDA call failed; caller holds S->mu). Once nothing of the stream's is in flight, the
// passes still listed (their bundles are among the failed) are dropped and the device
// queue is emptied, so that no later pass takes a descriptor of a released bundle.
void fail_admitted(rta_stream* S, int rc) {
    cudaStreamSynchronize(S->s_cmp);
    for (auto& sl : S->slots)
        if (sl.s) cudaStreamSynchronize(sl.s);
    for (auto& sl : S->slots) {
        if (!sl.busy) continue;
        Req& r = S->reqs[sl.ticket];
        S->arena.release(r.off, r.L.total);
        sl.busy = false;
        --S->running;
        r.state = REQ_FAILED;
        r.rc = rc;
        r.done_ns = now_ns();
    }
    S->passes.clear();
    S->need_pass = false;
    if (cudaMemsetAsync(S->d_ring, 0, sizeof(RingSlot) * RING, S->s_cmp) == cudaSuccess &&
        cudaMemsetAsync(S->d_ctl, 0, sizeof(QueueCtl), S->s_cmp) == cudaSuccess)
        cudaStreamSynchronize(S->s_cmp);
}

void worker_loop(rta_stream* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lock(S->mu);
    while (!S->stop) {
        bool progress = false;
        // bundles whose publication has run: a pass must take them
        for (auto& sl : S->slots) {
            if (!sl.busy) continue;
            Req& r = S->reqs[sl.ticket];
            if (r.state != REQ_COPYING) continue;
            const cudaError_t q = cudaEventQuery(sl.e_pub);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                fail_admitted(S, RTA_E_CUDA);
                progress = true;
                break;
            }
            r.state = REQ_PUBLISHED;
            S->need_pass = true;
        }
        // completed passes, oldest first
        while (!S->passes.empty()) {
            Pass& p = S->pass_pool[S->passes.front()];
            const cudaError_t q = cudaEventQuery(p.t_end);
            if (q == cudaErrorNotReady) break;
            S->passes.pop_front();
            if (q != cudaSuccess) {
                fail_admitted(S, RTA_E_CUDA);
            } else {
                finish_pass(S, p);
            }
            // bundles published but not taken (batch capacity) need another pass
            for (auto& sl : S->slots)
                if (sl.busy && S->reqs[sl.ticket].state == REQ_PUBLISHED) S->need_pass = true;
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
            r.state = REQ_COPYING;
            fs->busy = true;
            fs->ticket = r.ticket;
            ++S->running;
            bool pub = false;
            const int rc = dispatch(S, r, *fs, &pub);
            if (rc && pub) {
                fail_admitted(S, rc);        // its descriptor may be in the device queue
            } else if (rc) {   // nothing more is enqueued for it; let what was enqueued finish
                cudaStreamSynchronize(fs->s);
                S->arena.release(r.off, r.L.total);
                fs->busy = false;
                --S->running;
                r.state = REQ_FAILED;
                r.rc = rc;
                r.done_ns = now_ns();
            }
            progress = true;
        }
        // a pass over what is published, at most two queued on the compute stream
        if (S->need_pass && S->passes.size() < 2) {
            int idx = -1;
            for (int k = 0; k < int(S->pass_pool.size()); ++k)
                if (std::find(S->passes.begin(), S->passes.end(), k) == S->passes.end()) idx = k;
            const int rc = launch_pass(S, S->pass_pool[idx]);
            if (rc) {
                fail_admitted(S, rc);
            } else {
                S->passes.push_back(idx);
                S->need_pass = false;
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
        cudaEvent_t ev[] = {sl.e_pub, sl.t_in, sl.t_copied};
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
    }
    for (auto& p : S->pass_pool) {
        cudaEvent_t ev[] = {p.t_begin, p.t_computed, p.t_end};
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
        if (p.h_tab) cudaFreeHost(p.h_tab);
    }
    if (S->s_cmp) cudaStreamDestroy(S->s_cmp);
    void* d[] = {S->arena.base, S->d_ring, S->d_ctl, S->d_batch, S->d_head, S->d_off_m, S->d_tel_m, S->d_evt_m,
                 S->d_hil, S->d_ev, S->d_st, S->d_own, S->d_slabs, S->d_slabs_min, S->d_map, S->d_won, S->d_woff,
                 S->d_pre_on, S->d_pre_off, S->d_nal, S->d_hw, S->d_alerts, S->d_sig, S->d_son, S->d_soff};
    for (void* q : d) cudaFree(q);
}

#undef D_TRY

}  // namespace

extern "C" {

int rta_stream_create(rta_ctx* ctx, rta_model* model, size_t hbm_budget_bytes, int max_inflight, int64_t max_img,
                      int64_t max_evt, int window_mode, int start, int W, float t_hi, float t_lo,
                      int core_needs_neighbour, float fallback_deg, rta_stream** out) {
    if (!ctx || !out) return vfail(RTA_E_INVALID, "NULL argument");
    if (max_inflight < 1 || max_inflight > 16) return vfail(RTA_E_INVALID, "max_inflight %d outside 1..16", max_inflight);
    if (max_img < 1 || max_evt < 1 || max_img > (int64_t(1) << 29) || max_evt > (int64_t(1) << 29))
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
    // a pass takes up to two of the largest bundles (and any number of smaller ones up to that)
    S->cap_img = 2 * max_img;
    S->cap_evt = 2 * max_evt;
    for (auto& x : S->own.sec) x = -1;
    for (auto& x : S->own.mnt) x = INT64_MIN;
    const size_t slab_bytes = sizeof(unsigned int) * RTA_SKY_N * RTA_SKY_N;
    bool ok = cudaMalloc(&S->arena.base, hbm_budget_bytes) == cudaSuccess &&
              cudaMalloc(&S->d_slabs, slab_bytes * RTA_SKY_SLABS) == cudaSuccess &&
              cudaMalloc(&S->d_slabs_min, slab_bytes * RTA_SKY_MIN_SLABS) == cudaSuccess &&
              cudaMalloc(&S->d_map, slab_bytes) == cudaSuccess &&
              cudaMalloc(&S->d_ring, sizeof(RingSlot) * RING) == cudaSuccess &&
              cudaMalloc(&S->d_ctl, sizeof(QueueCtl)) == cudaSuccess &&
              cudaMalloc(&S->d_batch, sizeof(BatchEntry) * RING) == cudaSuccess &&
              cudaMalloc(&S->d_head, sizeof(BatchHead)) == cudaSuccess &&
              cudaMalloc(&S->d_own, sizeof(SkyOwn)) == cudaSuccess &&
              cudaMalloc(&S->d_off_m, sizeof(int64_t) * S->cap_img) == cudaSuccess &&
              cudaMalloc(&S->d_tel_m, sizeof(int32_t) * S->cap_img) == cudaSuccess &&
              cudaMalloc(&S->d_evt_m, sizeof(int32_t) * (S->cap_evt + 1)) == cudaSuccess &&
              cudaMalloc(&S->d_hil, sizeof(rta_hillas_t) * S->cap_img) == cudaSuccess &&
              cudaMalloc(&S->d_ev, sizeof(rta_event_t) * S->cap_evt) == cudaSuccess &&
              (model || cudaMalloc(&S->d_st, sizeof(rta_stereo_t) * S->cap_evt) == cudaSuccess) &&
              cudaStreamCreateWithFlags(&S->s_cmp, cudaStreamNonBlocking) == cudaSuccess;
    S->slots.resize(max_inflight);
    // staging per slot: the tables in, or the event list out, of the largest bundle
    const size_t stage_bytes = std::max(size_t(max_img) * 12 + size_t(max_evt + 1) * 4,
                                        size_t(max_evt) * sizeof(rta_event_t));
    for (auto& sl : S->slots) {
        ok = ok && cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) == cudaSuccess;
        ok = ok && cudaHostAlloc(reinterpret_cast<void**>(&sl.h_stage), stage_bytes, cudaHostAllocMapped) == cudaSuccess;
        ok = ok && cudaHostGetDevicePointer(reinterpret_cast<void**>(&sl.d_stage), sl.h_stage, 0) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&sl.e_pub, cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaEventCreate(&sl.t_in) == cudaSuccess && cudaEventCreate(&sl.t_copied) == cudaSuccess;
    }
    S->pass_pool.resize(2);
    for (auto& p : S->pass_pool) {
        ok = ok && cudaEventCreate(&p.t_begin) == cudaSuccess && cudaEventCreate(&p.t_computed) == cudaSuccess &&
             cudaEventCreate(&p.t_end) == cudaSuccess;
        ok = ok && cudaHostAlloc(reinterpret_cast<void**>(&p.h_tab), TAB_BYTES, cudaHostAllocDefault) == cudaSuccess;
    }
    if (!ok) {
        release_all(S);
        delete S;
        return vfail(RTA_E_NOMEM, "stream resources: allocation failed (budget %zu bytes)", hbm_budget_bytes);
    }
    S->arena.size = hbm_budget_bytes;
    S->arena.reset();
    bool zok = cudaMemset(S->d_slabs, 0, slab_bytes * RTA_SKY_SLABS) == cudaSuccess &&
               cudaMemset(S->d_slabs_min, 0, slab_bytes * RTA_SKY_MIN_SLABS) == cudaSuccess &&
               cudaMemset(S->d_ring, 0, sizeof(RingSlot) * RING) == cudaSuccess &&
               cudaMemset(S->d_ctl, 0, sizeof(QueueCtl)) == cudaSuccess &&
               cudaMemset(S->d_head, 0, sizeof(BatchHead)) == cudaSuccess &&
               cudaMemcpy(S->d_own, &S->own, sizeof(SkyOwn), cudaMemcpyHostToDevice) == cudaSuccess &&
               cudaDeviceSynchronize() == cudaSuccess;
    if (!zok) {
        release_all(S);
        delete S;
        return vfail(RTA_E_CUDA, "stream set-up failed");
    }
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
    // every image inside the bundle's own waveforms: in the batch the image kernel
    // addresses the whole arena
    int rc = rta::check_bundle_images(S->ctx, b->h_wave_off, b->h_img_tel, b->n_img, b->n_wave);
    if (rc) return rc;
    Req r;
    r.b = *b;
    r.times.arrival_ns = b->arrival_ns;
    r.times.submit_ns = now_ns();
    r.L = layout_of(*b);
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
    if (r.state != REQ_DONE && r.state != REQ_FAILED) return RTA_E_BUSY;
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
    cudaError_t e = read_own(S);
    const int64_t sec = now / 1000000000ll;
    unsigned long long use = 0;
    for (int k = 0; k < RTA_SKY_SLABS; ++k)
        if (S->own.sec[k] > sec - RTA_SKY_SLABS && S->own.sec[k] <= sec) use |= 1ull << k;
    if (e == cudaSuccess) e = rta::launch_skymap_sum(S->d_slabs, use, S->d_map, S->s_cmp);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_map, S->d_map, sizeof(uint32_t) * RTA_SKY_N * RTA_SKY_N, cudaMemcpyDeviceToHost, S->s_cmp);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->s_cmp);
    lock.unlock();
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
    if (e == cudaSuccess) e = cudaStreamWaitEvent(S->s_cmp, ev, 0);
    if (e == cudaSuccess) {
        BatchEntry be = {};
        be.d.n_evt = n_evt;
        be.d.arrival_ns = arrival_ns;
        k_claim_one<<<1, 1, 0, S->s_cmp>>>(be, S->d_batch, S->d_head, S->d_own);
        k_slab_reset<<<dim3(RTA_SKY_N * RTA_SKY_N / 4096, RTA_SKY_SLABS + RTA_SKY_MIN_SLABS), 256, 0, S->s_cmp>>>(
            S->d_head, S->d_slabs, S->d_slabs_min);
        if (n_evt > 0)
            k_sky_fill<<<int(std::min<int64_t>((n_evt + 255) / 256, 2048)), 256, 0, S->s_cmp>>>(
                d_events, S->d_batch, S->d_head, S->d_own, S->d_slabs, S->d_slabs_min);
        e = cudaGetLastError();
    }
    // the caller's stream must not reuse d_events before the fill has read it
    if (e == cudaSuccess) e = cudaEventRecord(ev, S->s_cmp);
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
            const int64_t t = S->own.sec[k];
            if (t > now_s - w.on_s && t <= now_s) *use_on |= 1ull << k;
            if (t > now_s - w.on_s - w.off_s && t <= now_s - w.on_s) *use_off |= 1ull << k;
        }
    } else {
        const int64_t now_m = floor_div(now_s, 60), on = w.on_s / 60, off = w.off_s / 60;
        *slabs = S->d_slabs_min;
        *n_slabs = RTA_SKY_MIN_SLABS;
        for (int k = 0; k < RTA_SKY_MIN_SLABS; ++k) {
            const int64_t t = S->own.mnt[k];
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
    return rta::launch_transient(t, S->s_cmp);
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
    cudaError_t e = read_own(S);
    if (e == cudaSuccess) e = ensure_work(S, size_t(n_windows) * RTA_SKY_N * RTA_SKY_N, false);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->d_hw, hw.data(), sizeof(int) * hw.size(), cudaMemcpyHostToDevice, S->s_cmp);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->d_nal, 0, sizeof(unsigned int), S->s_cmp);
    for (int i = 0; i < n_windows && e == cudaSuccess; ++i)
        e = enqueue_window(S, now_ns, windows[i], i, radius_bins, s_min, true, false);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&n_dev, S->d_nal, sizeof(unsigned int), cudaMemcpyDeviceToHost, S->s_cmp);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->s_cmp);
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
    cudaError_t e = read_own(S);
    if (e == cudaSuccess) e = ensure_work(S, 0, true);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->d_hw, hw.data(), sizeof(int) * hw.size(), cudaMemcpyHostToDevice, S->s_cmp);
    if (e == cudaSuccess) e = enqueue_window(S, now_ns, window, 0, radius_bins, 0.0, false, true);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_sig, S->d_sig, nb * 8, cudaMemcpyDeviceToHost, S->s_cmp);
    if (e == cudaSuccess && h_on) e = cudaMemcpyAsync(h_on, S->d_son, nb * 8, cudaMemcpyDeviceToHost, S->s_cmp);
    if (e == cudaSuccess && h_off) e = cudaMemcpyAsync(h_off, S->d_soff, nb * 8, cudaMemcpyDeviceToHost, S->s_cmp);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->s_cmp);
    lock.unlock();
    if (e != cudaSuccess) return vfail(RTA_E_CUDA, "significance map: %s", cudaGetErrorString(e));
    return RTA_OK;
}

}  // extern "C"
