// Host side of librta: the C ABI declared in include/rta.h. Argument checks,
// the context (registered cameras, array, calibration table, device status
// word, work counters), launch configuration and its autotuner, and the
// host-buffer path with double-buffered staging.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "rta.h"
#include "rta_launch.cuh"

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

#define CUDA_TRY(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(RTA_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

constexpr int N_COUNTERS = 1024;

struct HostCam {
    bool valid = false;
    int P = 0, S = 0, K = 0;
    float2* d_xy = nullptr;
    int4* d_nb = nullptr;
};

struct Slot {  // one half of the host-path double buffer
    cudaStream_t stream = nullptr;
    cudaEvent_t meta_done = nullptr;
    uint16_t* d_wave = nullptr;
    size_t wave_cap = 0;
    int64_t* d_off = nullptr;
    int32_t* d_tel = nullptr;
    int32_t* d_evt = nullptr;
    rta_hillas_t* d_h = nullptr;
    rta_stereo_t* d_s = nullptr;
    size_t img_cap = 0, evt_cap = 0;
    int64_t* h_off = nullptr;   // pinned
    int32_t* h_tel = nullptr;   // pinned (a copy from the caller's pageable table would block the enqueueing thread)
    int32_t* h_evt = nullptr;   // pinned
    // results of the slot's last chunk, staged in pinned memory so that the
    // device-to-host copies never block the thread that enqueues the next upload
    rta_hillas_t* h_hres = nullptr;
    rta_stereo_t* h_sres = nullptr;
    cudaEvent_t res_done = nullptr;
    cudaEvent_t up_done = nullptr;     // this slot's last upload has landed
    bool res_pending = false;
    int64_t res_i0 = 0, res_ni = 0, res_e0 = 0, res_ne = 0;
};

}  // namespace

void rta::set_last_error(const char* msg) {
    snprintf(g_err, sizeof g_err, "%s", msg);
}

struct rta_ctx {
    int device = 0;
    int n_sm = 0;
    size_t budget = 0;
    size_t staged_bytes = 0;
    HostCam cams[RTA_MAX_CAMS];
    rta::DevCam* d_cams = nullptr;
    int n_tel = 0;
    std::vector<int32_t> tel_cam;
    int32_t* d_tel_cam = nullptr;
    float2* d_tel_xy = nullptr;
    int64_t* d_tel_row = nullptr;
    int32_t* d_p16 = nullptr;
    float* d_scale = nullptr;
    unsigned int* d_status = nullptr;
    unsigned int* d_counters = nullptr;
    std::atomic<unsigned> next_counter{0};
    // launch configuration of the fused image kernel
    int filter_n = 0;     // digital-filter weights (RTA_WINDOW_FILTER), 0 = none
    int filter_w[RTA_MAX_W] = {};
    int variant = 4;      // tile shape, see chain_variant_* (the fastest on GB300 for the array cameras)
    int nstage = 2;
    int ctas_per_sm = 0;  // 0 = the variant's target, shrinking the stages to fit, else as many as fit
    // the neighbour-peak kernel's own configuration (more shared memory per CTA,
    // a per-image barrier: its fastest shape differs)
    int nb_variant = 0;
    int nb_nstage = 3;
    int nb_ctas_per_sm = 0;
    // the byte-stream kernel's configuration once rta_autotune_stream has tuned it
    // (st_variant < 0: the plain kernel's)
    int st_variant = -1;
    int st_nstage = 2;
    int st_ctas_per_sm = 0;
    int max_P = 0, max_S = 0;
    Slot slot[2];
    // workspace of rta_ingest (pieces, packet list), grown on demand
    void* d_ingest = nullptr;
    size_t ingest_bytes = 0;
    // per-image records of rta_reconstruct_stream, grown on demand
    void* d_smeta = nullptr;
    size_t smeta_bytes = 0;
    std::mutex host_mu;
};

namespace {

int check_ctx(rta_ctx* c) {
    if (!c) return fail(RTA_E_INVALID, "context is NULL");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(RTA_E_CUDA, "cudaSetDevice(%d) failed", c->device);
    return RTA_OK;
}

int check_array(rta_ctx* c) {
    if (c->n_tel <= 0) return fail(RTA_E_INVALID, "no array registered (rta_register_array)");
    return RTA_OK;
}

// Work counters for device-resident calls: a ring, so that calls in flight on
// different streams use different counters. The last two belong to the
// host-buffer path.
unsigned int* take_counter(rta_ctx* c) {
    unsigned i = c->next_counter.fetch_add(1) % (N_COUNTERS - 2);
    return c->d_counters + i;
}

// Upload the device camera table; the largest P and S size the kernel's buffers.
int refresh_cams(rta_ctx* c) {
    int maxS = 1, maxP = 1;
    for (auto& h : c->cams)
        if (h.valid) { maxS = std::max(maxS, h.S); maxP = std::max(maxP, h.P); }
    c->max_P = maxP;
    c->max_S = maxS;
    rta::DevCam dc[RTA_MAX_CAMS];
    memset(dc, 0, sizeof dc);
    for (int i = 0; i < RTA_MAX_CAMS; ++i) {
        const HostCam& h = c->cams[i];
        if (!h.valid) continue;
        dc[i].P = h.P;
        dc[i].S = h.S;
        dc[i].K = h.K;
        dc[i].xy = h.d_xy;
        dc[i].nb = h.d_nb;
    }
    CUDA_TRY(cudaMemcpy(c->d_cams, dc, sizeof dc, cudaMemcpyHostToDevice));
    return RTA_OK;
}

rta::DevArray dev_array(rta_ctx* c) {
    rta::DevArray a;
    a.cams = c->d_cams;
    a.tel_cam = c->d_tel_cam;
    a.tel_xy = c->d_tel_xy;
    a.tel_row = c->d_tel_row;
    a.p16 = c->d_p16;
    a.scale = c->d_scale;
    a.n_tel = c->n_tel;
    a.max_P = c->max_P;
    return a;
}

// Window and tailcut rules against every camera the array uses.
int check_proc(rta_ctx* c, int mode, int start, int W, bool need_clean, float t_hi, float t_lo) {
    if (mode != RTA_WINDOW_FIXED && mode != RTA_WINDOW_SLIDING && mode != RTA_WINDOW_FILTER &&
        mode != RTA_WINDOW_NEIGHBOUR)
        return fail(RTA_E_INVALID, "bad window mode %d", mode);
    if (mode == RTA_WINDOW_FILTER && c->filter_n != W)
        return fail(RTA_E_INVALID, "filter mode with W = %d but %d weights set", W, c->filter_n);
    if (W < 1 || W > RTA_MAX_W) return fail(RTA_E_INVALID, "window width %d outside 1..%d", W, RTA_MAX_W);
    for (int t = 0; t < c->n_tel; ++t) {
        const HostCam& h = c->cams[c->tel_cam[t]];
        if (W > h.S) return fail(RTA_E_INVALID, "window width %d exceeds %d samples of camera %d", W, h.S, c->tel_cam[t]);
        if (mode == RTA_WINDOW_FIXED && (start < 0 || start + W > h.S))
            return fail(RTA_E_INVALID, "fixed window [%d, %d) outside %d samples", start, start + W, h.S);
    }
    if (need_clean && !(t_hi >= t_lo && t_lo > 0.f))
        return fail(RTA_E_INVALID, "tailcut thresholds need t_hi >= t_lo > 0 (got %g, %g)", t_hi, t_lo);
    return RTA_OK;
}

// Per-call processing parameters of the kernels.
rta::ProcParams make_pp(const rta_ctx* c, int mode, int start, int W, int core_nb, float t_hi, float t_lo) {
    rta::ProcParams pp = {};
    pp.sliding = mode != RTA_WINDOW_FIXED;
    pp.start = start;
    pp.W = W;
    pp.core_nb = core_nb ? 1 : 0;
    pp.t_hi = t_hi;
    pp.t_lo = t_lo;
    pp.one = 1;
    pp.k128 = 128;
    pp.nbpeak = mode == RTA_WINDOW_NEIGHBOUR ? 1 : 0;
    if (mode == RTA_WINDOW_FILTER) {
        pp.filter = 1;
        for (int k = 0; k < W; ++k) {
            pp.wts[k] = c->filter_w[k];
            pp.csum += c->filter_w[k];
        }
    }
    return pp;
}

struct ChainCfg {
    int variant, nstage, ctas_per_sm;
};

// kind: which instantiation (rta::CHAIN_*); the neighbour-peak one also needs its keys in shared memory
int config_launch(rta_ctx* c, const ChainCfg& k, int64_t n_img, int* grid, size_t* smem, int* swb,
                  int kind = rta::CHAIN_PLAIN) {
    const int nb = kind == rta::CHAIN_NB;
    // the stream kernel keeps two per-image records (the neighbour-peak one too: it may run on a stream)
    const int st = kind == rta::CHAIN_STREAM || kind == rta::CHAIN_NB;
    if (k.variant < 0 || k.variant >= RTA_CHAIN_VARIANTS) return fail(RTA_E_INVALID, "variant %d", k.variant);
    const int nst = std::max(2, std::min(k.nstage, 8));
    *swb = rta::chain_stage_wave_bytes(k.variant, c->max_S);
    if (rta::chain_chunk_pixels(k.variant, *swb, c->max_S) < 32)
        return fail(RTA_E_INVALID, "tile variant %d has no room for %d samples", k.variant, c->max_S);
    *smem = rta::chain_smem_bytes(k.variant, nst, *swb, c->max_P, nb, st);
    int occ = rta::chain_occupancy(k.variant, *smem, kind);
    const int want = k.ctas_per_sm > 0 ? k.ctas_per_sm : rta::chain_variant_min_blocks(k.variant);
    if (occ < want) {
        // smaller stages (still at least 128 pixels of the longest camera per
        // chunk) so that the requested number of CTAs fits on an SM
        for (int s2 = (*swb - 1024) & ~127; s2 >= 4096; s2 -= 1024) {
            if (rta::chain_chunk_pixels(k.variant, s2, c->max_S) < 128) break;
            const size_t sm2 = rta::chain_smem_bytes(k.variant, nst, s2, c->max_P, nb, st);
            const int occ2 = rta::chain_occupancy(k.variant, sm2, kind);
            if (occ2 >= want) {
                *swb = s2;
                *smem = sm2;
                occ = occ2;
                break;
            }
        }
    }
    if (occ < 1) return fail(RTA_E_INVALID, "image kernel does not fit: %zu bytes of shared memory", *smem);
    if (k.ctas_per_sm > 0) {
        // a count set (or tuned) for the plain kernel is a ceiling for the other
        // instantiations, whose shared memory or registers may allow fewer
        if (occ < k.ctas_per_sm && kind == rta::CHAIN_PLAIN)
            return fail(RTA_E_INVALID, "%d CTAs/SM do not fit (%d do)", k.ctas_per_sm, occ);
        occ = std::min(occ, k.ctas_per_sm);
    }
    int64_t g = int64_t(c->n_sm) * occ;
    g = std::min<int64_t>(g, std::max<int64_t>(n_img, 1));
    *grid = int(g);
    return RTA_OK;
}

// The configuration the kernel of `kind` runs with: the neighbour-peak kernel has
// its own, the others share the plain kernel's.
ChainCfg cfg_of(const rta_ctx* c, int kind) {
    if (kind == rta::CHAIN_NB) return ChainCfg{c->nb_variant, c->nb_nstage, c->nb_ctas_per_sm};
    if (kind == rta::CHAIN_STREAM && c->st_variant >= 0) return ChainCfg{c->st_variant, c->st_nstage, c->st_ctas_per_sm};
    return ChainCfg{c->variant, c->nstage, c->ctas_per_sm};
}

int chain_launch_config(rta_ctx* c, int64_t n_img, int* grid, size_t* smem, int* swb, int kind = rta::CHAIN_PLAIN) {
    return config_launch(c, cfg_of(c, kind), n_img, grid, smem, swb, kind);
}

int run_chain(rta_ctx* c, const uint16_t* d_wave, int64_t n_wave, const int64_t* d_wave_off, const int32_t* d_img_tel,
              const int64_t* d_pix_off, int64_t n_img, const rta::ProcParams& pp, float* d_q, float* d_t,
              int64_t n_q, rta_hillas_t* d_out, int integrate_only, cudaStream_t s, unsigned int* counter,
              const int64_t* d_n_img = nullptr, const rta_segment_t* d_seg = nullptr,
              const int32_t* d_img_seg = nullptr, int64_t n_seg = 0, rta::StreamImg* d_smeta = nullptr,
              uint8_t* d_mask = nullptr) {
    int grid, swb;
    size_t smem;
    const int kind = pp.nbpeak ? rta::CHAIN_NB : d_smeta ? rta::CHAIN_STREAM : rta::CHAIN_PLAIN;
    int rc = chain_launch_config(c, n_img, &grid, &smem, &swb, kind);
    if (rc) return rc;
    rta::ChainArgs a{};
    a.arr = dev_array(c);
    a.pp = pp;
    a.wave = d_wave;
    a.n_wave = n_wave;
    a.wave_off = d_wave_off;
    a.img_tel = d_img_tel;
    a.pix_off = d_pix_off;
    a.n_q = n_q;
    a.n_img = n_img;
    a.n_img_dev = nullptr;
    a.q_out = d_q;
    a.t_out = d_t;
    a.out = d_out;
    a.mask_out = d_mask;
    a.counter = counter ? counter : take_counter(c);
    a.status = c->d_status;
    a.stage_wave_bytes = swb;
    const ChainCfg cfg = cfg_of(c, kind);
    a.nstage = std::max(2, std::min(cfg.nstage, 8));
    a.integrate_only = integrate_only;
    a.n_img_dev = d_n_img;
    a.seg = d_seg;
    a.img_seg = d_img_seg;
    a.n_seg = n_seg;
    a.smeta = d_smeta;
    if (d_smeta) CUDA_TRY(rta::launch_stream_meta(a, d_smeta, n_img, c->n_sm, s));
    CUDA_TRY(cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), s));
    CUDA_TRY(rta::launch_image_chain(cfg.variant, a, grid, smem, s));
    return RTA_OK;
}

// settled: the kernel before the stereo kernel on the stream is the image kernel, and the event
// offsets and counts were written before it started (read before the dependency wait).
int run_stereo(rta_ctx* c, const rta_hillas_t* d_h, const int32_t* d_img_tel, int64_t n_img, const int32_t* d_evt_off,
               int64_t n_evt, rta_stereo_t* d_out, cudaStream_t s, const int64_t* d_n_img = nullptr,
               const int64_t* d_n_evt = nullptr, bool settled = false) {
    rta::StereoArgs a = {};
    a.settled = settled ? 1 : 0;
    a.arr = dev_array(c);
    a.h = d_h;
    a.img_tel = d_img_tel;
    a.n_img = n_img;
    a.evt_off = d_evt_off;
    a.n_evt = n_evt;
    a.n_img_dev = d_n_img;
    a.n_evt_dev = d_n_evt;
    a.out = d_out;
    a.status = c->d_status;
    const int epb = rta::stereo_events_per_block();
    int64_t g = (n_evt + epb - 1) / epb;
    g = std::min<int64_t>(g, int64_t(c->n_sm) * 16);
    CUDA_TRY(rta::launch_stereo(a, int(std::max<int64_t>(g, 1)), s));
    return RTA_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int check_n(int64_t n, const char* what) {
    if (n < 0 || n > (int64_t(1) << 31) - 1) return fail(RTA_E_INVALID, "%s = %lld outside 0..2^31-1", what, (long long)n);
    return RTA_OK;
}

}  // namespace

// Context tables the surrogate needs, and the stereo pass over a device list of events.
int rta::serve_image_chain(rta_ctx* c, const uint16_t* d_wave, int64_t n_wave, const int64_t* d_wave_off,
                           const int32_t* d_img_tel, const int64_t* d_n_img, int64_t max_img, int window_mode,
                           int start, int W, float t_hi, float t_lo, int core_nb, rta_hillas_t* d_out, cudaStream_t s) {
    int rc = check_ctx(c);
    if (rc || (rc = check_array(c)) || (rc = check_n(max_img, "max_img"))) return rc;
    if ((rc = check_proc(c, window_mode, start, W, true, t_hi, t_lo))) return rc;
    if (!d_wave || !d_wave_off || !d_img_tel || !d_n_img || !d_out || max_img < 1)
        return fail(RTA_E_INVALID, "NULL pointer or empty capacity");
    if (!aligned16(d_wave)) return fail(RTA_E_ALIGN, "d_wave is not 16-byte aligned");
    const rta::ProcParams pp = make_pp(c, window_mode, start, W, core_nb, t_hi, t_lo);
    return run_chain(c, d_wave, n_wave, d_wave_off, d_img_tel, nullptr, max_img, pp, nullptr, nullptr, 0, d_out, 0, s,
                     nullptr, d_n_img);
}

int rta::serve_stereo(rta_ctx* c, const rta_hillas_t* d_h, const int32_t* d_img_tel, int64_t max_img,
                      const int32_t* d_evt_off, int64_t max_evt, const int64_t* d_n_img, const int64_t* d_n_evt,
                      rta_stereo_t* d_out, cudaStream_t s) {
    int rc = check_ctx(c);
    if (rc || (rc = check_array(c))) return rc;
    if (!d_h || !d_img_tel || !d_evt_off || !d_n_img || !d_n_evt || !d_out || max_img < 1 || max_evt < 1)
        return fail(RTA_E_INVALID, "NULL pointer or empty capacity");
    // the counts and offsets were written before the image kernel before it started
    return run_stereo(c, d_h, d_img_tel, max_img, d_evt_off, max_evt, d_out, s, d_n_img, d_n_evt, true);
}

int rta::check_bundle_images(rta_ctx* c, const int64_t* h_wave_off, const int32_t* h_img_tel, int64_t n_img,
                             int64_t n_wave) {
    int rc = check_ctx(c);
    if (rc || (rc = check_array(c))) return rc;
    for (int64_t i = 0; i < n_img; ++i) {
        const int tel = h_img_tel[i];
        if (tel < 0 || tel >= c->n_tel) return fail(RTA_E_INVALID, "image %lld has telescope id %d", (long long)i, tel);
        const HostCam& h = c->cams[c->tel_cam[tel]];
        if (h_wave_off[i] < 0 || (h_wave_off[i] & 7))
            return fail(RTA_E_ALIGN, "image %lld offset not a non-negative multiple of 8", (long long)i);
        if (h_wave_off[i] + int64_t(h.P) * h.S > n_wave) return fail(RTA_E_INVALID, "image %lld ends past n_wave", (long long)i);
    }
    return RTA_OK;
}

int rta::surrogate_ctx_tables(rta_ctx* c, const int32_t** tel_cam, const float2** tel_xy, int* n_tel, int* device) {
    int rc = check_ctx(c);
    if (rc || (rc = check_array(c))) return rc;
    if (tel_cam) *tel_cam = c->d_tel_cam;
    if (tel_xy) *tel_xy = c->d_tel_xy;
    if (n_tel) *n_tel = c->n_tel;
    if (device) *device = c->device;
    return RTA_OK;
}

unsigned int* rta::surrogate_ctx_status(rta_ctx* c) { return c ? c->d_status : nullptr; }

// ======================================================================= C ABI
extern "C" {

int rta_version(void) { return 100; }

const char* rta_last_error(void) { return g_err; }

int rta_create(rta_ctx** out, int device, size_t hbm_budget_bytes) {
    if (!out) return fail(RTA_E_INVALID, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(RTA_E_CUDA, "no CUDA device available");
    if (device < 0 || device >= ndev) return fail(RTA_E_INVALID, "device %d outside 0..%d", device, ndev - 1);
    CUDA_TRY(cudaSetDevice(device));
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, device));
    if (prop.major < 10) return fail(RTA_E_CUDA, "device %d is sm_%d%d; librta is built for sm_103a", device, prop.major, prop.minor);
    rta_ctx* c = new rta_ctx();
    c->device = device;
    c->n_sm = prop.multiProcessorCount;
    c->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t(4) << 30);
    if (cudaMalloc(&c->d_cams, sizeof(rta::DevCam) * RTA_MAX_CAMS) != cudaSuccess ||
        cudaMalloc(&c->d_status, sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc(&c->d_counters, sizeof(unsigned int) * N_COUNTERS) != cudaSuccess) {
        rta_destroy(c);
        return fail(RTA_E_NOMEM, "context allocation failed");
    }
    cudaMemset(c->d_cams, 0, sizeof(rta::DevCam) * RTA_MAX_CAMS);
    cudaMemset(c->d_status, 0, sizeof(unsigned int));
    cudaMemset(c->d_counters, 0, sizeof(unsigned int) * N_COUNTERS);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        rta_destroy(c);
        return fail(RTA_E_CUDA, "device initialisation failed");
    }
    *out = c;
    return RTA_OK;
}

int rta_destroy(rta_ctx* c) {
    if (!c) return RTA_OK;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto& h : c->cams) {
        cudaFree(h.d_xy);
        cudaFree(h.d_nb);
    }
    for (auto& s : c->slot) {
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.meta_done) cudaEventDestroy(s.meta_done);
        cudaFree(s.d_wave); cudaFree(s.d_off); cudaFree(s.d_tel); cudaFree(s.d_evt); cudaFree(s.d_h); cudaFree(s.d_s);
        cudaFreeHost(s.h_off); cudaFreeHost(s.h_tel); cudaFreeHost(s.h_evt);
        cudaFreeHost(s.h_hres); cudaFreeHost(s.h_sres);
        if (s.res_done) cudaEventDestroy(s.res_done);
        if (s.up_done) cudaEventDestroy(s.up_done);
    }
    cudaFree(c->d_cams); cudaFree(c->d_tel_cam); cudaFree(c->d_tel_xy); cudaFree(c->d_tel_row);
    cudaFree(c->d_p16); cudaFree(c->d_scale); cudaFree(c->d_status); cudaFree(c->d_counters);
    cudaFree(c->d_ingest);
    cudaFree(c->d_smeta);
    delete c;
    return RTA_OK;
}

int rta_register_camera(rta_ctx* c, int cam, int n_pix, int n_samples, const float* h_pix_xy, const int16_t* h_nb,
                        int K) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (cam < 0 || cam >= RTA_MAX_CAMS) return fail(RTA_E_INVALID, "camera id %d outside 0..%d", cam, RTA_MAX_CAMS - 1);
    if (n_pix < 1 || n_pix > RTA_MAX_PIX) return fail(RTA_E_INVALID, "n_pix %d outside 1..%d", n_pix, RTA_MAX_PIX);
    if (n_samples < 1 || n_samples > RTA_MAX_SAMPLES)
        return fail(RTA_E_INVALID, "n_samples %d outside 1..%d", n_samples, RTA_MAX_SAMPLES);
    if ((int64_t(n_pix) * n_samples) % 8 != 0)
        return fail(RTA_E_ALIGN, "n_pix*n_samples = %d is not a multiple of 8 (16-byte image rule)", n_pix * n_samples);
    if (K < 1 || K > RTA_NB_PAD) return fail(RTA_E_INVALID, "K = %d outside 1..%d", K, RTA_NB_PAD);
    if (!h_pix_xy || !h_nb) return fail(RTA_E_INVALID, "pixel table is NULL");
    std::vector<int16_t> nb(size_t(n_pix) * RTA_NB_PAD, int16_t(-1));
    for (int p = 0; p < n_pix; ++p)
        for (int j = 0; j < K; ++j) {
            int v = h_nb[size_t(p) * K + j];
            if (v < -1 || v >= n_pix || v == p) return fail(RTA_E_INVALID, "neighbour %d of pixel %d is invalid", v, p);
            nb[size_t(p) * RTA_NB_PAD + j] = int16_t(v);
        }
    HostCam& h = c->cams[cam];
    cudaFree(h.d_xy);
    cudaFree(h.d_nb);
    h = HostCam();
    CUDA_TRY(cudaMalloc(&h.d_xy, sizeof(float2) * n_pix));
    CUDA_TRY(cudaMalloc(&h.d_nb, sizeof(int4) * n_pix));
    CUDA_TRY(cudaMemcpy(h.d_xy, h_pix_xy, sizeof(float2) * n_pix, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(h.d_nb, nb.data(), sizeof(int4) * n_pix, cudaMemcpyHostToDevice));
    h.P = n_pix;
    h.S = n_samples;
    h.K = K;
    h.valid = true;
    return refresh_cams(c);
}

int rta_register_array(rta_ctx* c, int n_tel, const int32_t* h_tel_cam, const float* h_tel_xy, const int32_t* h_p16,
                       const float* h_scale) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (n_tel < 1 || n_tel > RTA_MAX_TEL) return fail(RTA_E_INVALID, "n_tel %d outside 1..%d", n_tel, RTA_MAX_TEL);
    if (!h_tel_cam || !h_tel_xy || !h_p16 || !h_scale) return fail(RTA_E_INVALID, "array table is NULL");
    {
        int64_t n_rows = 0;
        for (int t = 0; t < n_tel; ++t) {
            const int cam = h_tel_cam[t];
            if (cam >= 0 && cam < RTA_MAX_CAMS && c->cams[cam].valid) n_rows += c->cams[cam].P;
        }
        for (int64_t r = 0; r < n_rows; ++r)
            if (!std::isfinite(h_scale[r]) || !(h_scale[r] > 0.f))
                return fail(RTA_E_INVALID, "calibration scale %lld is not finite and positive", (long long)r);
    }
    std::vector<int64_t> row(n_tel);
    int64_t rows = 0, src_rows = 0;
    for (int t = 0; t < n_tel; ++t) {
        int cam = h_tel_cam[t];
        if (cam < 0 || cam >= RTA_MAX_CAMS || !c->cams[cam].valid)
            return fail(RTA_E_INVALID, "telescope %d uses unregistered camera %d", t, cam);
        row[t] = rows;
        rows += (c->cams[cam].P + RTA_CALIB_ALIGN - 1) / RTA_CALIB_ALIGN * RTA_CALIB_ALIGN;
        src_rows += c->cams[cam].P;
    }
    rows += RTA_CALIB_ALIGN;  // slack for the 16-byte rounded tail copy
    std::vector<int32_t> p16(rows, 0);
    std::vector<float> scale(rows, 0.f);
    int64_t s = 0;
    for (int t = 0; t < n_tel; ++t) {
        int P = c->cams[h_tel_cam[t]].P;
        for (int p = 0; p < P; ++p) {
            p16[row[t] + p] = h_p16[s + p];
            scale[row[t] + p] = h_scale[s + p];
        }
        s += P;
    }
    cudaFree(c->d_tel_cam); cudaFree(c->d_tel_xy); cudaFree(c->d_tel_row); cudaFree(c->d_p16); cudaFree(c->d_scale);
    c->d_tel_cam = nullptr; c->d_tel_xy = nullptr; c->d_tel_row = nullptr; c->d_p16 = nullptr; c->d_scale = nullptr;
    c->n_tel = 0;
    CUDA_TRY(cudaMalloc(&c->d_tel_cam, sizeof(int32_t) * n_tel));
    CUDA_TRY(cudaMalloc(&c->d_tel_xy, sizeof(float2) * n_tel));
    CUDA_TRY(cudaMalloc(&c->d_tel_row, sizeof(int64_t) * n_tel));
    CUDA_TRY(cudaMalloc(&c->d_p16, sizeof(int32_t) * rows));
    CUDA_TRY(cudaMalloc(&c->d_scale, sizeof(float) * rows));
    CUDA_TRY(cudaMemcpy(c->d_tel_cam, h_tel_cam, sizeof(int32_t) * n_tel, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->d_tel_xy, h_tel_xy, sizeof(float2) * n_tel, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->d_tel_row, row.data(), sizeof(int64_t) * n_tel, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->d_p16, p16.data(), sizeof(int32_t) * rows, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->d_scale, scale.data(), sizeof(float) * rows, cudaMemcpyHostToDevice));
    c->tel_cam.assign(h_tel_cam, h_tel_cam + n_tel);
    c->n_tel = n_tel;
    (void)src_rows;
    return RTA_OK;
}

int rta_check(rta_ctx* c, void* stream, uint32_t* status_bits) {
    int rc = check_ctx(c);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned int st = 0;
    CUDA_TRY(cudaMemcpy(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(c->d_status, 0, sizeof st));
    if (status_bits) *status_bits = st;
    if (st) return fail(RTA_E_DEVICE, "device status 0x%x (bit0 skipped image, bit1 wait timeout)", st);
    return RTA_OK;
}

int rta_set_chain_config(rta_ctx* c, int variant, int n_stages, int ctas_per_sm) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (n_stages < 2 || n_stages > 8) return fail(RTA_E_INVALID, "n_stages %d outside 2..8", n_stages);
    if (ctas_per_sm < 0 || ctas_per_sm > 8) return fail(RTA_E_INVALID, "ctas_per_sm %d outside 0..8", ctas_per_sm);
    int g, swb;
    size_t sm;
    if ((rc = config_launch(c, ChainCfg{variant, n_stages, ctas_per_sm}, int64_t(1) << 30, &g, &sm, &swb))) return rc;
    c->variant = c->nb_variant = variant;
    c->nstage = c->nb_nstage = n_stages;
    c->ctas_per_sm = c->nb_ctas_per_sm = ctas_per_sm;
    c->st_variant = -1;
    return RTA_OK;
}

int rta_set_filter_weights(rta_ctx* c, const int32_t* w, int W) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (W < 0 || W > RTA_MAX_W || (W > 0 && !w)) return fail(RTA_E_INVALID, "filter of %d weights outside 0..%d", W, RTA_MAX_W);
    int64_t sum = 0;
    for (int k = 0; k < W; ++k) {
        if (w[k] < -4096 || w[k] > 4096) return fail(RTA_E_INVALID, "filter weight %d outside -4096..4096", w[k]);
        sum += w[k];
    }
    if (W > 0 && sum <= 0) return fail(RTA_E_INVALID, "filter weights must have a positive sum");
    c->filter_n = W;
    for (int k = 0; k < RTA_MAX_W; ++k) c->filter_w[k] = k < W ? w[k] : 0;
    return RTA_OK;
}

int rta_get_chain_config(rta_ctx* c, int* variant, int* n_stages, int* ctas_per_sm, int* grid, size_t* smem_bytes) {
    int rc = check_ctx(c);
    if (rc) return rc;
    int g, swb;
    size_t sm;
    rc = chain_launch_config(c, int64_t(1) << 30, &g, &sm, &swb);
    if (rc) return rc;
    if (variant) *variant = c->variant;
    if (n_stages) *n_stages = c->nstage;
    if (ctas_per_sm) *ctas_per_sm = g / c->n_sm;
    if (grid) *grid = g;
    if (smem_bytes) *smem_bytes = sm;
    return RTA_OK;
}

int rta_chain_variant_info(int variant, int* integrator_warps, int* pixels_per_thread) {
    if (variant < 0 || variant >= RTA_CHAIN_VARIANTS) return fail(RTA_E_INVALID, "variant %d", variant);
    if (integrator_warps) *integrator_warps = rta::chain_variant_warps(variant);
    if (pixels_per_thread) *pixels_per_thread = rta::chain_variant_ppt(variant);
    return RTA_OK;
}

}  // extern "C"

namespace {

// Every configuration that fits (variant x 2..6 stages x 1..4 CTAs/SM) of the kernel of `kind`:
// *cv, *cn, *cc (the context's fields for that kind) are set to it, `run` launches the kernel once
// (one warm-up, then `reps` timed launches between CUDA events); the fastest is kept, or the
// previous configuration if a launch failed.
template <class Run>
int tune_sweep(rta_ctx* c, int kind, int64_t n_img, int reps, cudaStream_t s, int* cv, int* cn, int* cc, Run run,
               rta_tune_entry_t* h_entries, int max_entries, int* n_entries) {
    const ChainCfg saved{*cv, *cn, *cc};
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(RTA_E_CUDA, "cudaEventCreate failed");
    }
    ChainCfg best = saved;
    float best_ms = 1e30f;
    int n = 0, rc = RTA_OK;
    for (int v = 0; v < RTA_CHAIN_VARIANTS && !rc; ++v)
        for (int nst = 2; nst <= 6 && !rc; ++nst)
            for (int cps = 1; cps <= 4; ++cps) {
                int g, swb;
                size_t sm;
                if (config_launch(c, ChainCfg{v, nst, cps}, n_img, &g, &sm, &swb, kind) != RTA_OK) continue;
                *cv = v;
                *cn = nst;
                *cc = cps;
                if ((rc = run())) break;
                cudaEventRecord(e0, s);
                for (int r = 0; r < reps && !rc; ++r) rc = run();
                cudaEventRecord(e1, s);
                if (rc) break;
                if (cudaEventSynchronize(e1) != cudaSuccess) { rc = fail(RTA_E_CUDA, "autotune run failed"); break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= reps;
                if (h_entries && n < max_entries) h_entries[n] = rta_tune_entry_t{v, nst, cps, g, ms};
                ++n;
                if (ms < best_ms) { best_ms = ms; best = ChainCfg{v, nst, cps}; }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const ChainCfg keep = rc ? saved : best;
    *cv = keep.variant;
    *cn = keep.nstage;
    *cc = keep.ctas_per_sm;
    if (n_entries) *n_entries = n;
    return rc;
}

// The per-image records of the stream path, grown to max_img images.
int ensure_smeta(rta_ctx* c, int64_t max_img, cudaStream_t s) {
    const size_t need = sizeof(rta::StreamImg) * size_t(max_img);
    if (need <= c->smeta_bytes) return RTA_OK;
    CUDA_TRY(cudaStreamSynchronize(s));
    cudaFree(c->d_smeta);
    c->d_smeta = nullptr;
    c->smeta_bytes = 0;
    CUDA_TRY(cudaMalloc(&c->d_smeta, need));
    c->smeta_bytes = need;
    return RTA_OK;
}

}  // namespace

extern "C" {

int rta_autotune(rta_ctx* c, const uint16_t* d_wave, int64_t n_wave, const int64_t* d_wave_off, const int32_t* d_img_tel,
                 int64_t n_img, int window_mode, int start, int W, float t_hi, float t_lo, int core_needs_neighbour,
                 rta_hillas_t* d_out, int reps, rta_tune_entry_t* h_entries, int max_entries, int* n_entries,
                 void* stream) {
    int rc = check_ctx(c);
    if (rc || (rc = check_array(c)) || (rc = check_n(n_img, "n_img"))) return rc;
    if ((rc = check_proc(c, window_mode, start, W, true, t_hi, t_lo))) return rc;
    if (n_img == 0 || !d_wave || !d_wave_off || !d_img_tel || !d_out) return fail(RTA_E_INVALID, "empty or NULL bundle");
    if (!aligned16(d_wave)) return fail(RTA_E_ALIGN, "d_wave is not 16-byte aligned");
    if (reps < 1) reps = 3;
    cudaStream_t s = (cudaStream_t)stream;
    const rta::ProcParams pp = make_pp(c, window_mode, start, W, core_needs_neighbour, t_hi, t_lo);
    // the neighbour-peak window tunes its own configuration, the other modes the plain kernel's
    const int kind = pp.nbpeak ? rta::CHAIN_NB : rta::CHAIN_PLAIN;
    int* cv = pp.nbpeak ? &c->nb_variant : &c->variant;
    int* cn = pp.nbpeak ? &c->nb_nstage : &c->nstage;
    int* cc = pp.nbpeak ? &c->nb_ctas_per_sm : &c->ctas_per_sm;
    auto run = [&]() {
        return run_chain(c, d_wave, n_wave, d_wave_off, d_img_tel, nullptr, n_img, pp, nullptr, nullptr, 0, d_out, 0, s,
                         nullptr);
    };
    return tune_sweep(c, kind, n_img, reps, s, cv, cn, cc, run, h_entries, max_entries, n_entries);
}

int rta_autotune_stream(rta_ctx* c, const uint8_t* d_stream, int64_t n_bytes, const rta_segment_t* d_seg,
                        int64_t max_seg, const int32_t* d_img_seg, const int32_t* d_img_tel, int64_t max_img,
                        const int64_t* d_counts, int window_mode, int start, int W, float t_hi, float t_lo,
                        int core_needs_neighbour, rta_hillas_t* d_hillas, int reps, rta_tune_entry_t* h_entries,
                        int max_entries, int* n_entries, void* stream) {
    int rc = check_ctx(c);
    if (rc || (rc = check_array(c)) || (rc = check_n(max_img, "max_img"))) return rc;
    if ((rc = check_proc(c, window_mode, start, W, true, t_hi, t_lo))) return rc;
    if (window_mode == RTA_WINDOW_NEIGHBOUR)
        return fail(RTA_E_INVALID, "the neighbour-peak window has one configuration for bundles and streams: rta_autotune");
    if (max_img == 0 || !d_stream || !d_seg || !d_img_seg || !d_img_tel || !d_counts || !d_hillas)
        return fail(RTA_E_INVALID, "empty stream or NULL device pointer");
    if (!aligned16(d_stream)) return fail(RTA_E_ALIGN, "d_stream is not 16-byte aligned");
    if (n_bytes < 0 || max_seg < 1) return fail(RTA_E_INVALID, "bad stream size or segment capacity");
    if (reps < 1) reps = 3;
    cudaStream_t s = (cudaStream_t)stream;
    const rta::ProcParams pp = make_pp(c, window_mode, start, W, core_needs_neighbour, t_hi, t_lo);
    if ((rc = ensure_smeta(c, max_img, s))) return rc;
    // until tuned, the stream kernel follows the plain kernel's configuration: start from it
    // (and follow it again if the sweep fails)
    const int st_before = c->st_variant;
    if (c->st_variant < 0) {
        c->st_variant = c->variant;
        c->st_nstage = c->nstage;
        c->st_ctas_per_sm = c->ctas_per_sm;
    }
    auto run = [&]() {
        return run_chain(c, reinterpret_cast<const uint16_t*>(d_stream), n_bytes / 2, nullptr, d_img_tel, nullptr,
                         max_img, pp, nullptr, nullptr, 0, d_hillas, 0, s, nullptr, d_counts + 1, d_seg, d_img_seg,
                         max_seg, static_cast<rta::StreamImg*>(c->d_smeta));
    };
    rc = tune_sweep(c, rta::CHAIN_STREAM, max_img, reps, s, &c->st_variant, &c->st_nstage, &c->st_ctas_per_sm, run,
                    h_entries, max_entries, n_entries);
    if (rc && st_before < 0) c->st_variant = -1;
    return rc;
}

int rta_calibrate_integrate(rta_ctx* c, const uint16_t* d_wave, int64_t n_wave, const int64_t* d_wave_off,
                            const int32_t* d_img_tel, const int64_t* d_pix_off, int64_t n_img, int window_mode,
                            int start, int W, float* d_q, float* d_t, int64_t n_q, void* stream) {
    int rc = check_ctx(c);
    if (rc || (rc = check_array(c)) || (rc = check_n(n_img, "n_img"))) return rc;
    if ((rc = check_proc(c, window_mode, start, W, false, 0.f, 0.f))) return rc;
    if (n_img == 0) return RTA_OK;
    if (!d_wave || !d_wave_off || !d_img_tel || !d_pix_off || !d_q) return fail(RTA_E_INVALID, "NULL device pointer");
    if (!aligned16(d_wave)) return fail(RTA_E_ALIGN, "d_wave is not 16-byte aligned");
    const rta::ProcParams pp = make_pp(c, window_mode, start, W, 0, 0.f, 0.f);
    if (n_wave < 0 || n_q < 0) return fail(RTA_E_INVALID, "negative buffer length");
    return run_chain(c, d_wave, n_wave, d_wave_off, d_img_tel, d_pix_off, n_img, pp, d_q, d_t, n_q, nullptr, 1,
                     (cudaStream_t)stream, nullptr);
}

int rta_clean(rta_ctx* c, const float* d_q, int64_t n_q, const int32_t* d_img_tel, const int64_t* d_pix_off,
              int64_t n_img, float t_hi, float t_lo, int core_needs_neighbour, uint8_t* d_mask, void* stream) {
    int rc = check_ctx(c);
    if (rc || (rc = check_array(c)) || (rc = check_n(n_img, "n_img"))) return rc;
    if (!(t_hi >= t_lo && t_lo > 0.f)) return fail(RTA_E_INVALID, "tailcut thresholds need t_hi >= t_lo > 0");
    if (n_img == 0) return RTA_OK;
    if (!d_q || !d_img_tel || !d_pix_off || !d_mask) return fail(RTA_E_INVALID, "NULL device pointer");
    rta::CleanArgs a;
    a.arr = dev_array(c);
    a.pp = rta::ProcParams{0, 0, 1, core_needs_neighbour ? 1 : 0, t_hi, t_lo, 1, 128};
    a.q = d_q;
    a.n_q = n_q;
    a.img_tel = d_img_tel;
    a.pix_off = d_pix_off;
    a.n_img = n_img;
    a.mask = d_mask;
    a.status = c->d_status;
    int grid = int(std::min<int64_t>(n_img, int64_t(c->n_sm) * 8));
    CUDA_TRY(rta::launch_clean(a, grid, (cudaStream_t)stream));
    return RTA_OK;
}

int rta_hillas(rta_ctx* c, const float* d_q, const float* d_t, const uint8_t* d_mask, int64_t n_q,
               const int32_t* d_img_tel, const int64_t* d_pix_off, int64_t n_img, rta_hillas_t* d_out, void* stream) {
    int rc = check_ctx(c);
    if (rc || (rc = check_array(c)) || (rc = check_n(n_img, "n_img"))) return rc;
    if (n_img == 0) return RTA_OK;
    if (!d_q || !d_mask || !d_img_tel || !d_pix_off || !d_out) return fail(RTA_E_INVALID, "NULL device pointer");
    rta::HillasArgs a;
    a.arr = dev_array(c);
    a.q = d_q;
    a.t = d_t;
    a.mask = d_mask;
    a.n_q = n_q;
    a.img_tel = d_img_tel;
    a.pix_off = d_pix_off;
    a.n_img = n_img;
    a.out = d_out;
    a.status = c->d_status;
    int grid = int(std::min<int64_t>(n_img, int64_t(c->n_sm) * 8));
    CUDA_TRY(rta::launch_hillas(a, grid, (cudaStream_t)stream));
    return RTA_OK;
}

int rta_image_chain(rta_ctx* c, const uint16_t* d_wave, int64_t n_wave, const int64_t* d_wave_off,
                    const int32_t* d_img_tel, int64_t n_img, int window_mode, int start, int W, float t_hi,
                    float t_lo, int core_needs_neighbour, rta_hillas_t* d_out, void* stream) {
    int rc = check_ctx(c);
    if (rc || (rc = check_array(c)) || (rc = check_n(n_img, "n_img"))) return rc;
    if ((rc = check_proc(c, window_mode, start, W, true, t_hi, t_lo))) return rc;
    if (n_img == 0) return RTA_OK;
    if (!d_wave || !d_wave_off || !d_img_tel || !d_out) return fail(RTA_E_INVALID, "NULL device pointer");
    if (!aligned16(d_wave)) return fail(RTA_E_ALIGN, "d_wave is not 16-byte aligned");
    const rta::ProcParams pp = make_pp(c, window_mode, start, W, core_needs_neighbour, t_hi, t_lo);
    if (n_wave < 0) return fail(RTA_E_INVALID, "negative buffer length");
    return run_chain(c, d_wave, n_wave, d_wave_off, d_img_tel, nullptr, n_img, pp, nullptr, nullptr, 0, d_out, 0,
                     (cudaStream_t)stream, nullptr);
}

int rta_image_chain_masks(rta_ctx* c, const uint16_t* d_wave, int64_t n_wave, const int64_t* d_wave_off,
                          const int32_t* d_img_tel, const int64_t* d_pix_off, int64_t n_img, int window_mode,
                          int start, int W, float t_hi, float t_lo, int core_needs_neighbour, uint8_t* d_mask,
                          int64_t n_q, rta_hillas_t* d_out, void* stream) {
    int rc = check_ctx(c);
    if (rc || (rc = check_array(c)) || (rc = check_n(n_img, "n_img"))) return rc;
    if ((rc = check_proc(c, window_mode, start, W, true, t_hi, t_lo))) return rc;
    if (n_img == 0) return RTA_OK;
    if (!d_wave || !d_wave_off || !d_img_tel || !d_pix_off || !d_mask || !d_out)
        return fail(RTA_E_INVALID, "NULL device pointer");
    if (!aligned16(d_wave)) return fail(RTA_E_ALIGN, "d_wave is not 16-byte aligned");
    if (n_wave < 0 || n_q < 0) return fail(RTA_E_INVALID, "negative buffer length");
    const rta::ProcParams pp = make_pp(c, window_mode, start, W, core_needs_neighbour, t_hi, t_lo);
    return run_chain(c, d_wave, n_wave, d_wave_off, d_img_tel, d_pix_off, n_img, pp, nullptr, nullptr, n_q, d_out, 0,
                     (cudaStream_t)stream, nullptr, nullptr, nullptr, nullptr, 0, nullptr, d_mask);
}

int rta_stereo(rta_ctx* c, const rta_hillas_t* d_hillas, const int32_t* d_img_tel, int64_t n_img,
               const int32_t* d_evt_off, int64_t n_evt, rta_stereo_t* d_out, void* stream) {
    int rc = check_ctx(c);
    if (rc || (rc = check_array(c)) || (rc = check_n(n_evt, "n_evt")) || (rc = check_n(n_img, "n_img"))) return rc;
    if (n_evt == 0) return RTA_OK;
    if (!d_evt_off || !d_out || (n_img > 0 && (!d_hillas || !d_img_tel))) return fail(RTA_E_INVALID, "NULL device pointer");
    return run_stereo(c, d_hillas, d_img_tel, n_img, d_evt_off, n_evt, d_out, (cudaStream_t)stream);
}

int rta_reconstruct(rta_ctx* c, const uint16_t* d_wave, int64_t n_wave, const int64_t* d_wave_off,
                    const int32_t* d_img_tel, int64_t n_img, const int32_t* d_evt_off, int64_t n_evt, int window_mode,
                    int start, int W, float t_hi, float t_lo, int core_needs_neighbour, rta_hillas_t* d_hillas,
                    rta_stereo_t* d_stereo, void* stream) {
    int rc = rta_image_chain(c, d_wave, n_wave, d_wave_off, d_img_tel, n_img, window_mode, start, W, t_hi, t_lo,
                             core_needs_neighbour, d_hillas, stream);
    if (rc) return rc;
    if ((rc = check_n(n_evt, "n_evt"))) return rc;
    if (n_evt == 0) return RTA_OK;
    if (!d_evt_off || !d_stereo) return fail(RTA_E_INVALID, "NULL device pointer");
    // the kernel before the stereo kernel is the image kernel (launched when n_img > 0), which
    // started after the event offsets were written: they are read before the dependency wait
    return run_stereo(c, d_hillas, d_img_tel, n_img, d_evt_off, n_evt, d_stereo, (cudaStream_t)stream, nullptr,
                      nullptr, n_img > 0);
}

int rta_reconstruct_host(rta_ctx* c, const uint16_t* h_wave, int64_t n_wave, const int64_t* h_wave_off,
                         const int32_t* h_img_tel, int64_t n_img, const int32_t* h_evt_off, int64_t n_evt,
                         int window_mode, int start, int W, float t_hi, float t_lo, int core_needs_neighbour,
                         rta_hillas_t* h_hillas, rta_stereo_t* h_stereo) {
    int rc = check_ctx(c);
    if (rc || (rc = check_array(c)) || (rc = check_n(n_img, "n_img")) || (rc = check_n(n_evt, "n_evt"))) return rc;
    if ((rc = check_proc(c, window_mode, start, W, true, t_hi, t_lo))) return rc;
    if (n_evt == 0) return RTA_OK;
    if (!h_wave || !h_wave_off || !h_img_tel || !h_evt_off || !h_hillas || !h_stereo)
        return fail(RTA_E_INVALID, "NULL host pointer");
    if (h_evt_off[0] != 0 || h_evt_off[n_evt] != n_img) return fail(RTA_E_INVALID, "evt_off must run from 0 to n_img");
    // image byte extents from the host tables
    std::vector<int64_t> img_end(static_cast<size_t>(n_img));
    for (int64_t i = 0; i < n_img; ++i) {
        const int tel = h_img_tel[i];
        if (tel < 0 || tel >= c->n_tel) return fail(RTA_E_INVALID, "image %lld has telescope id %d", (long long)i, tel);
        const HostCam& h = c->cams[c->tel_cam[tel]];
        if (h_wave_off[i] < 0 || (h_wave_off[i] & 7)) return fail(RTA_E_ALIGN, "image %lld offset not a multiple of 8", (long long)i);
        if (i && h_wave_off[i] < img_end[i - 1]) return fail(RTA_E_INVALID, "image offsets must be increasing and non-overlapping");
        img_end[i] = h_wave_off[i] + int64_t(h.P) * h.S;
        if (img_end[i] > n_wave) return fail(RTA_E_INVALID, "image %lld ends past n_wave", (long long)i);
    }
    for (int64_t e = 0; e < n_evt; ++e)
        if (h_evt_off[e + 1] < h_evt_off[e]) return fail(RTA_E_INVALID, "evt_off must be non-decreasing");
    std::lock_guard<std::mutex> lock(c->host_mu);
    // chunk plan: whole events, at most `cap` waveform samples per chunk
    const size_t cap_bytes = std::max<size_t>(size_t(64) << 20, std::min<size_t>(c->budget / 2, size_t(512) << 20));
    const int64_t cap = int64_t(cap_bytes / 2);
    struct Chunk { int64_t e0, e1; };
    std::vector<Chunk> chunks;
    int64_t max_img = 0, max_evt = 0;
    for (int64_t e = 0; e < n_evt;) {
        int64_t e1 = e;
        const int64_t i0 = h_evt_off[e];
        while (e1 < n_evt) {
            const int64_t i1 = h_evt_off[e1 + 1];
            if (i1 > i0 && img_end[i1 - 1] - h_wave_off[i0] > cap && e1 > e) break;
            ++e1;
        }
        const int64_t i1 = h_evt_off[e1];
        if (i1 > i0 && img_end[i1 - 1] - h_wave_off[i0] > cap)
            return fail(RTA_E_NOMEM, "one event needs more than the %zu-byte staging buffer", cap_bytes);
        chunks.push_back({e, e1});
        max_img = std::max(max_img, i1 - i0);
        max_evt = std::max(max_evt, e1 - e);
        e = e1;
    }
    // staging buffers (grown on demand, bounded by the budget)
    for (auto& s : c->slot) {
        if (!s.stream) {
            CUDA_TRY(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
            CUDA_TRY(cudaEventCreateWithFlags(&s.meta_done, cudaEventDisableTiming));
            CUDA_TRY(cudaEventCreateWithFlags(&s.res_done, cudaEventDisableTiming));
            CUDA_TRY(cudaEventCreateWithFlags(&s.up_done, cudaEventDisableTiming));
        }
        s.res_pending = false;
        if (s.wave_cap < size_t(cap) * 2) {
            if (c->staged_bytes + size_t(cap) * 2 > c->budget) return fail(RTA_E_NOMEM, "staging exceeds the HBM budget");
            cudaFree(s.d_wave);
            s.d_wave = nullptr;
            CUDA_TRY(cudaMalloc(&s.d_wave, size_t(cap) * 2));
            s.wave_cap = size_t(cap) * 2;
            c->staged_bytes += s.wave_cap;
        }
        if (s.img_cap < size_t(max_img) || s.evt_cap < size_t(max_evt) + 1) {
            cudaFree(s.d_off); cudaFree(s.d_tel); cudaFree(s.d_evt); cudaFree(s.d_h); cudaFree(s.d_s);
            cudaFreeHost(s.h_off); cudaFreeHost(s.h_tel); cudaFreeHost(s.h_evt);
            cudaFreeHost(s.h_hres); cudaFreeHost(s.h_sres);
            s.img_cap = size_t(max_img) + 1024;
            s.evt_cap = size_t(max_evt) + 1024;
            CUDA_TRY(cudaMalloc(&s.d_off, sizeof(int64_t) * s.img_cap));
            CUDA_TRY(cudaMalloc(&s.d_tel, sizeof(int32_t) * s.img_cap));
            CUDA_TRY(cudaMalloc(&s.d_evt, sizeof(int32_t) * s.evt_cap));
            CUDA_TRY(cudaMalloc(&s.d_h, sizeof(rta_hillas_t) * s.img_cap));
            CUDA_TRY(cudaMalloc(&s.d_s, sizeof(rta_stereo_t) * s.evt_cap));
            CUDA_TRY(cudaMallocHost(&s.h_off, sizeof(int64_t) * s.img_cap));
            CUDA_TRY(cudaMallocHost(&s.h_tel, sizeof(int32_t) * s.img_cap));
            CUDA_TRY(cudaMallocHost(&s.h_evt, sizeof(int32_t) * s.evt_cap));
            CUDA_TRY(cudaMallocHost(&s.h_hres, sizeof(rta_hillas_t) * s.img_cap));
            CUDA_TRY(cudaMallocHost(&s.h_sres, sizeof(rta_stereo_t) * s.evt_cap));
        }
    }
    const rta::ProcParams pp = make_pp(c, window_mode, start, W, core_needs_neighbour, t_hi, t_lo);
    for (size_t k = 0; k < chunks.size(); ++k) {
        Slot& s = c->slot[k & 1];
        const int64_t e0 = chunks[k].e0, e1 = chunks[k].e1;
        const int64_t i0 = h_evt_off[e0], i1 = h_evt_off[e1];
        const int64_t ni = i1 - i0, ne = e1 - e0;
        // the pinned metadata of this slot may still feed the copy issued two chunks ago
        CUDA_TRY(cudaEventSynchronize(s.meta_done));
        // hand the slot's previous results to the caller before they are overwritten
        auto deliver = [&](Slot& d) -> int {
            if (!d.res_pending) return RTA_OK;
            CUDA_TRY(cudaEventSynchronize(d.res_done));
            memcpy(h_hillas + d.res_i0, d.h_hres, sizeof(rta_hillas_t) * d.res_ni);
            memcpy(h_stereo + d.res_e0, d.h_sres, sizeof(rta_stereo_t) * d.res_ne);
            d.res_pending = false;
            return RTA_OK;
        };
        if ((rc = deliver(s))) return rc;
        const int64_t base = ni ? h_wave_off[i0] : 0;
        for (int64_t i = 0; i < ni; ++i) s.h_off[i] = h_wave_off[i0 + i] - base;
        if (ni) memcpy(s.h_tel, h_img_tel + i0, sizeof(int32_t) * ni);
        for (int64_t e = 0; e <= ne; ++e) s.h_evt[e] = int32_t(h_evt_off[e0 + e] - i0);
        // uploads go one at a time, in chunk order: the host link is the bottleneck
        // and two concurrent uploads share it less well than one after the other;
        // the kernels of a chunk still overlap the next chunk's upload
        if (k > 0) CUDA_TRY(cudaStreamWaitEvent(s.stream, c->slot[(k - 1) & 1].up_done, 0));
        if (ni) {
            const size_t bytes = size_t(img_end[i1 - 1] - base) * 2;
            CUDA_TRY(cudaMemcpyAsync(s.d_wave, h_wave + base, bytes, cudaMemcpyHostToDevice, s.stream));
            CUDA_TRY(cudaMemcpyAsync(s.d_off, s.h_off, sizeof(int64_t) * ni, cudaMemcpyHostToDevice, s.stream));
            CUDA_TRY(cudaMemcpyAsync(s.d_tel, s.h_tel, sizeof(int32_t) * ni, cudaMemcpyHostToDevice, s.stream));
        }
        CUDA_TRY(cudaMemcpyAsync(s.d_evt, s.h_evt, sizeof(int32_t) * (ne + 1), cudaMemcpyHostToDevice, s.stream));
        CUDA_TRY(cudaEventRecord(s.meta_done, s.stream));
        CUDA_TRY(cudaEventRecord(s.up_done, s.stream));
        if (ni) {
            rc = run_chain(c, s.d_wave, int64_t(s.wave_cap / 2), s.d_off, s.d_tel, nullptr, ni, pp, nullptr, nullptr,
                           0, s.d_h, 0, s.stream, c->d_counters + N_COUNTERS - 1 - (k & 1));
            if (rc) return rc;
            CUDA_TRY(cudaMemcpyAsync(s.h_hres, s.d_h, sizeof(rta_hillas_t) * ni, cudaMemcpyDeviceToHost, s.stream));
        }
        rc = run_stereo(c, s.d_h, s.d_tel, ni, s.d_evt, ne, s.d_s, s.stream);
        if (rc) return rc;
        CUDA_TRY(cudaMemcpyAsync(s.h_sres, s.d_s, sizeof(rta_stereo_t) * ne, cudaMemcpyDeviceToHost, s.stream));
        CUDA_TRY(cudaEventRecord(s.res_done, s.stream));
        s.res_pending = true;
        s.res_i0 = i0;
        s.res_ni = ni;
        s.res_e0 = e0;
        s.res_ne = ne;
    }
    for (auto& d : c->slot) {
        if (!d.res_pending) continue;
        CUDA_TRY(cudaEventSynchronize(d.res_done));
        memcpy(h_hillas + d.res_i0, d.h_hres, sizeof(rta_hillas_t) * d.res_ni);
        memcpy(h_stereo + d.res_e0, d.h_sres, sizeof(rta_stereo_t) * d.res_ne);
        d.res_pending = false;
    }
    CUDA_TRY(cudaStreamSynchronize(c->slot[0].stream));
    CUDA_TRY(cudaStreamSynchronize(c->slot[1].stream));
    return RTA_OK;
}

int rta_selftest_wait_timeout(rta_ctx* c, int timeout_ms, uint64_t* waited_ns, void* stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (timeout_ms < 1 || timeout_ms > 10000) return fail(RTA_E_INVALID, "timeout_ms %d outside 1..10000", timeout_ms);
    unsigned long long* d_w = nullptr;
    CUDA_TRY(cudaMalloc(&d_w, sizeof(unsigned long long)));
    cudaError_t e = rta::launch_wait_selftest(c->d_status, uint64_t(timeout_ms) * 1000000ull, d_w, (cudaStream_t)stream);
    unsigned long long w = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&w, d_w, sizeof w, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    cudaFree(d_w);
    if (e != cudaSuccess) return fail(RTA_E_CUDA, "self-test: %s", cudaGetErrorString(e));
    if (waited_ns) *waited_ns = w;
    return RTA_OK;
}

struct rta_graph {
    rta_ctx* ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned int* counter = nullptr;
};

int rta_graph_create(rta_ctx* c, const uint16_t* d_wave, int64_t n_wave, const int64_t* d_wave_off,
                     const int32_t* d_img_tel, const int64_t* d_n_img, int64_t max_img, const int32_t* d_evt_off,
                     const int64_t* d_n_evt, int64_t max_evt, int window_mode, int start, int W, float t_hi,
                     float t_lo, int core_needs_neighbour, rta_hillas_t* d_hillas, rta_stereo_t* d_stereo,
                     rta_graph** out) {
    int rc = check_ctx(c);
    if (rc || (rc = check_array(c)) || (rc = check_n(max_img, "max_img")) || (rc = check_n(max_evt, "max_evt")))
        return rc;
    if ((rc = check_proc(c, window_mode, start, W, true, t_hi, t_lo))) return rc;
    if (!out || !d_wave || !d_wave_off || !d_img_tel || !d_n_img || !d_evt_off || !d_n_evt || !d_hillas || !d_stereo ||
        max_img < 1 || max_evt < 1)
        return fail(RTA_E_INVALID, "NULL pointer or empty capacity");
    if (!aligned16(d_wave)) return fail(RTA_E_ALIGN, "d_wave is not 16-byte aligned");
    rta_graph* g = new rta_graph();
    g->ctx = c;
    g->counter = take_counter(c);
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        delete g;
        return fail(RTA_E_CUDA, "stream creation failed");
    }
    const rta::ProcParams pp = make_pp(c, window_mode, start, W, core_needs_neighbour, t_hi, t_lo);
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = run_chain(c, d_wave, n_wave, d_wave_off, d_img_tel, nullptr, max_img, pp, nullptr, nullptr, 0, d_hillas, 0,
                       s, g->counter, d_n_img);
        if (!rc) rc = run_stereo(c, d_hillas, d_img_tel, max_img, d_evt_off, max_evt, d_stereo, s, d_n_img, d_n_evt);
        cudaError_t e2 = cudaStreamEndCapture(s, &g->graph);
        if (!rc && e2 != cudaSuccess) rc = fail(RTA_E_CUDA, "capture failed: %s", cudaGetErrorString(e2));
    } else {
        rc = fail(RTA_E_CUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
    }
    if (!rc && cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) rc = fail(RTA_E_CUDA, "graph instantiation failed");
    cudaStreamDestroy(s);
    if (rc) {
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return rc;
    }
    *out = g;
    return RTA_OK;
}

int rta_graph_launch(rta_graph* g, void* stream) {
    if (!g) return fail(RTA_E_INVALID, "graph is NULL");
    int rc = check_ctx(g->ctx);
    if (rc) return rc;
    CUDA_TRY(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return RTA_OK;
}

int rta_graph_destroy(rta_graph* g) {
    if (!g) return RTA_OK;
    cudaSetDevice(g->ctx->device);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return RTA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Lookup tables (k_lut.cu)
// ---------------------------------------------------------------------------
namespace {

int check_lut_axes(const float* se, int n_size, const float* de, int n_dist) {
    if (!se || !de) return fail(RTA_E_INVALID, "NULL edge array");
    if (n_size < 1 || n_size > RTA_LUT_MAX_BINS || n_dist < 1 || n_dist > RTA_LUT_MAX_BINS)
        return fail(RTA_E_INVALID, "bins per axis must be 1..%d (got %d, %d)", RTA_LUT_MAX_BINS, n_size, n_dist);
    return RTA_OK;
}

rta::LutArgs lut_args(rta_ctx* c, const rta_hillas_t* d_h, const int32_t* d_img_tel, int64_t n_img,
                      const int32_t* d_evt_off, int64_t n_evt, const float* se, int n_size, const float* de,
                      int n_dist) {
    rta::LutArgs a{};
    a.arr = dev_array(c);
    a.h = d_h;
    a.img_tel = d_img_tel;
    a.n_img = n_img;
    a.evt_off = d_evt_off;
    a.n_evt = n_evt;
    a.size_edges = se;
    a.n_size = n_size;
    a.dist_edges = de;
    a.n_dist = n_dist;
    a.status = c->d_status;
    return a;
}

}  // namespace

int rta_lut_accumulate(rta_ctx* c, const rta_hillas_t* d_hillas, const int32_t* d_img_tel, int64_t n_img,
                       const int32_t* d_evt_off, int64_t n_evt, const float* d_log_energy, const float* d_core_xy,
                       const uint8_t* d_use, const float* d_size_edges, int n_size, const float* d_dist_edges,
                       int n_dist, double* d_acc, void* stream) {
    int rc = check_ctx(c);
    if (rc || (rc = check_array(c)) || (rc = check_n(n_evt, "n_evt")) || (rc = check_n(n_img, "n_img"))) return rc;
    if ((rc = check_lut_axes(d_size_edges, n_size, d_dist_edges, n_dist))) return rc;
    if (n_evt == 0) return RTA_OK;
    if (!d_evt_off || !d_log_energy || !d_core_xy || !d_acc || (n_img > 0 && (!d_hillas || !d_img_tel)))
        return fail(RTA_E_INVALID, "NULL device pointer");
    if (!aligned16(d_hillas) || (reinterpret_cast<uintptr_t>(d_acc) & 7u))
        return fail(RTA_E_ALIGN, "d_hillas must be 16-byte and d_acc 8-byte aligned");
    rta::LutArgs a = lut_args(c, d_hillas, d_img_tel, n_img, d_evt_off, n_evt, d_size_edges, n_size, d_dist_edges,
                              n_dist);
    a.log_e = d_log_energy;
    a.core_xy = d_core_xy;
    a.use = d_use;
    a.acc = d_acc;
    const int64_t g = std::min<int64_t>((n_evt + 255) / 256, int64_t(c->n_sm) * 8);
    CUDA_TRY(rta::launch_lut_accumulate(a, int(g), (cudaStream_t)stream));
    return RTA_OK;
}

int rta_lut_finalize(rta_ctx* c, const double* d_acc, int64_t n_cells, int min_count, rta_lut_cell_t* d_cells,
                     void* stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (n_cells < 0 || n_cells > int64_t(RTA_MAX_CAMS) * RTA_LUT_MAX_BINS * RTA_LUT_MAX_BINS)
        return fail(RTA_E_INVALID, "n_cells = %lld out of range", (long long)n_cells);
    if (min_count < 1) return fail(RTA_E_INVALID, "min_count must be >= 1");
    if (n_cells == 0) return RTA_OK;
    if (!d_acc || !d_cells) return fail(RTA_E_INVALID, "NULL device pointer");
    if (!aligned16(d_cells) || (reinterpret_cast<uintptr_t>(d_acc) & 7u))
        return fail(RTA_E_ALIGN, "d_cells must be 16-byte and d_acc 8-byte aligned");
    const int64_t g = std::min<int64_t>((n_cells + 255) / 256, int64_t(c->n_sm) * 8);
    CUDA_TRY(rta::launch_lut_finalize(d_acc, n_cells, min_count, d_cells, int(g), (cudaStream_t)stream));
    return RTA_OK;
}

int rta_lut_prepare(rta_ctx* c, const rta_lut_cell_t* d_cells, int64_t n_cells, void* d_lookup, void* stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (n_cells < 0 || n_cells > int64_t(RTA_MAX_CAMS) * RTA_LUT_MAX_BINS * RTA_LUT_MAX_BINS)
        return fail(RTA_E_INVALID, "n_cells = %lld out of range", (long long)n_cells);
    if (n_cells == 0) return RTA_OK;
    if (!d_cells || !d_lookup) return fail(RTA_E_INVALID, "NULL device pointer");
    if (!aligned16(d_cells) || !aligned16(d_lookup)) return fail(RTA_E_ALIGN, "d_cells and d_lookup must be 16-byte aligned");
    const int64_t g = std::min<int64_t>((n_cells + 255) / 256, int64_t(c->n_sm) * 8);
    CUDA_TRY(rta::launch_lut_prepare(d_cells, n_cells, d_lookup, int(g), (cudaStream_t)stream));
    return RTA_OK;
}

int rta_lut_reconstruct(rta_ctx* c, const rta_hillas_t* d_hillas, const int32_t* d_img_tel, int64_t n_img,
                        const int32_t* d_evt_off, int64_t n_evt, const rta_stereo_t* d_stereo,
                        const void* d_lookup, const float* d_size_edges, int n_size,
                        const float* d_dist_edges, int n_dist, float mscw_lo, float mscw_hi, float mscl_lo,
                        float mscl_hi, rta_lut_event_t* d_out, void* stream) {
    int rc = check_ctx(c);
    if (rc || (rc = check_array(c)) || (rc = check_n(n_evt, "n_evt")) || (rc = check_n(n_img, "n_img"))) return rc;
    if ((rc = check_lut_axes(d_size_edges, n_size, d_dist_edges, n_dist))) return rc;
    if (n_evt == 0) return RTA_OK;
    if (!d_evt_off || !d_stereo || !d_lookup || !d_out || (n_img > 0 && (!d_hillas || !d_img_tel)))
        return fail(RTA_E_INVALID, "NULL device pointer");
    if (!aligned16(d_hillas) || !aligned16(d_stereo) || !aligned16(d_lookup) || !aligned16(d_out))
        return fail(RTA_E_ALIGN, "d_hillas, d_stereo, d_lookup and d_out must be 16-byte aligned");
    rta::LutArgs a = lut_args(c, d_hillas, d_img_tel, n_img, d_evt_off, n_evt, d_size_edges, n_size, d_dist_edges,
                              n_dist);
    a.stereo = d_stereo;
    a.lookup = static_cast<const unsigned char*>(d_lookup);
    a.cut[0] = mscw_lo;
    a.cut[1] = mscw_hi;
    a.cut[2] = mscl_lo;
    a.cut[3] = mscl_hi;
    a.out = d_out;
    a.events_per_block = rta::lut_events_per_block(n_evt, c->n_sm);
    const int64_t g = std::min<int64_t>((n_evt + a.events_per_block - 1) / a.events_per_block, int64_t(c->n_sm) * 16);
    CUDA_TRY(rta::launch_lut_reconstruct(a, int(g), (cudaStream_t)stream));
    return RTA_OK;
}

// ---------------------------------------------------------------------------
// DL0 byte-stream ingest (k_ingest.cu) and the zero-copy reconstruction
// ---------------------------------------------------------------------------
int rta_ingest(rta_ctx* c, const uint8_t* d_stream, int64_t n_bytes, int verify_crc, rta_segment_t* d_seg,
               int64_t seg_cap, int32_t* d_img_seg, int32_t* d_img_tel, int64_t img_cap, int32_t* d_evt_off,
               uint64_t* d_evt_number, int64_t* d_evt_time_ns, int64_t evt_cap, int64_t* d_counts, void* stream) {
    int rc = check_ctx(c);
    if (rc || (rc = check_array(c))) return rc;
    if (n_bytes < 0 || seg_cap < 0 || img_cap < 0 || evt_cap < 0 || seg_cap > (int64_t(1) << 31) - 2 ||
        img_cap > (int64_t(1) << 31) - 2 || evt_cap > (int64_t(1) << 31) - 2)
        return fail(RTA_E_INVALID, "negative size or capacity above 2^31 - 2");
    if (!d_counts || !d_seg || !d_img_seg || !d_img_tel || !d_evt_off || !d_evt_number || (n_bytes > 0 && !d_stream))
        return fail(RTA_E_INVALID, "NULL device pointer");
    if (!aligned16(d_stream) || !aligned16(d_seg)) return fail(RTA_E_ALIGN, "d_stream and d_seg must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (n_bytes == 0) {
        // an empty stream is an empty directory
        CUDA_TRY(cudaMemsetAsync(d_counts, 0, 6 * sizeof(int64_t), s));
        const int64_t minus1 = -1;
        CUDA_TRY(cudaMemcpyAsync(d_counts + 5, &minus1, sizeof minus1, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemsetAsync(d_img_seg, 0, sizeof(int32_t), s));
        CUDA_TRY(cudaMemsetAsync(d_evt_off, 0, sizeof(int32_t), s));
        return RTA_OK;
    }
    const int64_t nc = rta::ingest_chunks(n_bytes);
    const int64_t max_pk = seg_cap + 1;
    const int64_t n_blk = (max_pk + 1023) / 1024;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t b_chunks = up(sizeof(rta::IngChunk) * size_t(nc));
    const size_t b_hdr = up(sizeof(rta::IngHdr));
    const size_t b_off = up(sizeof(int64_t) * size_t(max_pk));
    const size_t b_err = up(sizeof(int) * size_t(max_pk));
    const size_t b_scan = up(sizeof(unsigned long long) * size_t(max_pk));
    const size_t b_blk = up(sizeof(unsigned long long) * size_t(n_blk));
    const size_t need = b_chunks + b_hdr + b_off + b_err + b_scan + b_blk;
    if (need > c->ingest_bytes) {
        CUDA_TRY(cudaStreamSynchronize(s));
        cudaFree(c->d_ingest);
        c->d_ingest = nullptr;
        c->ingest_bytes = 0;
        CUDA_TRY(cudaMalloc(&c->d_ingest, need));
        c->ingest_bytes = need;
    }
    unsigned char* w = static_cast<unsigned char*>(c->d_ingest);
    rta::IngestArgs a{};
    a.arr = dev_array(c);
    a.stream = d_stream;
    a.n_bytes = n_bytes;
    a.n_chunks = nc;
    a.chunks = reinterpret_cast<rta::IngChunk*>(w);
    a.hdr = reinterpret_cast<rta::IngHdr*>(w + b_chunks);
    a.pk_off = reinterpret_cast<int64_t*>(w + b_chunks + b_hdr);
    a.pk_err = reinterpret_cast<int*>(w + b_chunks + b_hdr + b_off);
    a.pk_scan = reinterpret_cast<unsigned long long*>(w + b_chunks + b_hdr + b_off + b_err);
    a.blk_sum = reinterpret_cast<unsigned long long*>(w + b_chunks + b_hdr + b_off + b_err + b_scan);
    a.seg = d_seg;
    a.seg_cap = seg_cap;
    a.img_seg = d_img_seg;
    a.img_tel = d_img_tel;
    a.img_cap = img_cap;
    a.evt_off = d_evt_off;
    a.evt_number = d_evt_number;
    a.evt_time = d_evt_time_ns;
    a.evt_cap = evt_cap;
    a.counts = d_counts;
    a.status = c->d_status;
    CUDA_TRY(rta::launch_ingest(a, verify_crc, c->n_sm, s));
    return RTA_OK;
}

int rta_reconstruct_stream(rta_ctx* c, const uint8_t* d_stream, int64_t n_bytes, const rta_segment_t* d_seg,
                           int64_t max_seg, const int32_t* d_img_seg, const int32_t* d_img_tel, int64_t max_img,
                           const int32_t* d_evt_off, int64_t max_evt, const int64_t* d_counts, int window_mode,
                           int start, int W, float t_hi, float t_lo, int core_needs_neighbour,
                           rta_hillas_t* d_hillas, rta_stereo_t* d_stereo, void* stream) {
    int rc = check_ctx(c);
    if (rc || (rc = check_array(c)) || (rc = check_n(max_img, "max_img")) || (rc = check_n(max_evt, "max_evt")))
        return rc;
    if ((rc = check_proc(c, window_mode, start, W, true, t_hi, t_lo))) return rc;
    if (max_img == 0) return RTA_OK;
    if (!d_stream || !d_seg || !d_img_seg || !d_img_tel || !d_counts || !d_hillas || (max_evt > 0 && (!d_evt_off || !d_stereo)))
        return fail(RTA_E_INVALID, "NULL device pointer");
    if (!aligned16(d_stream)) return fail(RTA_E_ALIGN, "d_stream is not 16-byte aligned");
    if (n_bytes < 0 || max_seg < 1) return fail(RTA_E_INVALID, "bad stream size or segment capacity");
    cudaStream_t s = (cudaStream_t)stream;
    const rta::ProcParams pp = make_pp(c, window_mode, start, W, core_needs_neighbour, t_hi, t_lo);
    if ((rc = ensure_smeta(c, max_img, s))) return rc;
    rc = run_chain(c, reinterpret_cast<const uint16_t*>(d_stream), n_bytes / 2, nullptr, d_img_tel, nullptr, max_img,
                   pp, nullptr, nullptr, 0, d_hillas, 0, s, nullptr, d_counts + 1, d_seg, d_img_seg, max_seg,
                   static_cast<rta::StreamImg*>(c->d_smeta));
    if (rc || max_evt == 0) return rc;
    return run_stereo(c, d_hillas, d_img_tel, max_img, d_evt_off, max_evt, d_stereo, s, d_counts + 1, d_counts + 2);
}
