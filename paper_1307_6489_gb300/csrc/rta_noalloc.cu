// rta_image_chain_noalloc: the fused image kernel for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at all or not at the moment they need a
// reconstruction: a real-time process that must not stall (cudaMalloc and
// cudaFree may synchronise the whole device), a host framework that owns every
// byte of device memory through its own pool and forbids other allocations, or
// code that runs inside a region where new allocations are not allowed. Such a
// caller cannot create an rta_ctx, because creating and filling a context
// allocates (camera tables, calibration copies, work counters, status word).
//
// This entry point allocates nothing. The caller passes every input and output
// buffer; the small per-call tables (camera descriptors and the telescope ->
// camera / calibration-row maps) and the kernel's scratch (its work counter and
// status word) live in one file-scope __device__ array of a fixed size. Every
// GPU that loads this library holds that array until the process exits.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "rta.h"
#include "rta_launch.cuh"

namespace {

// Layout of the scratch array, in 32-bit words.
constexpr int kCounterWord = 0;
constexpr int kStatusWord = 1;
constexpr int kCamWord = 64;                                   // DevCam[RTA_NOALLOC_MAX_CAMS]
constexpr int kCamWords = RTA_NOALLOC_MAX_CAMS * int(sizeof(rta::DevCam) / 4);
constexpr int kTelCamWord = kCamWord + kCamWords;              // int32[RTA_NOALLOC_MAX_TEL]
constexpr int kTelRowWord = kTelCamWord + RTA_NOALLOC_MAX_TEL; // int64[RTA_NOALLOC_MAX_TEL]
constexpr int kScratchWords = kTelRowWord + 2 * RTA_NOALLOC_MAX_TEL;

static_assert(sizeof(rta::DevCam) % 8 == 0, "camera table entries are 8-byte multiples");
static_assert(kTelRowWord % 2 == 0, "telescope rows need 8-byte alignment");

// The scratch itself. Its host-side name is only a stand-in: host code must use
// the device address obtained from cudaGetSymbolAddress, never &g_noalloc_scratch.
static __device__ __align__(256) unsigned int g_noalloc_scratch[kScratchWords];

// Failures are reported through rta_last_error(), like every other call.
int nfail(int code, const char* fmt, ...) {
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    rta::set_last_error(msg);
    return code;
}

// Device address of the scratch array, resolved once per device with that device current.
std::mutex g_mu;
unsigned int* g_addr[64] = {};

int scratch_address(int dev, unsigned int** out) {
    if (dev < 0 || dev >= 64) return nfail(RTA_E_INVALID, "device %d not supported", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return nfail(RTA_E_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_addr[dev] = static_cast<unsigned int*>(p);
    }
    *out = g_addr[dev];
    return RTA_OK;
}

#define NA_TRY(call)                                                                              \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return nfail(RTA_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

extern "C" int rta_image_chain_noalloc(const rta_camera_desc_t* h_cams, int n_cams, const int32_t* h_tel_cam,
                                       const int64_t* h_tel_row, int n_tel, const int32_t* d_p16,
                                       const float* d_scale, int64_t n_calib_rows, const uint16_t* d_wave,
                                       int64_t n_wave, const int64_t* d_wave_off, const int32_t* d_img_tel,
                                       int64_t n_img, int window_mode, int start, int W, float t_hi, float t_lo,
                                       int core_needs_neighbour, rta_hillas_t* d_out, uint32_t* d_status,
                                       void* stream) {
    // ---- sizes against the fixed scratch capacity, then the rest of the arguments
    if (!h_cams || n_cams < 1 || n_cams > RTA_NOALLOC_MAX_CAMS)
        return nfail(RTA_E_INVALID, "n_cams = %d outside 1..%d (the fixed scratch holds %d camera descriptors)",
                     n_cams, RTA_NOALLOC_MAX_CAMS, RTA_NOALLOC_MAX_CAMS);
    if (!h_tel_cam || !h_tel_row || n_tel < 1 || n_tel > RTA_NOALLOC_MAX_TEL)
        return nfail(RTA_E_INVALID, "n_tel = %d outside 1..%d (the fixed scratch holds %d telescopes)", n_tel,
                     RTA_NOALLOC_MAX_TEL, RTA_NOALLOC_MAX_TEL);
    if (n_img < 0 || n_img > (int64_t(1) << 31) - 1) return nfail(RTA_E_INVALID, "n_img out of range");
    if (window_mode != RTA_WINDOW_FIXED && window_mode != RTA_WINDOW_SLIDING)
        return nfail(RTA_E_INVALID, "bad window mode %d", window_mode);
    if (W < 1 || W > RTA_MAX_W) return nfail(RTA_E_INVALID, "window width %d outside 1..%d", W, RTA_MAX_W);
    if (!(t_hi >= t_lo && t_lo > 0.f)) return nfail(RTA_E_INVALID, "tailcut thresholds need t_hi >= t_lo > 0");
    rta::DevCam cams[RTA_NOALLOC_MAX_CAMS];
    memset(cams, 0, sizeof cams);
    int max_P = 1, max_S = 1;
    for (int c = 0; c < n_cams; ++c) {
        const rta_camera_desc_t& d = h_cams[c];
        if (d.n_pix < 1 || d.n_pix > RTA_MAX_PIX || d.n_samples < 1 || d.n_samples > RTA_MAX_SAMPLES ||
            d.K < 1 || d.K > RTA_NB_PAD || !d.d_pix_xy || !d.d_nb8)
            return nfail(RTA_E_INVALID, "camera %d: bad size or NULL table", c);
        if ((int64_t(d.n_pix) * d.n_samples) % 8) return nfail(RTA_E_ALIGN, "camera %d: n_pix*n_samples not a multiple of 8", c);
        if ((reinterpret_cast<uintptr_t>(d.d_pix_xy) & 7) || (reinterpret_cast<uintptr_t>(d.d_nb8) & 15))
            return nfail(RTA_E_ALIGN, "camera %d: pixel table misaligned", c);
        if (W > d.n_samples || (window_mode == RTA_WINDOW_FIXED && (start < 0 || start + W > d.n_samples)))
            return nfail(RTA_E_INVALID, "window does not fit the %d samples of camera %d", d.n_samples, c);
        cams[c].P = d.n_pix;
        cams[c].S = d.n_samples;
        cams[c].K = d.K;
        cams[c].xy = reinterpret_cast<const float2*>(d.d_pix_xy);
        cams[c].nb = reinterpret_cast<const int4*>(d.d_nb8);
        max_P = max_P > d.n_pix ? max_P : d.n_pix;
        max_S = max_S > d.n_samples ? max_S : d.n_samples;
    }
    for (int t = 0; t < n_tel; ++t) {
        const int c = h_tel_cam[t];
        if (c < 0 || c >= n_cams) return nfail(RTA_E_INVALID, "telescope %d uses camera %d of %d", t, c, n_cams);
        const int64_t r = h_tel_row[t];
        // calibration rows are read 16 bytes at a time: 8-aligned start, 8 rows of slack after the last pixel
        if (r < 0 || (r & 7) || r + cams[c].P + 8 > n_calib_rows)
            return nfail(RTA_E_INVALID, "telescope %d: calibration row %lld bad for %lld rows", t, (long long)r,
                         (long long)n_calib_rows);
    }
    if (n_img == 0) return RTA_OK;
    if (!d_p16 || !d_scale || !d_wave || !d_wave_off || !d_img_tel || !d_out)
        return nfail(RTA_E_INVALID, "NULL device pointer");
    if ((reinterpret_cast<uintptr_t>(d_wave) & 15) || (reinterpret_cast<uintptr_t>(d_p16) & 15) ||
        (reinterpret_cast<uintptr_t>(d_scale) & 15))
        return nfail(RTA_E_ALIGN, "d_wave, d_p16 and d_scale must be 16-byte aligned");

    // ---- set-up: the scratch's device address on this device
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    NA_TRY(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) return nfail(RTA_E_INVALID, "the stream is being captured");
    int dev = 0;
    NA_TRY(cudaGetDevice(&dev));
    unsigned int* scratch = nullptr;
    int rc = scratch_address(dev, &scratch);
    if (rc) return rc;
    // The tables travel as one copy of a stack image of the scratch's table
    // region, with the work counter and status word (zero) in front: a copy
    // from pageable host memory is staged before cudaMemcpyAsync returns, so
    // no caller array (pinned or not) is read after this call has returned.
    unsigned int image[kScratchWords];
    memset(image, 0, sizeof(unsigned int) * kTelRowWord);
    memcpy(image + kCamWord, cams, sizeof cams);
    memcpy(image + kTelCamWord, h_tel_cam, sizeof(int32_t) * n_tel);
    memcpy(image + kTelRowWord, h_tel_row, sizeof(int64_t) * n_tel);
    NA_TRY(cudaMemcpyAsync(scratch, image, sizeof(unsigned int) * kTelRowWord + sizeof(int64_t) * n_tel,
                           cudaMemcpyHostToDevice, s));

    // ---- the launch: the fused kernel's default tile (8 integrator warps, 1 pixel per thread, 3 stages)
    const int variant = 0, nstage = 3;
    const int swb = rta::chain_stage_wave_bytes(variant, max_S);
    const size_t smem = rta::chain_smem_bytes(variant, nstage, swb, max_P);
    int occ = rta::chain_occupancy(variant, smem);
    if (occ < 1) return nfail(RTA_E_INVALID, "cameras too large for the image kernel's shared memory");
    int n_sm = 0;
    NA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    int64_t grid = int64_t(n_sm) * occ;
    if (grid > n_img) grid = n_img;
    rta::ChainArgs a{};
    memset(&a, 0, sizeof a);
    a.arr.cams = reinterpret_cast<const rta::DevCam*>(scratch + kCamWord);
    a.arr.tel_cam = reinterpret_cast<const int32_t*>(scratch + kTelCamWord);
    a.arr.tel_xy = nullptr;
    a.arr.tel_row = reinterpret_cast<const int64_t*>(scratch + kTelRowWord);
    a.arr.p16 = d_p16;
    a.arr.scale = d_scale;
    a.arr.n_tel = n_tel;
    a.arr.max_P = max_P;
    a.pp = rta::ProcParams{window_mode == RTA_WINDOW_SLIDING, start, W, core_needs_neighbour ? 1 : 0, t_hi, t_lo, 1,
                           128};
    a.wave = d_wave;
    a.n_wave = n_wave;
    a.wave_off = d_wave_off;
    a.img_tel = d_img_tel;
    a.n_img = n_img;
    a.out = d_out;
    a.counter = scratch + kCounterWord;
    a.status = scratch + kStatusWord;
    a.stage_wave_bytes = swb;
    a.nstage = nstage;
    a.integrate_only = 0;
    NA_TRY(rta::launch_image_chain(variant, a, int(grid), smem, s));
    if (d_status)
        NA_TRY(cudaMemcpyAsync(d_status, scratch + kStatusWord, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    return RTA_OK;
}
