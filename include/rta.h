/*
 * librta -- C ABI of the GB300 real-time reconstruction path for Cherenkov
 * telescope arrays: waveform calibration and charge integration, tailcut
 * cleaning, Hillas moments and stereo Hillas intersection.
 *
 * The paper (Bulgarelli et al., "The Real-Time Analysis of the CTA
 * Observatory", ICRC 2013) defines the problem these calls solve: the RT-RECO
 * stage turns the DL0 data of the central event builder (the waveforms of the
 * telescopes triggered by one event, Sec. 2.2 and Sec. 4.1) into an event
 * list through calibration with the calibration matrices and direction (and
 * energy) reconstruction (Sec. 4.1), event by event and with the emphasis on
 * speed (Sec. 4.2), keeping up with 0.5-8 GB/s of input (abstract, Sec. 2.2);
 * Sec. 5 names GPU ports of signal-extraction algorithms. The paper prints no
 * formula; each call below states the definition it computes.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Return value: RTA_OK (0) or a negative rta_status. On failure
 *    rta_last_error() returns a thread-local message. Nothing is launched when
 *    argument checks fail.
 *  - "d_" pointers are device pointers owned by the caller; "h_" pointers are
 *    host pointers owned by the caller. The library owns the context, its copies
 *    of geometry and calibration, and its scratch memory.
 *  - Launch calls are asynchronous on the caller's stream (a cudaStream_t passed
 *    as void*, NULL = legacy default stream). Kernel-side input faults (an image
 *    offset that is not 16-byte aligned, a telescope id out of range) never
 *    fault the GPU: the image is skipped, its output row carries
 *    RTA_HF_BAD_INPUT, and a bit is set in the context's device status word,
 *    which rta_check() reports as RTA_E_DEVICE.
 *  - There is no CPU fallback: every call runs CUDA kernels for sm_103a.
 *
 * Data layout (the bundle)
 * ------------------------
 *  - Waveforms: uint16 ADC samples, pixel-major and sample-minor: image i
 *    occupies d_wave[d_wave_off[i] + p*S + k] for pixel p < P and sample k < S of
 *    its camera. d_wave must be 16-byte aligned and every d_wave_off[i] a
 *    multiple of 8 samples (16 bytes); each registered camera needs P*S to be a
 *    multiple of 8.
 *  - n_wave: number of uint16 samples in d_wave; an image whose samples do not
 *    lie inside [0, n_wave) is skipped (RTA_HF_BAD_INPUT), never read.
 *  - d_img_tel[i]: telescope id of image i (0 <= id < n_tel of rta_register_array).
 *  - d_pix_off[i]: first row of image i in per-pixel arrays (q, t, mask) of
 *    n_q rows; an image whose rows do not fit is skipped.
 *  - d_evt_off[e] .. d_evt_off[e+1]: the images of event e (CSR, ascending,
 *    within [0, n_img)); an event that breaks this is flagged RTA_SF_INVALID.
 *  - Calibration rows: telescope t's pixel p uses row tel_row[t] + p where the
 *    rows of all telescopes are concatenated in telescope order.
 */
#ifndef RTA_H
#define RTA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rta_ctx rta_ctx;

typedef enum {
    RTA_OK = 0,
    RTA_E_INVALID = -1, /* bad argument (size, range, NULL) */
    RTA_E_ALIGN = -2,   /* pointer or camera size violates the 16-byte layout rule */
    RTA_E_NOMEM = -3,   /* device allocation failed or the HBM budget is exceeded */
    RTA_E_CUDA = -4,    /* a CUDA runtime call failed */
    RTA_E_BUSY = -5,    /* a resource is in use; retry later */
    RTA_E_TIMEOUT = -6, /* a bounded device wait ran out */
    RTA_E_DEVICE = -7   /* the device status word reports a skipped input */
} rta_status;

/* Window modes of rta_calibrate_integrate / rta_image_chain */
#define RTA_WINDOW_FIXED 0   /* samples [start, start+W) */
#define RTA_WINDOW_SLIDING 1 /* the W-window of maximal integer sum, lowest start on ties */
#define RTA_WINDOW_FILTER 2  /* the sliding window, charge as an integer-weighted sum over it
                                (digital-filter-style extractor; weights per context, see
                                rta_set_filter_weights) */
#define RTA_WINDOW_NEIGHBOUR 3 /* neighbour-peak window: every pixel's sliding window and its
                                  charge first; then a pixel integrates its own samples in the
                                  window of the brightest pixel (largest charge, then earliest
                                  start) of itself and its registered neighbours. The image is
                                  read twice (the second time from L2); `start` is ignored. */

/* Hillas row flags */
#define RTA_HF_EMPTY 1u     /* no pixel survived cleaning: every field but n_pix is 0 */
#define RTA_HF_NO_TIME 2u   /* fewer than two pixels: time_grad is 0 */
#define RTA_HF_BAD_INPUT 4u /* image skipped (misaligned offset or bad telescope id) */

/* Stereo row flags */
#define RTA_SF_INVALID 1u   /* no usable image pair: direction and core are 0 */

/* Device status word bits (rta_check) */
#define RTA_DEV_BAD_IMAGE 1u
#define RTA_DEV_TIMEOUT 2u
#define RTA_DEV_BAD_STREAM 4u   /* rta_ingest met a malformed byte stream (see its counts) */

/* One image's parameters, 64 bytes. Angles in radians, positions in degrees of
 * the flat camera (nominal) frame, time in samples (ns at 1 GS/s). */
typedef struct rta_hillas_t {
    float size;      /* sum of cleaned charges, photoelectrons */
    float x, y;      /* charge-weighted centroid */
    float length;    /* sqrt(lambda1) of the charge-weighted covariance */
    float width;     /* sqrt(lambda2), computed as sqrt(det / lambda1) */
    float psi;       /* major-axis angle, atan2(2 sxy, sxx - syy) / 2, in (-pi/2, pi/2] */
    float r, phi;    /* polar coordinates of the centroid */
    float time_grad; /* charge-weighted least-squares slope of pixel time along the major axis */
    float time_mean; /* charge-weighted mean pixel time */
    int32_t n_pix;   /* pixels that survived cleaning */
    uint32_t flags;  /* RTA_HF_* */
    float reserved[4];
} rta_hillas_t;

/* One event's stereo result, 32 bytes. */
typedef struct rta_stereo_t {
    float dir_x, dir_y;   /* reconstructed direction, degrees in the nominal frame */
    float core_x, core_y; /* reconstructed impact point, metres on the ground */
    int32_t n_valid;      /* images used (n_pix >= 3) */
    uint32_t flags;       /* RTA_SF_* */
    float reserved[2];
} rta_stereo_t;

/* One event of the learned reconstruction, 32 bytes. */
typedef struct rta_event_t {
    float log_energy;     /* log10(E / TeV) */
    float dir_x, dir_y;   /* direction, degrees in the nominal frame */
    float gammaness;      /* gamma-likeness in (0, 1) */
    int32_t n_used;       /* images with >= 3 pixels (-1: malformed event) */
    uint32_t flags;       /* RTA_EF_* */
    float base_x, base_y; /* the two-image baseline the learned offsets refer to */
} rta_event_t;

#define RTA_EF_NO_DIRECTION 1u /* fewer than 2 used images: no direction (geometric undefined too) */
#define RTA_EF_FALLBACK 2u     /* learned and baseline directions disagree: geometric direction used */

/* ---------------------------------------------------------------------- */
/* Context                                                                 */
/* ---------------------------------------------------------------------- */

/* Library ABI version (major*100 + minor). */
int rta_version(void);

/* Thread-local description of the last failure on this thread ("" if none). */
const char* rta_last_error(void);

/* Create a context on CUDA device `device`. hbm_budget_bytes bounds the
 * device memory the library itself may allocate for staging buffers of the
 * host-buffer calls (0 = 4 GiB). Allocates the context's device status word
 * and work counters. Returns RTA_E_CUDA if the device cannot be used. */
int rta_create(rta_ctx** out, int device, size_t hbm_budget_bytes);

/* Release every device and host resource of the context. Synchronises the
 * device first. NULL is accepted. */
int rta_destroy(rta_ctx* ctx);

/* Register camera type `cam` (0 <= cam < 16): n_pix pixels (1..4096), n_samples
 * samples per pixel (1..128, n_pix*n_samples a multiple of 8), pixel centres
 * h_pix_xy[2*p], h_pix_xy[2*p+1] in degrees, and neighbour lists
 * h_nb[p*K + j] (pixel ids, -1 padded, 1 <= K <= 8). Host arrays are copied. */
int rta_register_camera(rta_ctx* ctx, int cam, int n_pix, int n_samples, const float* h_pix_xy,
                        const int16_t* h_nb, int K);

/* Register the array: n_tel telescopes (1..1024) with camera type h_tel_cam[t]
 * (already registered), ground position h_tel_xy[2t], h_tel_xy[2t+1] in metres,
 * and the calibration table (Sec. 4.1 "calibration matrices"): per row the
 * pedestal in 1/16 ADC fixed point h_p16[row] and the FP32 factor
 * h_scale[row] = 1 / (16 * gain * window containment) that converts the
 * 1/16-ADC window numerator into photoelectrons (finite and > 0, else
 * RTA_E_INVALID). Rows of telescope t start at sum of n_pix of telescopes < t.
 * Host arrays are copied. */
int rta_register_array(rta_ctx* ctx, int n_tel, const int32_t* h_tel_cam, const float* h_tel_xy,
                       const int32_t* h_p16, const float* h_scale);

/* Synchronise `stream`, then read and clear the device status word.
 * Returns RTA_OK, RTA_E_DEVICE (bits in *status_bits, may be NULL) or RTA_E_CUDA. */
int rta_check(rta_ctx* ctx, void* stream, uint32_t* status_bits);

/* Failure-detection self-test (availability > 98 %, Sec. 2.1): a one-thread
 * kernel waits, through the same bounded mbarrier wait as the image kernel, on a
 * barrier nothing completes. After timeout_ms (1..10000) the wait gives up, the
 * device status word gets RTA_DEV_TIMEOUT (read it with rta_check) and the
 * kernel returns normally; the context stays usable. *waited_ns (may be NULL)
 * receives the device-measured wait. Synchronises `stream`. */
int rta_selftest_wait_timeout(rta_ctx* ctx, int timeout_ms, uint64_t* waited_ns, void* stream);

/* Launch configuration of the fused image kernel (rta_image_chain and the
 * calls built on it). variant selects the tile shape (rta_chain_variant_info:
 * integrator warps per CTA and pixels per thread), n_stages the shared-memory
 * pipeline depth (2..8), ctas_per_sm the resident CTAs per SM (0 = as many as
 * fit). Sets the configuration of every window mode, the neighbour-peak
 * window's included (whose kernel runs with as many of the CTAs as fit), and
 * of the byte-stream path (rta_reconstruct_stream), undoing what
 * rta_autotune_stream tuned. Returns RTA_E_INVALID if the combination does not fit in shared memory for
 * the registered cameras. Results do not depend on the configuration. */
int rta_set_chain_config(rta_ctx* ctx, int variant, int n_stages, int ctas_per_sm);

/* The configuration a launch outside the neighbour-peak mode would use now (the
 * byte-stream path too, unless rta_autotune_stream has tuned its own):
 * variant, stages, CTAs per SM, grid size and dynamic shared memory per CTA in
 * bytes (NULL outputs are skipped). */
int rta_get_chain_config(rta_ctx* ctx, int* variant, int* n_stages, int* ctas_per_sm, int* grid,
                         size_t* smem_bytes);

/* Weights of the digital-filter-style extractor (window_mode RTA_WINDOW_FILTER;
 * a signal-extraction alternative to the flat window sum, Sec. 5): W integer
 * weights c_k, |c_k| <= 4096, sum > 0. With st the sliding window's start, the
 * charge is q = fl32(16 * sum_k c_k s[st+k] - (sum_k c_k) * p16) * scale: exact
 * 64-bit integers, one rounding to FP32, one FP32 multiply (the calibration
 * scale then normalises the filter); st and the peak time are those of the flat
 * window. A call in RTA_WINDOW_FILTER mode must pass this W. Copied; W = 0
 * clears. Not available to rta_image_chain_noalloc. */
int rta_set_filter_weights(rta_ctx* ctx, const int32_t* weights, int W);

/* Tile shape of a variant (0 .. RTA_CHAIN_VARIANTS-1). Variant 4 has the shape of
 * variant 0, compiled for at most 68 registers per thread so that three CTAs fit on
 * an SM (with stages shrunk to fit their shared memory). */
#define RTA_CHAIN_VARIANTS 5
int rta_chain_variant_info(int variant, int* integrator_warps, int* pixels_per_thread);

/* One measured configuration of rta_autotune. */
typedef struct rta_tune_entry_t {
    int variant, n_stages, ctas_per_sm, grid;
    float ms; /* mean duration of one rta_image_chain launch */
} rta_tune_entry_t;

/* The autotuner: runs rta_image_chain on the given device-resident bundle for
 * every configuration that fits (variant x 2..6 stages x 1..4 CTAs/SM), `reps`
 * timed launches each (CUDA events on `stream`), keeps the fastest in the
 * context and reports every measurement in h_entries (up to max_entries;
 * *n_entries = number measured). The neighbour-peak window
 * (RTA_WINDOW_NEIGHBOUR) has a configuration of its own, which a call in that
 * mode tunes; a call in any other mode tunes the configuration all other modes
 * share. d_out receives the (configuration-independent) Hillas rows.
 * Synchronises `stream`. */
int rta_autotune(rta_ctx* ctx, const uint16_t* d_wave, int64_t n_wave, const int64_t* d_wave_off,
                 const int32_t* d_img_tel, int64_t n_img, int window_mode, int start, int W, float t_hi,
                 float t_lo, int core_needs_neighbour, rta_hillas_t* d_out, int reps, rta_tune_entry_t* h_entries,
                 int max_entries, int* n_entries, void* stream);

/* ---------------------------------------------------------------------- */
/* Stage calls (Sec. 4.1 calibration; Sec. 5 signal extraction)            */
/* ---------------------------------------------------------------------- */

/* Calibration + charge integration of n_img images. Per pixel:
 *   window start s: `start` (RTA_WINDOW_FIXED) or the first start maximising the
 *   integer W-sample sum (RTA_WINDOW_SLIDING);
 *   num = 16 * sum - W * p16 (exact integer);  q = fp32(num) * scale (one FP32
 *   multiply, round to nearest, never fused);
 *   t = s + sum_j j * (16 * w[s+j] - p16) / num in FP32, or s + (W-1)/2 if num <= 0.
 * Writes d_q[d_pix_off[i] + p] (photoelectrons) and, if d_t != NULL, d_t (samples).
 * 1 <= W <= min(S, 16) for every camera the bundle uses; fixed windows need
 * start + W <= S. */
int rta_calibrate_integrate(rta_ctx* ctx, const uint16_t* d_wave, int64_t n_wave, const int64_t* d_wave_off,
                            const int32_t* d_img_tel, const int64_t* d_pix_off, int64_t n_img, int window_mode,
                            int start, int W, float* d_q, float* d_t, int64_t n_q, void* stream);

/* Two-threshold tailcut cleaning of n_img images (charges d_q as written by
 * rta_calibrate_integrate):
 *   core     = q >= t_hi, and (if core_needs_neighbour) a neighbour with q >= t_hi
 *   boundary = q >= t_lo and a core neighbour;   mask = core | boundary (one pass).
 * Writes d_mask[d_pix_off[i] + p] in {0, 1}. Requires t_hi >= t_lo > 0. */
int rta_clean(rta_ctx* ctx, const float* d_q, int64_t n_q, const int32_t* d_img_tel, const int64_t* d_pix_off,
              int64_t n_img, float t_hi, float t_lo, int core_needs_neighbour, uint8_t* d_mask, void* stream);

/* Hillas moments of n_img cleaned images (FP32, two-pass about the centroid),
 * plus the time gradient when d_t != NULL. Writes d_out[i]. */
int rta_hillas(rta_ctx* ctx, const float* d_q, const float* d_t, const uint8_t* d_mask, int64_t n_q,
               const int32_t* d_img_tel, const int64_t* d_pix_off, int64_t n_img, rta_hillas_t* d_out, void* stream);

/* The fused hot path: calibrate + integrate + clean + Hillas in one persistent
 * launch over a mixed-camera bundle; per-pixel values stay in shared memory and
 * only d_out[i] is written. Same definitions and argument rules as the three
 * calls above. */
int rta_image_chain(rta_ctx* ctx, const uint16_t* d_wave, int64_t n_wave, const int64_t* d_wave_off,
                    const int32_t* d_img_tel, int64_t n_img, int window_mode, int start, int W, float t_hi,
                    float t_lo, int core_needs_neighbour, rta_hillas_t* d_out, void* stream);

/* rta_image_chain that also writes each image's cleaning mask, for checking or
 * displaying cleaned images: d_mask[d_pix_off[i] + p] = 1 when pixel p of image
 * i survived cleaning, else 0 (the rule of rta_clean). The same kernel template,
 * definitions and Hillas rows (bit for bit) as rta_image_chain, compiled with
 * this per-pixel output. Rows of skipped images (RTA_HF_BAD_INPUT) are not
 * written; an image whose rows do not fit n_q mask rows keeps its Hillas row,
 * is not written, and sets RTA_DEV_BAD_IMAGE. */
int rta_image_chain_masks(rta_ctx* ctx, const uint16_t* d_wave, int64_t n_wave, const int64_t* d_wave_off,
                          const int32_t* d_img_tel, const int64_t* d_pix_off, int64_t n_img, int window_mode,
                          int start, int W, float t_hi, float t_lo, int core_needs_neighbour, uint8_t* d_mask,
                          int64_t n_q, rta_hillas_t* d_out, void* stream);

/* Stereo Hillas intersection of n_evt events (direction reconstruction,
 * Sec. 4.1). Images with n_pix >= 3 are used. For each used pair i < j with
 * |sin(psi_j - psi_i)| >= 1e-6, the major axes u = (cos psi, sin psi) through
 * the centroids meet at p_ij = c_i + u_i * cross(c_j - c_i, u_j) / sin(psi_j - psi_i)
 * and, drawn through the telescope positions T, at g_ij on the ground; with
 * w_ij = |sin(psi_i - psi_j)| * s_i s_j / (s_i + s_j) * (1 - W_i/L_i)(1 - W_j/L_j)
 * the direction is sum w p / sum w and the core sum w g / sum w. Events with no
 * usable pair get RTA_SF_INVALID. d_evt_off has n_evt + 1 entries; at most 64
 * images per event are used. */
int rta_stereo(rta_ctx* ctx, const rta_hillas_t* d_hillas, const int32_t* d_img_tel, int64_t n_img,
               const int32_t* d_evt_off, int64_t n_evt, rta_stereo_t* d_out, void* stream);

/* One pass of the whole path over a device-resident bundle:
 * rta_image_chain followed by rta_stereo, stream-ordered, no host sync and no
 * allocation (capturable in a CUDA graph). d_hillas must hold n_img rows.
 * Because the kernel before the stereo kernel is then the image kernel, the
 * stereo kernel reads the event offsets while the image kernel is finishing:
 * d_evt_off must not change between the call and the end of its work on the
 * stream. The same rows as the two calls made one after the other. */
int rta_reconstruct(rta_ctx* ctx, const uint16_t* d_wave, int64_t n_wave, const int64_t* d_wave_off,
                    const int32_t* d_img_tel, int64_t n_img, const int32_t* d_evt_off, int64_t n_evt, int window_mode,
                    int start, int W, float t_hi, float t_lo, int core_needs_neighbour, rta_hillas_t* d_hillas,
                    rta_stereo_t* d_stereo, void* stream);

/* The pass of rta_reconstruct captured once into a CUDA graph (one memset and
 * two kernel launches) for repeated launches on fixed buffers. The graph is
 * captured at capacity (max_img images, max_evt events); the actual counts are
 * read at run time from the device-resident int64 values *d_n_img (<= max_img)
 * and *d_n_evt (<= max_evt), so one graph serves bundles of any size up to its
 * capacity: write the counts (and the bundle) on the launch stream, then
 * rta_graph_launch. All buffers must stay valid for the graph's lifetime; the
 * launch configuration is the context's at capture time. Launches of one graph
 * must not overlap on the GPU (they share a work counter). */
typedef struct rta_graph rta_graph;
int rta_graph_create(rta_ctx* ctx, const uint16_t* d_wave, int64_t n_wave, const int64_t* d_wave_off,
                     const int32_t* d_img_tel, const int64_t* d_n_img, int64_t max_img, const int32_t* d_evt_off,
                     const int64_t* d_n_evt, int64_t max_evt, int window_mode, int start, int W, float t_hi,
                     float t_lo, int core_needs_neighbour, rta_hillas_t* d_hillas, rta_stereo_t* d_stereo,
                     rta_graph** out);
int rta_graph_launch(rta_graph* graph, void* stream);
int rta_graph_destroy(rta_graph* graph);

/* The same pass over a bundle in HOST memory (pinned memory gives full copy
 * speed): the library copies the bundle to its own device staging buffers in
 * event-aligned chunks, overlapping the copy of chunk k+1 with the work on
 * chunk k, and copies the results back into h_hillas[n_img] and
 * h_stereo[n_evt]. Blocks until the results are in host memory. Host offsets
 * are as on the device. Staging memory is bounded by the context's budget. */
int rta_reconstruct_host(rta_ctx* ctx, const uint16_t* h_wave, int64_t n_wave, const int64_t* h_wave_off,
                         const int32_t* h_img_tel, int64_t n_img, const int32_t* h_evt_off, int64_t n_evt,
                         int window_mode, int start, int W, float t_hi, float t_lo, int core_needs_neighbour,
                         rta_hillas_t* h_hillas, rta_stereo_t* h_stereo);

/* ---------------------------------------------------------------------- */
/* Learned reconstruction: deep-sets surrogate (Sec. 4.1 energy, direction, */
/* gamma/hadron separation)                                                */
/* ---------------------------------------------------------------------- */
/* Features per image (from its Hillas row and telescope; images with >= 3
 * pixels are used): log10 size, centroid minus the event baseline b (x, y),
 * length, width, cos 2psi, sin 2psi, time_grad / 10, |centroid - b|, camera type
 * code, telescope x / 1000 m, y / 1000 m. The baseline b is the axis
 * intersection of the event's two brightest used images when
 * |sin(psi_2 - psi_1)| >= 0.1, else their size-weighted mean centroid.
 * Network: phi 12 -> 128 -> 128 (ReLU) per image; pooling
 * [sum / 40, mean] over used images (256); rho 256 -> 256 (ReLU) -> 4 =
 * (log10 E/TeV, direction offset from b in x and y (deg), gammaness logit).
 * Weights are BF16 copies of FP32 master weights; the GEMMs run on the tensor
 * cores with FP32 accumulation; activations are stored in BF16.
 * Loss (mean over events): gammas (y0 - log10 E)^2 + |y_12 - (src - b)|^2 / 0.1^2,
 * all events BCE(sigmoid(y3), is_gamma). Adam(0.9, 0.999, 1e-8), bias-corrected.
 * Packed parameter order (rta_surrogate_num_params() floats, row-major):
 * W1[12x128], b1[128], W2[128x128], b2[128], V1[256x256], c1[256], V2[256x4], c2[4].
 * The model borrows the context's telescope tables and must not outlive it.
 * Forward and training calls that need a larger batch than any before grow the
 * model's device workspace (an allocation); inference needs none. */
typedef struct rta_model rta_model;
int rta_surrogate_num_params(void);
/* h_cam_code: RTA_MAX_CAMS floats, the type code of each camera id (NULL = zeros). */
int rta_surrogate_create(rta_ctx* ctx, uint64_t seed, const float* h_cam_code, rta_model** out);
int rta_surrogate_destroy(rta_model* model);
/* Replaces the FP32 parameters (packed order) and rebuilds the BF16 copy and the
 * tensor-core layout; waits for all work on the device first. Synchronous. */
int rta_surrogate_set_params(rta_model* model, const float* h_params);
/* which: 0 parameters, 1 last gradients, 2 Adam first moments, 3 second moments. Synchronises. */
int rta_surrogate_get_params(rta_model* model, int which, float* h_out);
/* Checkpoint and resume of training: the FP32 parameters, Adam's first and
 * second moments (each rta_surrogate_num_params() floats in the packed order of
 * rta_surrogate_set_params) and the number of Adam steps taken, which sets the
 * bias corrections of the next step. get_state synchronises the device and
 * fills the non-NULL arrays; set_state waits for all work on the device, then
 * replaces the whole state (the BF16 copy
 * and the tensor-core layout of the weights are rebuilt), so that training
 * resumed from a saved state takes the same steps as training that never
 * stopped. Synchronous. */
int rta_surrogate_get_state(rta_model* model, float* h_params, float* h_m, float* h_v, int64_t* step);
int rta_surrogate_set_state(rta_model* model, const float* h_params, const float* h_m, const float* h_v,
                            int64_t step);
/* Raw network outputs d_y[n_evt*4] and baselines d_base[n_evt*2] (either may be NULL). */
int rta_surrogate_forward(rta_model* model, const rta_hillas_t* d_hillas, const int32_t* d_img_tel, int64_t n_img,
                          const int32_t* d_evt_off, int64_t n_evt, float* d_y, float* d_base, void* stream);
/* One training step on a batch: loss into *d_loss (may be NULL), gradients into
 * the model and, when apply_update != 0, one Adam update with learning rate lr.
 * Labels per event: d_log_energy (log10 E/TeV), d_src_xy (true direction, 2
 * floats, deg), d_is_gamma (0/1). */
int rta_surrogate_train_step(rta_model* model, const rta_hillas_t* d_hillas, const int32_t* d_img_tel, int64_t n_img,
                             const int32_t* d_evt_off, int64_t n_evt, const float* d_log_energy, const float* d_src_xy,
                             const uint8_t* d_is_gamma, float lr, int apply_update, float* d_loss, void* stream);
/* Inference: energy, direction (baseline + learned offset), gammaness. Events
 * with fewer than 2 used images get RTA_EF_NO_DIRECTION (the geometric method
 * is undefined too); events whose learned offset from the baseline exceeds
 * fallback_deg get the geometric intersection of rta_stereo (computed for those
 * events only, the same bits as rta_stereo gives them) and RTA_EF_FALLBACK, or
 * RTA_EF_NO_DIRECTION when that intersection is invalid. One kernel launch, no
 * model workspace and no allocation: calls on different streams may overlap. */
int rta_surrogate_infer(rta_model* model, const rta_hillas_t* d_hillas, const int32_t* d_img_tel, int64_t n_img,
                        const int32_t* d_evt_off, int64_t n_evt, float fallback_deg, rta_event_t* d_out, void* stream);

/* The learned reconstruction of a bundle (Sec. 4.1) in one call: rta_image_chain on the
 * waveforms (Hillas rows into d_hillas, as that call) followed, on the same
 * stream, by rta_surrogate_infer on those rows (event rows into d_events, as
 * that call), with the model's context and camera set-up. Because the kernel
 * before the inference kernel is then known to be the image kernel, the
 * inference kernel reads the event offsets, telescope ids and weights while
 * the image kernel is still finishing, and waits only for the Hillas rows:
 * d_evt_off, d_img_tel and the model's weights must not change between the
 * call and the end of its work on the stream (no training step of the model on
 * another stream meanwhile). Errors as the
 * two calls; nothing is allocated. The same events and rows as the two calls
 * made one after the other, bit for bit. */
int rta_reconstruct_learned(rta_model* model, const uint16_t* d_wave, int64_t n_wave, const int64_t* d_wave_off,
                            const int32_t* d_img_tel, int64_t n_img, const int32_t* d_evt_off, int64_t n_evt,
                            int window_mode, int start, int W, float t_hi, float t_lo, int core_needs_neighbour,
                            float fallback_deg, rta_hillas_t* d_hillas, rta_event_t* d_events, void* stream);

/* ---------------------------------------------------------------------- */
/* DL0 byte-stream ingest (Sec. 5: the telescope data as a stream of bytes  */
/* formatted like satellite telemetry)                                     */
/* ---------------------------------------------------------------------- */
/* The paper names the standard (CCSDS space packets with a PUS telemetry
 * secondary header), not the packet contents; this is the layout librta reads.
 * A packet carries a pixel range (segment) of one image. Packets start on
 * 16-byte boundaries and follow one another with no gap; header fields are
 * big-endian, samples little-endian.
 *   bytes   field
 *   0-1     version 0 (3 bits) | type 0 = telemetry (1) | secondary header 1 (1)
 *           | APID = telescope id (11)
 *   2-3     sequence flags (2 bits: 3 = the whole image, 1 = first, 0 =
 *           continuation, 2 = last segment) | sequence count (14, not checked)
 *   4-5     packet data length = packet bytes - 7
 *   6       0x10: PUS version 1 in the high nibble
 *   7       service type 200 (camera data)
 *   8       service subtype 1 (waveform segment)
 *   9       destination id (not checked)
 *   10-13   event time, seconds (CUC coarse time)
 *   14-15   event time, 1/65536 s (CUC fine time)
 *   16-23   event number
 *   24-25   first pixel of the segment
 *   26-27   pixels in the segment, n (n x samples a multiple of 8)
 *   28-29   pixels of the image (must equal the camera's)
 *   30-31   samples per pixel (must equal the camera's)
 *   32 ...  n x samples uint16 samples, pixel-major (the DL0 bundle layout)
 *   +14     zero padding
 *   +2      packet error control: CRC-16-CCITT (polynomial 0x1021, initial
 *           value 0xFFFF, no reflection, no final XOR) of every byte before it
 * A packet is 48 + 2 n S bytes, at most 65536. The segments of an image follow
 * one another in pixel order, starting at pixel 0 and ending at the image's last
 * pixel; an event is a run of images with the same event number. */
#define RTA_PKT_HEADER_BYTES 32
#define RTA_PKT_TRAILER_BYTES 16
#define RTA_PKT_MAX_BYTES 65536
#define RTA_PKT_SERVICE 200
#define RTA_PKT_SUBSERVICE 1

/* One segment of the stream directory: where its samples are and which pixels. */
typedef struct rta_segment_t {
    int64_t offset;      /* byte offset of the first sample in the stream */
    int32_t first_pixel; /* first pixel of the image it carries */
    int32_t n_pixels;    /* pixels it carries */
} rta_segment_t;

/* Why rta_ingest stopped (d_counts[4]); the byte offset of the packet is d_counts[5]. */
#define RTA_STREAM_OK 0
#define RTA_STREAM_FRAMING 1   /* no valid packet where the previous one ends, or bytes left over */
#define RTA_STREAM_HEADER 2    /* a fixed header field is wrong */
#define RTA_STREAM_CAMERA 3    /* unknown telescope, or pixels/samples differ from its camera */
#define RTA_STREAM_SEGMENT 4   /* segments out of order, overlapping or incomplete */
#define RTA_STREAM_CRC 5       /* packet error control mismatch (verify_crc) */
#define RTA_STREAM_CAPACITY 6  /* more segments, images or events than the capacities */

/* Decode a device-resident byte stream into a directory: segments (in stream
 * order), images (d_img_seg[i] = first segment of image i, n_img + 1 entries;
 * d_img_tel[i]) and events (d_evt_off: n_evt + 1 image offsets; event number
 * and event time in ns = seconds * 1e9 + floor(fine * 1e9 / 65536)). Nothing is
 * copied: rta_reconstruct_stream reads the samples where they are. Packets are
 * found in parallel: the stream is cut into 1 MiB pieces, each piece looks for
 * its first valid packet (a header whose fixed fields hold and whose successor
 * also starts a valid header) and walks from there; the walks must join up.
 * verify_crc != 0 also checks every packet's CRC (reads every byte once).
 * Capacities: d_seg seg_cap entries, d_img_seg img_cap + 1, d_img_tel img_cap,
 * d_evt_off evt_cap + 1, d_evt_number and d_evt_time_ns (may be NULL) evt_cap.
 * d_counts (6 int64, device): n_segments, n_img, n_evt, n_samples, error code
 * (RTA_STREAM_*), byte offset of the first bad packet (-1). On an error the
 * directory is incomplete and RTA_DEV_BAD_STREAM is set in the status word.
 * The stream must be 16-byte aligned. Asynchronous on stream; grows the
 * context's workspace (an allocation) when a stream is larger than any before. */
int rta_ingest(rta_ctx* ctx, const uint8_t* d_stream, int64_t n_bytes, int verify_crc, rta_segment_t* d_seg,
               int64_t seg_cap, int32_t* d_img_seg, int32_t* d_img_tel, int64_t img_cap, int32_t* d_evt_off,
               uint64_t* d_evt_number, int64_t* d_evt_time_ns, int64_t evt_cap, int64_t* d_counts, void* stream);

/* rta_reconstruct over an ingested stream, zero copy: the image kernel's bulk
 * copies read each chunk of pixels from the segment(s) that hold it. Counts are
 * read on the device (d_counts from rta_ingest: [1] images, [2] events), at
 * most max_img and max_evt; d_seg holds max_seg entries, d_img_seg max_img + 1.
 * An image whose segments do not tile its pixels with 16-byte-aligned runs
 * inside the stream is skipped (RTA_HF_BAD_INPUT). Stream-ordered, no host sync.
 * d_hillas: max_img rows, d_stereo: max_evt rows. Grows the context's
 * per-image workspace (an allocation) when max_img is larger than any before. */
int rta_reconstruct_stream(rta_ctx* ctx, const uint8_t* d_stream, int64_t n_bytes, const rta_segment_t* d_seg,
                           int64_t max_seg, const int32_t* d_img_seg, const int32_t* d_img_tel, int64_t max_img,
                           const int32_t* d_evt_off, int64_t max_evt, const int64_t* d_counts, int window_mode,
                           int start, int W, float t_hi, float t_lo, int core_needs_neighbour,
                           rta_hillas_t* d_hillas, rta_stereo_t* d_stereo, void* stream);

/* The autotuner of the byte-stream path: runs the image kernel of
 * rta_reconstruct_stream (the per-image records included; no stereo) on an
 * ingested stream for every configuration that fits (variant x 2..6 stages x
 * 1..4 CTAs/SM), `reps` timed launches each, and keeps the fastest as the
 * stream path's own configuration (its producer copies chunks from packet
 * segments, so its best pipeline depth can differ from the contiguous
 * bundle's). Arguments as rta_reconstruct_stream; d_hillas (max_img rows)
 * receives the configuration-independent rows. Every measurement goes to
 * h_entries (up to max_entries; *n_entries = number measured). The
 * neighbour-peak window is tuned for bundles and streams alike by rta_autotune:
 * RTA_WINDOW_NEIGHBOUR returns RTA_E_INVALID here. On a failed launch the
 * previous configuration stays. Synchronises `stream`; may grow the context's
 * per-image workspace (an allocation). */
int rta_autotune_stream(rta_ctx* ctx, const uint8_t* d_stream, int64_t n_bytes, const rta_segment_t* d_seg,
                        int64_t max_seg, const int32_t* d_img_seg, const int32_t* d_img_tel, int64_t max_img,
                        const int64_t* d_counts, int window_mode, int start, int W, float t_hi, float t_lo,
                        int core_needs_neighbour, rta_hillas_t* d_hillas, int reps, rta_tune_entry_t* h_entries,
                        int max_entries, int* n_entries, void* stream);

/* ---------------------------------------------------------------------- */
/* Lookup tables: the calibration matrices of the real-time reconstruction  */
/* (Sec. 4.1: energy and gamma/hadron separation), a non-learned second     */
/* path beside the surrogate                                               */
/* ---------------------------------------------------------------------- */
/* A table has RTA_MAX_CAMS * n_size * n_dist cells in device memory, cell
 * (camera id * n_size + size bin) * n_dist + distance bin. Size bin i holds
 * size_edges[i] <= size < size_edges[i + 1] (photoelectrons); distance bin j
 * holds dist_edges[j] <= R < dist_edges[j + 1], R the ground distance (m) from
 * the telescope to the shower core, sqrt(dx * dx + dy * dy) in FP32 with one
 * rounding per operation. Both decisions are FP32 comparisons. Edge arrays
 * (n + 1 floats, device memory, 1 <= n <= RTA_LUT_MAX_BINS) must increase
 * strictly; unsorted edges give unspecified bins but no access outside the
 * table. An image counts when its telescope id exists, it has >= 3 cleaned
 * pixels and is neither RTA_HF_EMPTY nor RTA_HF_BAD_INPUT (the stereo rule). */
#define RTA_MAX_CAMS 16
#define RTA_LUT_MAX_BINS 64
typedef struct rta_lut_cell_t {
    int32_t n;             /* training images that fell in the cell */
    float mean_w, sigma_w; /* image width (deg): mean and population standard deviation */
    float mean_l, sigma_l; /* image length (deg) */
    float mean_e, sigma_e; /* log10(E / TeV) */
    float reserved;
} rta_lut_cell_t;          /* a cell is used when n >= 1 and all three sigmas are > 0 */

typedef struct rta_lut_event_t {
    float log_energy;       /* sum(mean_e / sigma_e^2) / sum(1 / sigma_e^2) over the used images */
    float sigma_log_energy; /* sqrt(1 / sum(1 / sigma_e^2)) */
    float mscw, mscl;       /* means over the used images of (width - mean_w) / sigma_w, likewise length */
    int32_t n_used;         /* images in a used cell (-1: malformed image range) */
    uint32_t flags;         /* RTA_LF_* */
    float reserved[2];
} rta_lut_event_t;
#define RTA_LF_GAMMA 1u     /* mscw and mscl inside the cut box (inclusive) */
#define RTA_LF_NO_CORE 2u   /* the stereo row is RTA_SF_INVALID: no impact distances, fields 0 */
#define RTA_LF_NO_IMAGE 4u  /* no image fell in a used cell: fields 0 */
#define RTA_LF_MALFORMED 8u /* the image range is outside [0, n_img]; also sets a device status bit */

/* Training sums for the tables. d_acc: RTA_MAX_CAMS * n_size * n_dist rows of
 * 8 doubles (count, sum w, sum w^2, sum l, sum l^2, sum e, sum e^2, unused),
 * zeroed by the caller; this call adds to them, so several batches accumulate.
 * The distance is taken from the TRUE impact point. d_log_energy[n_evt]: true
 * log10(E / TeV); d_core_xy[2 n_evt]: true impact point (m); d_use[n_evt]:
 * events to take (gamma showers), NULL = all. Events with a malformed image
 * range are skipped. FP64 atomic sums: the order of additions varies between
 * runs, the sums by a few units in their last place. Asynchronous on stream.
 * Alignment (RTA_E_ALIGN otherwise): d_hillas, d_stereo, d_cells, d_lookup and
 * d_out on 16 bytes, d_acc on 8. RTA_E_INVALID for NULL pointers or bin counts outside
 * 1..RTA_LUT_MAX_BINS. */
int rta_lut_accumulate(rta_ctx* ctx, const rta_hillas_t* d_hillas, const int32_t* d_img_tel, int64_t n_img,
                       const int32_t* d_evt_off, int64_t n_evt, const float* d_log_energy, const float* d_core_xy,
                       const uint8_t* d_use, const float* d_size_edges, int n_size, const float* d_dist_edges,
                       int n_dist, double* d_acc, void* stream);
/* Cells from the sums: mean = S / n, sigma = sqrt(max(S2 / n - mean^2, 0)) in
 * FP64, rounded once to FP32; cells with n < min_count (min_count >= 1) keep n
 * and are zero elsewhere, i.e. unused. n_cells = RTA_MAX_CAMS * n_size * n_dist. */
int rta_lut_finalize(rta_ctx* ctx, const double* d_acc, int64_t n_cells, int min_count, rta_lut_cell_t* d_cells,
                     void* stream);
/* The lookup form of a table, made once per table: per cell, in FP64 with one
 * rounding per operation, 1 / sigma_w, 1 / sigma_l, the energy weight
 * w_e = 1 / (sigma_e * sigma_e) and w_e * mean_e, and the FP32 means; unused
 * cells get zeros. d_lookup: n_cells * RTA_LUT_LOOKUP_BYTES bytes, 16-byte
 * aligned, device memory; its layout is private to the library. */
#define RTA_LUT_LOOKUP_BYTES 64
int rta_lut_prepare(rta_ctx* ctx, const rta_lut_cell_t* d_cells, int64_t n_cells, void* d_lookup, void* stream);
/* Energy and scaled width and length of each event from a table in lookup
 * form and the event's stereo row (the reconstructed core gives the
 * distances). Per used image: (w - mean_w) * (1 / sigma_w), likewise the
 * length, the weight w_e and w_e * mean_e, in FP64 with one rounding per
 * operation; the four are summed in image order and divided once per event
 * (the order and the roundings are fixed, so results are reproducible bit for
 * bit). Gamma-like (RTA_LF_GAMMA): mscw_lo <= mscw <= mscw_hi and
 * mscl_lo <= mscl <= mscl_hi, compared in FP64. d_out: n_evt rows.
 * Asynchronous on stream. */
int rta_lut_reconstruct(rta_ctx* ctx, const rta_hillas_t* d_hillas, const int32_t* d_img_tel, int64_t n_img,
                        const int32_t* d_evt_off, int64_t n_evt, const rta_stereo_t* d_stereo,
                        const void* d_lookup, const float* d_size_edges, int n_size,
                        const float* d_dist_edges, int n_dist, float mscw_lo, float mscw_hi, float mscl_lo,
                        float mscl_hi, rta_lut_event_t* d_out, void* stream);

/* ---------------------------------------------------------------------- */
/* Serving: a stream of bundles with continuous batching, and the sky map   */
/* (Sec. 4.2 event-by-event RTA; Sec. 2.1 30 s alert latency and           */
/* transient search on several timescales)                                 */
/* ---------------------------------------------------------------------- */
#define RTA_SKY_N 256      /* sky-map bins per axis, 0.02 deg each, [-2.56, 2.56) deg */
#define RTA_SKY_SLABS 30   /* one-second slabs; a map is the sum of the last 30 */
#define RTA_SKY_MIN_SLABS 60   /* one-minute slabs: windows up to one hour */
#define RTA_MAX_DISK_RADIUS 32 /* largest on-region radius of the transient search, in bins */

/* One bundle of events in HOST memory (pinned memory gives full copy speed).
 * Layout as the device calls (offsets from h_wave, CSR from 0). Every buffer
 * must stay valid until rta_stream_poll reports the bundle done; h_events
 * (n_evt rows) then holds its event list. */
typedef struct rta_bundle_t {
    const uint16_t* h_wave;
    int64_t n_wave;
    const int64_t* h_wave_off;
    const int32_t* h_img_tel;
    int64_t n_img;
    const int32_t* h_evt_off;
    int64_t n_evt;
    int64_t arrival_ns;      /* steady clock (CLOCK_MONOTONIC) nanoseconds of arrival */
    rta_event_t* h_events;   /* out */
} rta_bundle_t;

typedef struct rta_stream rta_stream;

/* Create the serving engine. hbm_budget_bytes is allocated once and
 * sub-allocated per bundle (its waveforms and tables): a bundle is admitted,
 * in arrival order, when one of max_inflight copy slots (CUDA streams) is free
 * and the budget has room; its slot's stream copies it in and then publishes
 * its descriptor into a queue held in device memory. Reconstruction runs as
 * passes on one compute stream, each of which takes on the device every bundle
 * published and not yet taken (up to twice max_img images and twice max_evt
 * events), and runs once over all of them: rta_image_chain, then
 * rta_surrogate_infer with the given model (events with a learned direction,
 * geometric fallback) or, with model = NULL, rta_stereo (geometric direction,
 * no energy or gammaness); each bundle's event rows go straight into its
 * slot's mapped host staging, and its events into the sky-map slabs of its
 * arrival (slab ownership is kept on the device). Bundles published while a
 * pass runs are taken by the next one: copies of arriving bundles overlap the
 * reconstruction of earlier ones. max_img / max_evt bound one bundle (at most
 * 2^29). A scheduler thread owned by the stream issues the copies and the
 * passes. Each slot keeps a pinned, mapped host staging buffer of
 * max(12 max_img + 4 (max_evt + 1), 32 max_evt) bytes for the bundle's tables
 * and its event list, so that only h_wave needs to be pinned for the copies to
 * run asynchronously. A bundle's event rows do not depend on the bundles that
 * share its pass. */
int rta_stream_create(rta_ctx* ctx, rta_model* model, size_t hbm_budget_bytes, int max_inflight, int64_t max_img,
                      int64_t max_evt, int window_mode, int start, int W, float t_hi, float t_lo,
                      int core_needs_neighbour, float fallback_deg, rta_stream** out);
/* Queue a bundle; returns at once with its ticket. RTA_E_NOMEM if it can never
 * fit the budget, RTA_E_BUSY if 4096 bundles are already waiting, RTA_E_INVALID
 * or RTA_E_ALIGN if an image lies outside h_wave, has an offset that is not a
 * multiple of 8 samples, or names an unregistered telescope. */
int rta_stream_submit(rta_stream* stream, const rta_bundle_t* bundle, uint64_t* ticket);
/* Non-blocking: RTA_OK once the bundle's event list is in host memory (its
 * completion time in *done_ns, same clock as arrival_ns; the ticket is then
 * released), RTA_E_BUSY while it is queued or running. */
int rta_stream_poll(rta_stream* stream, uint64_t ticket, int64_t* done_ns);
/* Where a bundle's time went: host steady-clock instants (ns, the clock of
 * arrival_ns) of its arrival, submission, admission to a copy slot and
 * completion; device durations from timing events: the copies in (waveforms
 * and tables, on its slot's stream), the wait of its published data for the
 * pass that took it, that pass's device work (image kernel and learned or
 * geometric reconstruction over the whole batch) and the pass's output (event
 * rows to host memory and the sky-map fill); and the number of bundles in its
 * pass. The host queue wait is admit_ns - arrival_ns. */
typedef struct rta_bundle_times_t {
    int64_t arrival_ns, submit_ns, admit_ns, done_ns;
    float h2d_ms, compute_ms, d2h_ms;
    int32_t slot;
    float ready_wait_ms;
    int32_t batch_bundles;
} rta_bundle_times_t;
/* rta_stream_poll that also returns the bundle's times (times may be NULL). */
int rta_stream_poll_times(rta_stream* stream, uint64_t ticket, int64_t* done_ns, rta_bundle_times_t* times);
/* Wait until every submitted bundle has finished (RTA_E_TIMEOUT after timeout_ms). */
int rta_stream_drain(rta_stream* stream, int timeout_ms);
/* The sky-count map at time now_ns: per bin (row y, column x, RTA_SKY_N each)
 * the events of the slabs of the last 30 seconds, into h_map. Bin of a
 * direction: floor((v + 2.56f) * 50.0f) in FP32 (round to nearest, no
 * contraction), kept when in [0, 256); events without direction are not
 * counted. Synchronises the map's stream. */
int rta_skymap_read(rta_stream* stream, int64_t now_ns, uint32_t* h_map);
/* Count externally reconstructed events (device rows) into the sky map as if
 * they had arrived at arrival_ns; ordered after the work already queued on
 * `stream` and before later work on it that reuses d_events. */
int rta_stream_add_events(rta_stream* stream, const rta_event_t* d_events, int64_t n_evt, int64_t arrival_ns,
                          void* cuda_stream);
int rta_stream_destroy(rta_stream* stream);

/* ---------------------------------------------------------------------- */
/* Transient search on the sky map (Sec. 2.1 requirement (ii): multiple    */
/* timescales from seconds to hours, in a source region and elsewhere in   */
/* the field of view)                                                      */
/* ---------------------------------------------------------------------- */

/* One timescale: an "on" window of on_s seconds ending at the search time and
 * the "off" (background) window of off_s seconds just before it, in whole
 * seconds of bundle arrival: with now_s = now_ns / 1e9 (integer division), on
 * covers the seconds (now_s - on_s, now_s] and off (now_s - on_s - off_s,
 * now_s - on_s]. Either on_s + off_s <= RTA_SKY_SLABS (read from the one-second
 * slabs), or both are multiples of 60 and on_s + off_s <= 60 * RTA_SKY_MIN_SLABS
 * (read from the one-minute slabs; minute of a second: floor(s / 60)). The
 * stream fills both rings as it bins events. */
typedef struct rta_window_t {
    int32_t on_s, off_s;
} rta_window_t;

/* One alert: a (window, bin) whose significance reached the threshold. n_on and
 * n_off are the event counts in the disk of radius_bins around the bin (bins
 * with (dx^2 + dy^2) <= radius^2, clipped at the map edge) in the on and off
 * windows; alpha = on_s / off_s; significance = Li & Ma (1983) Eq. 17, signed
 * (negative for a deficit, n_on < alpha * n_off), computed in FP64. 48 bytes. */
typedef struct rta_alert_t {
    int32_t window; /* index into the windows array */
    int32_t ix, iy; /* bin column and row */
    int32_t pad;
    int64_t n_on, n_off;
    double alpha, significance;
} rta_alert_t;

/* Transient search over every bin of the sky map for each of n_windows windows:
 * writes the alerts with significance >= s_min, sorted by (window, iy, ix), to
 * h_alerts (at most max_alerts; *n_alerts gets the number found, which may be
 * larger). radius_bins in 0..RTA_MAX_DISK_RADIUS (0: single bins). Errors:
 * RTA_E_INVALID for a window outside the rules above or a bad radius.
 * Synchronises the map's stream. */
int rta_transient_search(rta_stream* stream, int64_t now_ns, const rta_window_t* windows, int n_windows,
                         int radius_bins, double s_min, rta_alert_t* h_alerts, int max_alerts, int* n_alerts);

/* The full significance map of one window: h_sig (RTA_SKY_N x RTA_SKY_N
 * doubles, row y then column x) and, when not NULL, the disk counts h_on and
 * h_off (int64). Same definitions as rta_transient_search. */
int rta_significance_map(rta_stream* stream, int64_t now_ns, rta_window_t window, int radius_bins, double* h_sig,
                         int64_t* h_on, int64_t* h_off);

/* ---------------------------------------------------------------------- */
/* Entry point that allocates nothing                                      */
/* ---------------------------------------------------------------------- */
/* The paper has no counterpart of this call; it exists for callers that may
 * not allocate device memory: real-time processes that must not stall
 * (cudaMalloc and cudaFree can synchronise the whole device), frameworks that
 * own all device memory through their own pool, and code running where new
 * allocations are not allowed. Such callers cannot use an rta_ctx, because
 * creating and filling one allocates. */

#define RTA_NOALLOC_MAX_CAMS 16   /* camera descriptors per call */
#define RTA_NOALLOC_MAX_TEL 1024  /* telescopes per call */

/* One camera type, tables in caller-owned device memory. */
typedef struct rta_camera_desc_t {
    int n_pix, n_samples, K;  /* as rta_register_camera; n_pix*n_samples a multiple of 8 */
    const float* d_pix_xy;    /* 2*n_pix floats (deg), 8-byte aligned */
    const int16_t* d_nb8;     /* n_pix rows of 8 int16 neighbour ids, 16-byte aligned: the first K
                                 of row p are ids in [0, n_pix) other than p, or -1 for none;
                                 an id outside [0, n_pix) counts as -1 (it is not validated
                                 here, unlike rta_register_camera, and is never read) */
} rta_camera_desc_t;

/* rta_image_chain without a context and without any allocation: the same
 * fused kernel (calibrate + integrate + clean + Hillas, same definitions and
 * same rows) on the current device, in its default launch configuration.
 * The caller passes every buffer:
 *   h_cams[n_cams]          camera descriptors; telescopes refer to them by index;
 *   h_tel_cam[n_tel]        camera index of each telescope (host);
 *   h_tel_row[n_tel]        first calibration row of each telescope (host): a
 *                           multiple of 8, with at least 8 rows after its last
 *                           pixel inside the n_calib_rows of d_p16 / d_scale;
 *   d_p16, d_scale          the calibration table (as rta_register_array),
 *                           16-byte aligned;
 *   d_wave ... d_out        the bundle and the Hillas rows, as rta_image_chain;
 *   d_status                optional (NULL = none): receives the device status
 *                           word (RTA_DEV_* bits) when the kernel has finished.
 * Limits: n_cams <= RTA_NOALLOC_MAX_CAMS and n_tel <= RTA_NOALLOC_MAX_TEL;
 * larger values return RTA_E_INVALID before anything is launched.
 * Scratch: the per-call tables, the work counter and the status word live in a
 * fixed ~13 KiB file-scope __device__ array that every GPU which loads this
 * library keeps until the process exits. All calls share it and it keeps the
 * last call's contents (each call resets what must start at zero), so calls
 * whose work overlaps on the GPU (other streams, other host threads) race and
 * must be serialised by the caller. The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current.
 * Not capturable: the tables travel by a copy from a stack buffer of this call,
 * so no call (the first or a later one) may be made while `stream` is being
 * captured into a graph (such a call returns RTA_E_INVALID and leaves the
 * capture as it was). This call makes no
 * cudaMalloc, cudaFree or other allocating call. Asynchronous on `stream`;
 * the host arrays (h_cams, h_tel_cam, h_tel_row) are consumed before it
 * returns, whatever memory they are in. */
int rta_image_chain_noalloc(const rta_camera_desc_t* h_cams, int n_cams, const int32_t* h_tel_cam,
                            const int64_t* h_tel_row, int n_tel, const int32_t* d_p16, const float* d_scale,
                            int64_t n_calib_rows, const uint16_t* d_wave, int64_t n_wave, const int64_t* d_wave_off,
                            const int32_t* d_img_tel, int64_t n_img, int window_mode, int start, int W, float t_hi,
                            float t_lo, int core_needs_neighbour, rta_hillas_t* d_out, uint32_t* d_status,
                            void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RTA_H */
