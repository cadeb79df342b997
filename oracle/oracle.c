/*
 * CPU ORACLE of the real-time reconstruction path -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct C. Only the tests, the package smoke check and
 * the benchmark's CPU-baseline leg may load this file; the product path never
 * does. It shares no code with the CUDA library.
 *
 * The paper (Bulgarelli et al., "The Real-Time Analysis of the CTA
 * Observatory", ICRC 2013) names the steps but prints no formula: the RT-RECO
 * pipeline turns DL0 waveforms into an event list through calibration with
 * the calibration matrices and energy/direction reconstruction (Sec. 4.1),
 * processed event by event (Sec. 4.2), with signal-extraction algorithms for
 * the charge (Sec. 5). The definitions written out here are the textbook ones
 * for imaging atmospheric Cherenkov telescopes, in the readings this project
 * fixes for the paper's silent points:
 *
 *   integrate  charge = (sum of W samples - W * pedestal) / (gain * window
 *              containment); fixed window, or the W-window of maximal integer
 *              sum with the lowest start on ties. The pedestal arrives in 1/16
 *              ADC fixed point (p16), so the numerator 16*sum - W*p16 is an
 *              exact integer and the calibration scale is 1/(16 gain f_W). The
 *              one floating-point step is a single FP32 multiply of that
 *              integer by the FP32 scale; it is done in FP32 here on purpose.
 *   nbpeak     the neighbour-peak window: a pixel integrates its own samples
 *              in the sliding window of the brightest pixel (largest charge,
 *              then earliest start) of its closed neighbourhood.
 *   clean      two-threshold tailcut: core pixels q >= t_hi (optionally with a
 *              neighbour also >= t_hi), boundary pixels q >= t_lo next to a core
 *              pixel; one pass.
 *   hillas     charge-weighted first and second moments of the cleaned image
 *              (Hillas 1985), two-pass in FP64, plus the charge-weighted
 *              least-squares slope of pixel time along the major axis.
 *   stereo     weighted intersection of the image major axes in the camera
 *              (direction) and, through the telescope positions, on the ground
 *              (core) -- the "Hillas intersection" method.
 *
 * Everything except the deliberate FP32 multiply is FP64.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Hillas output row (doubles), indices */
enum {
    OH_SIZE = 0, OH_X, OH_Y, OH_LENGTH, OH_WIDTH, OH_PSI, OH_R, OH_PHI, OH_TGRAD, OH_TMEAN, OH_NPIX, OH_FLAGS, OH_N
};
/* flags */
#define OF_EMPTY 1u    /* no pixel survived cleaning (or size <= 0) */
#define OF_NO_TIME 2u  /* fewer than two pixels, or no times: no time gradient */

/* stereo output row */
enum { OS_DIR_X = 0, OS_DIR_Y, OS_CORE_X, OS_CORE_Y, OS_NVALID, OS_FLAGS, OS_N };
#define OF_STEREO_INVALID 1u

/* ------------------------------------------------------------------ */
/* Calibration + charge integration (Sec. 4.1 calibration, Sec. 5      */
/* signal extraction)                                                   */
/* ------------------------------------------------------------------ */
/*
 * One image: wave[p*S + k]. Per pixel: window start s (fixed, or the first
 * maximising start of the W-sample sum), integer window sum, the exact integer
 * numerator num = 16*sum - W*p16, q = fp32(num) * scale in FP32, and the
 * pedestal-subtracted sample-index centroid of the window
 * t = s + sum_j j*(16*w[s+j] - p16) / num, or the window centre s + (W-1)/2
 * when num <= 0. Returns 0, or -1 if an argument is out of range.
 */
int or_integrate(const uint16_t* wave, int P, int S, const int32_t* p16, const float* scale, int sliding,
                 int start, int W, const int32_t* weights, float* q, double* t, int32_t* wstart, int64_t* wsum) {
    if (P < 0 || S <= 0 || W <= 0 || W > S) return -1;
    if (!sliding && (start < 0 || start + W > S)) return -1;
    for (int p = 0; p < P; ++p) {
        const uint16_t* w = wave + (size_t)p * S;
        int best_s = sliding ? 0 : start;
        int64_t best = -1;
        if (sliding) {
            for (int s = 0; s + W <= S; ++s) {
                int64_t sum = 0;
                for (int k = s; k < s + W; ++k) sum += w[k];
                if (sum > best) { best = sum; best_s = s; }
            }
        } else {
            best = 0;
            for (int k = start; k < start + W; ++k) best += w[k];
        }
        int64_t num = 16 * best - (int64_t)W * p16[p];
        /* digital-filter-style extractor: integer weights over the same window,
           pedestal weighted by their sum; one rounding to FP32, one multiply */
        int64_t qnum = num;
        if (weights) {
            int64_t a = 0, c = 0;
            for (int k = 0; k < W; ++k) {
                a += (int64_t)weights[k] * w[best_s + k];
                c += weights[k];
            }
            qnum = 16 * a - c * p16[p];
        }
        volatile float fnum = (float)qnum;
        volatile float qq = fnum * scale[p];
        q[p] = qq;
        if (t) {
            int64_t numt = 0;
            for (int j = 0; j < W; ++j) numt += (int64_t)j * (16 * (int64_t)w[best_s + j] - p16[p]);
            t[p] = num > 0 ? (double)best_s + (double)numt / (double)num : (double)best_s + 0.5 * (W - 1);
        }
        if (wstart) wstart[p] = best_s;
        if (wsum) wsum[p] = best;
    }
    return 0;
}

/*
 * Neighbour-peak window (an extractor of the Sec. 5 family; the paper names
 * the family, not a definition). Step 1: every pixel's own sliding window
 * (first maximal W-sum) and the charge q0 it gives, with the same FP32
 * multiply as above. Step 2: pixel p integrates its OWN samples in the window
 * of the brightest pixel of its closed neighbourhood {p} and nb[p*K + j]: the
 * largest q0, and among equal q0 the earliest window start. Charge and time
 * then follow the flat-window rules above at that start. wstart receives the
 * chosen start.
 */
int or_integrate_nbpeak(const uint16_t* wave, int P, int S, const int32_t* p16, const float* scale,
                        const int16_t* nb, int K, int W, float* q, double* t, int32_t* wstart) {
    if (P < 0 || S <= 0 || W <= 0 || W > S || K < 0) return -1;
    float* q0 = (float*)malloc(sizeof(float) * (size_t)(P + 1));
    int32_t* s0 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(P + 1));
    if (!q0 || !s0) { free(q0); free(s0); return -1; }
    /* step 1: the sliding window of every pixel */
    if (or_integrate(wave, P, S, p16, scale, 1, 0, W, NULL, q0, NULL, s0, NULL) != 0) {
        free(q0); free(s0); return -1;
    }
    /* step 2: the window of the brightest pixel in the closed neighbourhood */
    for (int p = 0; p < P; ++p) {
        int b = p;
        for (int j = 0; j < K; ++j) {
            int n = nb[(size_t)p * K + j];
            if (n < 0 || n >= P) continue;
            if (q0[n] > q0[b] || (q0[n] == q0[b] && s0[n] < s0[b])) b = n;
        }
        const int st = s0[b];
        const uint16_t* w = wave + (size_t)p * S;
        int64_t sum = 0;
        for (int k = st; k < st + W; ++k) sum += w[k];
        int64_t num = 16 * sum - (int64_t)W * p16[p];
        volatile float fnum = (float)num;
        volatile float qq = fnum * scale[p];
        q[p] = qq;
        if (t) {
            int64_t numt = 0;
            for (int j = 0; j < W; ++j) numt += (int64_t)j * (16 * (int64_t)w[st + j] - p16[p]);
            t[p] = num > 0 ? (double)st + (double)numt / (double)num : (double)st + 0.5 * (W - 1);
        }
        if (wstart) wstart[p] = st;
    }
    free(q0); free(s0);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Tailcut cleaning                                                     */
/* ------------------------------------------------------------------ */
/*
 * nb[p*K + j] lists the neighbours of pixel p (-1 = none).
 *   above[p]   = q[p] >= t_hi
 *   core[p]    = above[p] and (not core_needs_neighbour or some neighbour is above)
 *   boundary[p]= q[p] >= t_lo and some neighbour is core
 *   mask       = core or boundary
 */
void or_clean(int P, const float* q, const int16_t* nb, int K, float t_hi, float t_lo, int core_needs_neighbour,
              uint8_t* mask) {
    uint8_t* above = (uint8_t*)calloc((size_t)P + 1, 1);
    uint8_t* core = (uint8_t*)calloc((size_t)P + 1, 1);
    for (int p = 0; p < P; ++p) above[p] = q[p] >= t_hi;
    for (int p = 0; p < P; ++p) {
        int c = above[p];
        if (c && core_needs_neighbour) {
            int any = 0;
            for (int j = 0; j < K; ++j) {
                int n = nb[(size_t)p * K + j];
                if (n >= 0 && above[n]) any = 1;
            }
            c = any;
        }
        core[p] = (uint8_t)c;
    }
    for (int p = 0; p < P; ++p) {
        int b = 0;
        if (q[p] >= t_lo)
            for (int j = 0; j < K; ++j) {
                int n = nb[(size_t)p * K + j];
                if (n >= 0 && core[n]) b = 1;
            }
        mask[p] = (uint8_t)(core[p] || b);
    }
    free(above);
    free(core);
}

/* ------------------------------------------------------------------ */
/* Hillas moments + time gradient (direction reconstruction, Sec. 4.1) */
/* ------------------------------------------------------------------ */
/*
 * Over pixels with mask[p] != 0, weights q[p], positions xy[2p], xy[2p+1]:
 *   size = sum q;  centroid (x, y) = sum q xy / size
 *   sxx, syy, sxy = sum q dx dx / size, ... with dx = x_p - x (second pass)
 *   lambda1 = (sxx+syy)/2 + sqrt(((sxx-syy)/2)^2 + sxy^2)
 *   length = sqrt(lambda1), width = sqrt(max(det,0)/lambda1), det = sxx syy - sxy^2
 *   psi = atan2(2 sxy, sxx - syy) / 2 in (-pi/2, pi/2]
 *   r = |centroid|, phi = atan2(y, x)
 *   tmean = sum q t / size; time gradient = sum q l (t - tmean) / sum q l^2,
 *   l = dx cos psi + dy sin psi (third pass), when n_pix >= 2.
 * t may be NULL (no time gradient). out has OH_N entries.
 */
void or_hillas(int P, const float* xy, const float* q, const double* t, const uint8_t* mask, double* out) {
    for (int i = 0; i < OH_N; ++i) out[i] = 0.0;
    double size = 0.0, sx = 0.0, sy = 0.0;
    int n = 0;
    for (int p = 0; p < P; ++p) {
        if (!mask[p]) continue;
        double w = q[p];
        size += w;
        sx += w * (double)xy[2 * p];
        sy += w * (double)xy[2 * p + 1];
        ++n;
    }
    out[OH_NPIX] = n;
    if (n == 0 || !(size > 0.0)) {
        out[OH_FLAGS] = OF_EMPTY | OF_NO_TIME;
        return;
    }
    double cx = sx / size, cy = sy / size;
    double sxx = 0.0, syy = 0.0, sxy = 0.0, st = 0.0;
    for (int p = 0; p < P; ++p) {
        if (!mask[p]) continue;
        double w = q[p], dx = (double)xy[2 * p] - cx, dy = (double)xy[2 * p + 1] - cy;
        sxx += w * dx * dx;
        syy += w * dy * dy;
        sxy += w * dx * dy;
        if (t) st += w * t[p];
    }
    sxx /= size; syy /= size; sxy /= size;
    double half_d = 0.5 * (sxx - syy);
    double lam1 = 0.5 * (sxx + syy) + sqrt(half_d * half_d + sxy * sxy);
    double det = sxx * syy - sxy * sxy;
    double length = lam1 > 0.0 ? sqrt(lam1) : 0.0;
    double width = lam1 > 0.0 ? sqrt((det > 0.0 ? det : 0.0) / lam1) : 0.0;
    double psi = 0.5 * atan2(2.0 * sxy, sxx - syy);
    out[OH_SIZE] = size;
    out[OH_X] = cx;
    out[OH_Y] = cy;
    out[OH_LENGTH] = length;
    out[OH_WIDTH] = width;
    out[OH_PSI] = psi;
    out[OH_R] = sqrt(cx * cx + cy * cy);
    out[OH_PHI] = atan2(cy, cx);
    unsigned flags = 0;
    if (t && n >= 2) {
        double tmean = st / size, cp = cos(psi), sp = sin(psi);
        double sll = 0.0, slt = 0.0;
        for (int p = 0; p < P; ++p) {
            if (!mask[p]) continue;
            double w = q[p], dx = (double)xy[2 * p] - cx, dy = (double)xy[2 * p + 1] - cy;
            double l = dx * cp + dy * sp;
            sll += w * l * l;
            slt += w * l * (t[p] - tmean);
        }
        out[OH_TMEAN] = tmean;
        out[OH_TGRAD] = sll > 0.0 ? slt / sll : 0.0;
    } else {
        if (t) out[OH_TMEAN] = st / size;
        flags |= OF_NO_TIME;
    }
    out[OH_FLAGS] = flags;
}

/* ------------------------------------------------------------------ */
/* Stereo Hillas intersection (direction + core, Sec. 4.1)              */
/* ------------------------------------------------------------------ */
/*
 * m images of one event: hillas rows h[i*OH_N ...], telescope positions txy[2i]
 * (metres). An image is used when it has at least 3 pixels. For every used
 * pair (i < j) with |sin(psi_j - psi_i)| >= 1e-6:
 *   u = (cos psi, sin psi)
 *   direction: p_ij = c_i + u_i * cross(c_j - c_i, u_j) / sin(psi_j - psi_i)
 *   core:      g_ij = T_i + u_i * cross(T_j - T_i, u_j) / sin(psi_j - psi_i)
 *   weight     w_ij = |sin(psi_i - psi_j)| * s_i s_j / (s_i + s_j)
 *                     * (1 - W_i/L_i) * (1 - W_j/L_j)
 * result = sum w p / sum w. With no usable pair (or zero total weight) the
 * event is flagged invalid and zeros are returned.
 */
void or_stereo(int m, const double* h, const double* txy, double* out) {
    for (int i = 0; i < OS_N; ++i) out[i] = 0.0;
    int nvalid = 0;
    for (int i = 0; i < m; ++i) nvalid += h[i * OH_N + OH_NPIX] >= 3.0;
    out[OS_NVALID] = nvalid;
    double sw = 0.0, swx = 0.0, swy = 0.0, swgx = 0.0, swgy = 0.0;
    int npair = 0;
    for (int i = 0; i < m; ++i) {
        const double* a = h + i * OH_N;
        if (a[OH_NPIX] < 3.0) continue;
        for (int j = i + 1; j < m; ++j) {
            const double* b = h + j * OH_N;
            if (b[OH_NPIX] < 3.0) continue;
            double s = sin(b[OH_PSI] - a[OH_PSI]);
            if (fabs(s) < 1e-6) continue;
            double uax = cos(a[OH_PSI]), uay = sin(a[OH_PSI]);
            double ubx = cos(b[OH_PSI]), uby = sin(b[OH_PSI]);
            double dx = b[OH_X] - a[OH_X], dy = b[OH_Y] - a[OH_Y];
            double k = (dx * uby - dy * ubx) / s;
            double px = a[OH_X] + k * uax, py = a[OH_Y] + k * uay;
            double gx0 = txy[2 * j] - txy[2 * i], gy0 = txy[2 * j + 1] - txy[2 * i + 1];
            double kg = (gx0 * uby - gy0 * ubx) / s;
            double gx = txy[2 * i] + kg * uax, gy = txy[2 * i + 1] + kg * uay;
            double w = fabs(s) * a[OH_SIZE] * b[OH_SIZE] / (a[OH_SIZE] + b[OH_SIZE]) *
                       (1.0 - a[OH_WIDTH] / a[OH_LENGTH]) * (1.0 - b[OH_WIDTH] / b[OH_LENGTH]);
            sw += w;
            swx += w * px; swy += w * py;
            swgx += w * gx; swgy += w * gy;
            ++npair;
        }
    }
    if (npair == 0 || !(sw > 0.0)) {
        out[OS_FLAGS] = OF_STEREO_INVALID;
        return;
    }
    out[OS_DIR_X] = swx / sw;
    out[OS_DIR_Y] = swy / sw;
    out[OS_CORE_X] = swgx / sw;
    out[OS_CORE_Y] = swgy / sw;
}

/* ------------------------------------------------------------------ */
/* Whole-bundle driver (threads over images, then over events)         */
/* ------------------------------------------------------------------ */
typedef struct {
    /* bundle */
    int64_t n_img;
    const uint16_t* wave;
    const int64_t* wave_off;
    const int32_t* img_tel;
    const int32_t* tel_cam;
    const int64_t* tel_pix_off;
    const int32_t* p16;
    const float* scale;
    const int32_t* cam_info;        /* per cam id: P, S, K */
    const float* const* cam_xy;
    const int16_t* const* cam_nb;
    int sliding, start, W, core_nb;
    const int32_t* weights;   /* NULL: flat window sum */
    int nbpeak;               /* 1: neighbour-peak window (sliding ignored) */
    float t_hi, t_lo;
    /* outputs */
    double* hillas;                 /* n_img * OH_N */
    const int64_t* pix_off;         /* optional per-pixel outputs */
    float* q_out;
    double* t_out;
    uint8_t* mask_out;
    /* stereo */
    int64_t n_evt;
    const int32_t* evt_off;
    const float* tel_xy;
    double* stereo;                 /* n_evt * OS_N, may be NULL */
    int64_t next_img, next_evt;
    int status;
} bundle_job_t;

static void* bundle_worker(void* arg) {
    bundle_job_t* J = (bundle_job_t*)arg;
    int maxP = 0;
    for (int c = 0; c < 16; ++c)
        if (J->cam_info[3 * c] > maxP) maxP = J->cam_info[3 * c];
    float* q = (float*)malloc(sizeof(float) * (size_t)(maxP + 1));
    double* t = (double*)malloc(sizeof(double) * (size_t)(maxP + 1));
    uint8_t* mk = (uint8_t*)malloc((size_t)maxP + 1);
    for (;;) {
        int64_t i = __atomic_fetch_add(&J->next_img, 1, __ATOMIC_RELAXED);
        if (i >= J->n_img) break;
        int tel = J->img_tel[i], cam = J->tel_cam[tel];
        int P = J->cam_info[3 * cam], S = J->cam_info[3 * cam + 1], K = J->cam_info[3 * cam + 2];
        int64_t row = J->tel_pix_off[tel];
        const int rc = J->nbpeak
            ? or_integrate_nbpeak(J->wave + J->wave_off[i], P, S, J->p16 + row, J->scale + row, J->cam_nb[cam], K,
                                  J->W, q, t, NULL)
            : or_integrate(J->wave + J->wave_off[i], P, S, J->p16 + row, J->scale + row, J->sliding, J->start, J->W,
                           J->weights, q, t, NULL, NULL);
        if (rc != 0) {
            J->status = -1;
            continue;
        }
        or_clean(P, q, J->cam_nb[cam], K, J->t_hi, J->t_lo, J->core_nb, mk);
        or_hillas(P, J->cam_xy[cam], q, t, mk, J->hillas + i * OH_N);
        if (J->pix_off) {
            int64_t o = J->pix_off[i];
            if (J->q_out) memcpy(J->q_out + o, q, sizeof(float) * (size_t)P);
            if (J->t_out) memcpy(J->t_out + o, t, sizeof(double) * (size_t)P);
            if (J->mask_out) memcpy(J->mask_out + o, mk, (size_t)P);
        }
    }
    free(q); free(t); free(mk);
    return NULL;
}

static void* stereo_worker(void* arg) {
    bundle_job_t* J = (bundle_job_t*)arg;
    double txy[2 * 64];
    for (;;) {
        int64_t e = __atomic_fetch_add(&J->next_evt, 1, __ATOMIC_RELAXED);
        if (e >= J->n_evt) break;
        int a = J->evt_off[e], b = J->evt_off[e + 1], m = b - a;
        if (m > 64) m = 64;
        for (int k = 0; k < m; ++k) {
            int tel = J->img_tel[a + k];
            txy[2 * k] = J->tel_xy[2 * tel];
            txy[2 * k + 1] = J->tel_xy[2 * tel + 1];
        }
        or_stereo(m, J->hillas + (int64_t)a * OH_N, txy, J->stereo + e * OS_N);
    }
    return NULL;
}

static void run_threads(void* (*fn)(void*), void* arg, int n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 512) n_threads = 512;
    pthread_t th[512];
    int started = 0;
    for (int i = 1; i < n_threads; ++i)
        if (pthread_create(&th[started], NULL, fn, arg) == 0) ++started;
    fn(arg);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
}

/*
 * Full chain over a bundle: integrate -> clean -> hillas for every image, then
 * stereo for every event (if stereo != NULL). cam_info[3*cam] = (P, S, K) for
 * cam ids 0..15 (unused ids zero). Returns 0, or -1 on a bad image.
 */
int or_reconstruct(int64_t n_img, const uint16_t* wave, const int64_t* wave_off, const int32_t* img_tel,
                   const int32_t* tel_cam, const int64_t* tel_pix_off, const int32_t* p16, const float* scale,
                   const int32_t* cam_info, const float* const* cam_xy, const int16_t* const* cam_nb, int sliding,
                   int start, int W, float t_hi, float t_lo, int core_nb, double* hillas, const int64_t* pix_off,
                   float* q_out, double* t_out, uint8_t* mask_out, int64_t n_evt, const int32_t* evt_off,
                   const float* tel_xy, double* stereo, int n_threads, const int32_t* weights, int nbpeak) {
    bundle_job_t J;
    memset(&J, 0, sizeof J);
    J.n_img = n_img; J.wave = wave; J.wave_off = wave_off; J.img_tel = img_tel; J.tel_cam = tel_cam;
    J.tel_pix_off = tel_pix_off; J.p16 = p16; J.scale = scale; J.cam_info = cam_info; J.cam_xy = cam_xy;
    J.cam_nb = cam_nb; J.sliding = sliding; J.start = start; J.W = W; J.weights = weights; J.core_nb = core_nb;
    J.nbpeak = nbpeak;
    J.t_hi = t_hi;
    J.t_lo = t_lo; J.hillas = hillas; J.pix_off = pix_off; J.q_out = q_out; J.t_out = t_out;
    J.mask_out = mask_out; J.n_evt = n_evt; J.evt_off = evt_off; J.tel_xy = tel_xy; J.stereo = stereo;
    run_threads(bundle_worker, &J, n_threads);
    if (stereo && n_evt > 0) run_threads(stereo_worker, &J, n_threads);
    return J.status;
}

/* ------------------------------------------------------------------ */
/* CRC of the DL0 packets (Sec. 5: telemetry-formatted byte stream)     */
/* ------------------------------------------------------------------ */
/*
 * CRC-16-CCITT by its definition: the message bits, most significant bit of
 * each byte first, are divided by x^16 + x^12 + x^5 + 1 with the register
 * preset to 0xFFFF; no reflection, no final XOR. One bit at a time.
 */
uint32_t or_crc16(const uint8_t* p, int64_t n) {
    uint32_t r = 0xFFFFu;
    for (int64_t i = 0; i < n; ++i) {
        for (int b = 7; b >= 0; --b) {
            const uint32_t in = (p[i] >> b) & 1u;
            const uint32_t top = (r >> 15) & 1u;
            r = (r << 1) & 0xFFFFu;
            if (top ^ in) r ^= 0x1021u;
        }
    }
    return r;
}
