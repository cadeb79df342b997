/*
 * Seeded synthetic inputs for the CTA real-time reconstruction path.
 *
 * This module makes INPUTS only: camera lattices and neighbour lists, the
 * telescope array layout, per-pixel pedestal/gain truth and the calibration
 * table derived from it, shower (image) parameters, and uint16 waveforms.
 * It contains none of the reconstruction arithmetic (window integration,
 * cleaning, moments, intersection); both the CUDA library and the CPU oracle
 * consume what it writes.
 *
 * Every random draw comes from a Philox-4x32-10 counter-based generator
 * (Salmon, Moraes, Dror, Shaw, SC'11), keyed by the seed and addressed by
 * (purpose, event, telescope, pixel), so the output does not depend on the
 * number of threads or on the order in which images are rendered.
 *
 * The paper (Sec. 2.2) describes the data as several time samples per pixel of
 * each triggered telescope, three telescope sizes (Sec. 1) and a central event
 * builder that groups the telescopes of one event (Sec. 4.1); the concrete
 * distributions below are the synthetic stand-in for the Prod2 simulations
 * the paper's assessment used (Sec. 5), which are not available.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* Philox-4x32-10                                                       */
/* ------------------------------------------------------------------ */
typedef struct {
    uint32_t key[2];
    uint32_t ctr[4];
    uint32_t buf[4];
    int used; /* words of buf already consumed (4 = empty) */
} rng_t;

static void philox4x32_10(const uint32_t in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = in[0], c1 = in[1], c2 = in[2], c3 = in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* purpose tags keep independent streams apart */
enum { P_EVENT = 1, P_IMAGE = 2, P_PIXEL = 3, P_CALIB = 4, P_TEST = 5 };

static void rng_init(rng_t* g, uint64_t seed, uint32_t purpose, uint32_t a, uint32_t b, uint32_t c) {
    g->key[0] = (uint32_t)seed;
    g->key[1] = (uint32_t)(seed >> 32) ^ (purpose * 0x85EBCA6Bu);
    g->ctr[0] = 0; g->ctr[1] = a; g->ctr[2] = b; g->ctr[3] = c;
    g->used = 4;
}

static uint32_t rng_u32(rng_t* g) {
    if (g->used == 4) {
        philox4x32_10(g->ctr, g->key, g->buf);
        g->ctr[0]++;
        g->used = 0;
    }
    return g->buf[g->used++];
}

/* uniform in the open interval (0, 1), 53-bit resolution */
static double rng_uniform(rng_t* g) {
    uint64_t a = rng_u32(g) >> 5, b = rng_u32(g) >> 6;
    return ((double)((a << 26) | b) + 0.5) * (1.0 / 9007199254740992.0);
}

/* standard normal, Box-Muller (one value per call; the pair partner is kept) */
typedef struct { rng_t r; int has; double spare; } nrng_t;
static double rng_normal(nrng_t* g) {
    if (g->has) { g->has = 0; return g->spare; }
    double u1 = rng_uniform(&g->r), u2 = rng_uniform(&g->r);
    double rad = sqrt(-2.0 * log(u1)), ang = 2.0 * M_PI * u2;
    g->spare = rad * sin(ang);
    g->has = 1;
    return rad * cos(ang);
}

/* Poisson deviate: inversion by sequential search for small means, PTRS
 * (Hormann 1993, "The transformed rejection method for generating Poisson
 * random variables") for mean >= 10. */
static int64_t rng_poisson(rng_t* g, double mu) {
    if (!(mu > 0.0)) return 0;
    if (mu < 10.0) {
        double u = rng_uniform(g), p = exp(-mu), cdf = p;
        int64_t k = 0;
        while (u > cdf && k < 1000) { ++k; p *= mu / (double)k; cdf += p; }
        return k;
    }
    double smu = sqrt(mu), lmu = log(mu);
    double b = 0.931 + 2.53 * smu;
    double a = -0.059 + 0.02483 * b;
    double inv_alpha = 1.1239 + 1.1328 / (b - 3.4);
    double vr = 0.9277 - 3.6224 / (b - 2.0);
    for (;;) {
        double U = rng_uniform(g) - 0.5, V = rng_uniform(g);
        double us = 0.5 - fabs(U);
        double kf = floor((2.0 * a / us + b) * U + mu + 0.43);
        if (us >= 0.07 && V <= vr) return (int64_t)kf;
        if (kf < 0.0 || (us < 0.013 && V > us)) continue;
        if (log(V) + log(inv_alpha) - log(a / (us * us) + b) <= -mu + kf * lmu - lgamma(kf + 1.0))
            return (int64_t)kf;
    }
}

/* exported for the generator's own tests */
void synth_test_uniforms(uint64_t seed, int n, double* out) {
    rng_t g; rng_init(&g, seed, P_TEST, 0, 0, 0);
    for (int i = 0; i < n; ++i) out[i] = rng_uniform(&g);
}
void synth_test_normals(uint64_t seed, int n, double* out) {
    nrng_t g; memset(&g, 0, sizeof g); rng_init(&g.r, seed, P_TEST, 1, 0, 0);
    for (int i = 0; i < n; ++i) out[i] = rng_normal(&g);
}
void synth_test_poisson(uint64_t seed, double mu, int n, int64_t* out) {
    rng_t g; rng_init(&g, seed, P_TEST, 2, 0, 0);
    for (int i = 0; i < n; ++i) out[i] = rng_poisson(&g, mu);
}
void synth_philox_block(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------ */
/* Camera lattices                                                      */
/* ------------------------------------------------------------------ */
enum { LAT_GRID = 0, LAT_HEX_FIRST_N = 1, LAT_SQUARE_FIRST_N = 2 };

typedef struct { double x, y; long long rkey; double ang; } latpt_t;

static int cmp_latpt(const void* pa, const void* pb) {
    const latpt_t* a = (const latpt_t*)pa;
    const latpt_t* b = (const latpt_t*)pb;
    if (a->rkey != b->rkey) return a->rkey < b->rkey ? -1 : 1;
    if (a->ang != b->ang) return a->ang < b->ang ? -1 : 1;
    return 0;
}

/*
 * Pixel centres (degrees) and a -1 padded neighbour table for a lattice.
 *   LAT_GRID:           nx*ny rectangular grid (nx = ny = sqrt(n_pix)), centred, row-major.
 *   LAT_HEX_FIRST_N:    hexagonal lattice points ordered by (distance rounded to
 *                       1e-9 pitch, polar angle in [0, 2pi)); the first n_pix kept.
 *   LAT_SQUARE_FIRST_N: square lattice, same ordering rule.
 * Neighbours are lattice points at one pitch (4 for square, 6 for hex), listed
 * in increasing pixel index, padded with -1 up to K.
 * Returns 0, or -1 on bad arguments.
 */
int synth_lattice(int kind, int n_pix, double pitch, int K, float* xy, int16_t* nb) {
    if (n_pix <= 0 || n_pix > 32767 || pitch <= 0.0 || K <= 0) return -1;
    double* px = (double*)malloc(sizeof(double) * 2 * (size_t)n_pix);
    if (!px) return -1;
    if (kind == LAT_GRID) {
        int nx = (int)llround(sqrt((double)n_pix));
        if (nx * nx != n_pix) { free(px); return -1; }
        for (int j = 0; j < nx; ++j)
            for (int i = 0; i < nx; ++i) {
                px[2 * (j * nx + i)] = (i - 0.5 * (nx - 1)) * pitch;
                px[2 * (j * nx + i) + 1] = (j - 0.5 * (nx - 1)) * pitch;
            }
    } else if (kind == LAT_HEX_FIRST_N || kind == LAT_SQUARE_FIRST_N) {
        int R = (int)ceil(sqrt((double)n_pix)) + 3;
        size_t cap = (size_t)(2 * R + 1) * (size_t)(2 * R + 1);
        latpt_t* pts = (latpt_t*)malloc(sizeof(latpt_t) * cap);
        if (!pts) { free(px); return -1; }
        size_t n = 0;
        for (int b = -R; b <= R; ++b)
            for (int a = -R; a <= R; ++a) {
                double x, y;
                if (kind == LAT_HEX_FIRST_N) { x = (a + 0.5 * b); y = b * (sqrt(3.0) / 2.0); }
                else { x = a; y = b; }
                latpt_t p;
                p.x = x * pitch; p.y = y * pitch;
                p.rkey = llround(sqrt(x * x + y * y) * 1e9);
                double ang = atan2(y, x);
                if (ang < 0) ang += 2.0 * M_PI;
                p.ang = ang;
                pts[n++] = p;
            }
        qsort(pts, n, sizeof(latpt_t), cmp_latpt);
        for (int i = 0; i < n_pix; ++i) { px[2 * i] = pts[i].x; px[2 * i + 1] = pts[i].y; }
        free(pts);
    } else {
        free(px);
        return -1;
    }
    for (int i = 0; i < n_pix; ++i) { xy[2 * i] = (float)px[2 * i]; xy[2 * i + 1] = (float)px[2 * i + 1]; }
    if (nb) {
        for (int i = 0; i < n_pix; ++i) {
            int c = 0;
            for (int j = 0; j < n_pix; ++j) {
                if (j == i) continue;
                double dx = px[2 * j] - px[2 * i], dy = px[2 * j + 1] - px[2 * i + 1];
                double d = sqrt(dx * dx + dy * dy);
                if (fabs(d - pitch) < 1e-6 * pitch && c < K) nb[(size_t)i * K + c++] = (int16_t)j;
            }
            for (; c < K; ++c) nb[(size_t)i * K + c] = -1;
        }
    }
    free(px);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Camera presets and array layout                                      */
/* ------------------------------------------------------------------ */
/* cam ids: 0 = 16x16 square 0.1 deg (16 samples), 1 = large (hex 1855, 0.1 deg, 40
 * samples), 2 = medium (hex 1764, 0.16 deg, 30 samples), 3 = small (square
 * first-2048, 0.19 deg, 25 samples). */
typedef struct { int kind, n_pix, n_samp, K; double pitch, area; double mirror_area_m2; double amp; } cam_preset_t;

static cam_preset_t cam_preset(int cam) {
    cam_preset_t c;
    memset(&c, 0, sizeof c);
    double hexa = sqrt(3.0) / 2.0;
    switch (cam) {
    case 0: c.kind = LAT_GRID; c.n_pix = 256; c.n_samp = 16; c.K = 4; c.pitch = 0.1; c.area = 0.01; c.mirror_area_m2 = 370.0; c.amp = 1.0; break;
    case 1: c.kind = LAT_HEX_FIRST_N; c.n_pix = 1855; c.n_samp = 40; c.K = 6; c.pitch = 0.1; c.area = hexa * 0.01; c.mirror_area_m2 = 370.0; c.amp = 1.0; break;
    case 2: c.kind = LAT_HEX_FIRST_N; c.n_pix = 1764; c.n_samp = 30; c.K = 6; c.pitch = 0.16; c.area = hexa * 0.0256; c.mirror_area_m2 = 100.0; c.amp = 0.4; break;
    case 3: c.kind = LAT_SQUARE_FIRST_N; c.n_pix = 2048; c.n_samp = 25; c.K = 4; c.pitch = 0.19; c.area = 0.0361; c.mirror_area_m2 = 8.0; c.amp = 0.15; break;
    default: c.n_pix = 0;
    }
    return c;
}

/* info[0..3] = n_pix, n_samples, K, lattice kind; finfo[0..2] = pitch deg, pixel area deg^2, mirror area m^2 */
int synth_camera_info(int cam, int32_t* info, double* finfo) {
    cam_preset_t c = cam_preset(cam);
    if (c.n_pix == 0) return -1;
    info[0] = c.n_pix; info[1] = c.n_samp; info[2] = c.K; info[3] = c.kind;
    finfo[0] = c.pitch; finfo[1] = c.area; finfo[2] = c.mirror_area_m2;
    return 0;
}

int synth_camera(int cam, float* xy, int16_t* nb) {
    cam_preset_t c = cam_preset(cam);
    if (c.n_pix == 0) return -1;
    return synth_lattice(c.kind, c.n_pix, c.pitch, c.K, xy, nb);
}

/* The 69-telescope layout: 4 large on a 160 m square, 5 + 10 medium on rings
 * of 200 m and 350 m, 20 + 30 small on rings of 450 m and 560 m. */
#define N_ARRAY_TEL 69
int synth_array(int32_t* tel_cam, float* tel_xy) {
    int t = 0;
    for (int i = 0; i < 4; ++i) {
        tel_cam[t] = 1;
        tel_xy[2 * t] = (i & 1) ? 80.f : -80.f;
        tel_xy[2 * t + 1] = (i & 2) ? 80.f : -80.f;
        ++t;
    }
    struct { int n, cam; double r, phase; } rings[4] = {{5, 2, 200.0, 0.0}, {10, 2, 350.0, 0.5}, {20, 3, 450.0, 0.0}, {30, 3, 560.0, 0.5}};
    for (int k = 0; k < 4; ++k)
        for (int i = 0; i < rings[k].n; ++i) {
            double a = 2.0 * M_PI * (i + rings[k].phase) / rings[k].n;
            tel_cam[t] = rings[k].cam;
            tel_xy[2 * t] = (float)(rings[k].r * cos(a));
            tel_xy[2 * t + 1] = (float)(rings[k].r * sin(a));
            ++t;
        }
    return t;
}

/* ------------------------------------------------------------------ */
/* Pulse shape and calibration                                          */
/* ------------------------------------------------------------------ */
#define PULSE_SIGMA 1.5
#define PULSE_PEAK 6.0
#define TIME_GRAD 2.0 /* samples per degree along the major axis */
#define PED_MEAN 400.0
#define PED_SIGMA 5.0
#define GAIN_MEAN 8.0
#define GAIN_REL_SIGMA 0.05
#define NSB_MEAN 0.3
#define ENOISE 2.0

static double pulse_norm(void) {
    double z = 0.0;
    for (int k = -60; k <= 60; ++k) z += exp(-(double)k * k / (2.0 * PULSE_SIGMA * PULSE_SIGMA));
    return z;
}
/* point-sampled unit-sum Gaussian pulse, g(x) with sum_k g(k) = 1 */
static double pulse(double x, double inv_norm) {
    return exp(-x * x / (2.0 * PULSE_SIGMA * PULSE_SIGMA)) * inv_norm;
}

/* Fraction of an on-grid pulse that the processing window contains:
 * sliding W: best W-window around a pulse at an integer sample, lowest start on ties;
 * fixed: samples [start, start+W) around the pulse at PULSE_PEAK. */
double synth_window_fraction(int sliding, int start, int W) {
    double inv = 1.0 / pulse_norm();
    if (!sliding) {
        double f = 0.0;
        for (int k = start; k < start + W; ++k) f += pulse(k - PULSE_PEAK, inv);
        return f;
    }
    double best = -1.0;
    for (int s = -W; s <= 0; ++s) {
        double f = 0.0;
        for (int k = s; k < s + W; ++k) f += pulse((double)k, inv);
        if (f > best + 1e-15) best = f;
    }
    return best;
}

/* Per (telescope, pixel) truth: pedestal (ADC/sample) and gain (ADC/pe), and
 * the calibration table the reconstruction receives: the pedestal in 1/16 ADC
 * fixed point, p16 = round(16 ped), and scale = fp32(1 / (16 gain f_W)), which
 * turns a window sum in the same 1/16 ADC units into photoelectrons.
 * tel_cam[n_tel]; pix_off[n_tel] gives each telescope's first row. */
int synth_calibration(uint64_t seed, int n_tel, const int32_t* tel_cam, const int64_t* pix_off,
                      double f_window, double* ped, double* gain, int32_t* p16, float* scale) {
    for (int t = 0; t < n_tel; ++t) {
        cam_preset_t c = cam_preset(tel_cam[t]);
        if (c.n_pix == 0) return -1;
        for (int p = 0; p < c.n_pix; ++p) {
            nrng_t g; memset(&g, 0, sizeof g);
            rng_init(&g.r, seed, P_CALIB, (uint32_t)t, (uint32_t)p, 0);
            double pd = PED_MEAN + PED_SIGMA * rng_normal(&g);
            double gn = GAIN_MEAN * (1.0 + GAIN_REL_SIGMA * rng_normal(&g));
            int64_t row = pix_off[t] + p;
            ped[row] = pd; gain[row] = gn;
            p16[row] = (int32_t)llround(16.0 * pd);
            scale[row] = (float)(1.0 / (16.0 * gn * f_window));
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Event / image planning                                               */
/* ------------------------------------------------------------------ */
/* One image = up to 3 Gaussian ellipses. Per ellipse 6 values:
 * (size pe, cx deg, cy deg, length deg, width deg, psi rad). Ellipse 0 also
 * carries the pulse-time gradient axis. */
#define MAX_ELL 3
#define ELL_STRIDE (MAX_ELL * 6)

static double log_uniform(rng_t* g, double lo, double hi) {
    return exp(log(lo) + (log(hi) - log(lo)) * rng_uniform(g));
}
static double uni(rng_t* g, double lo, double hi) { return lo + (hi - lo) * rng_uniform(g); }

/*
 * Single-telescope workload (one image per event, telescope 0): sizes
 * log-uniform in [size_lo, size_hi] pe, length U(0.1,0.4) deg, width
 * U(0.03,0.1) deg, centroid uniform in a disc of 0.6 deg, psi U(0, pi).
 * ell[n_evt*ELL_STRIDE], n_ell[n_evt].
 */
int synth_plan_single(uint64_t seed, int64_t n_evt, double size_lo, double size_hi, float* ell, int32_t* n_ell) {
    for (int64_t e = 0; e < n_evt; ++e) {
        rng_t g; rng_init(&g, seed, P_IMAGE, (uint32_t)e, (uint32_t)(e >> 32), 0xFFFFu);
        double size = log_uniform(&g, size_lo, size_hi);
        double len = uni(&g, 0.1, 0.4), wid = uni(&g, 0.03, 0.1);
        double rr = 0.6 * sqrt(rng_uniform(&g)), ra = 2.0 * M_PI * rng_uniform(&g);
        double psi = M_PI * rng_uniform(&g);
        float* o = ell + e * ELL_STRIDE;
        memset(o, 0, sizeof(float) * ELL_STRIDE);
        o[0] = (float)size; o[1] = (float)(rr * cos(ra)); o[2] = (float)(rr * sin(ra));
        o[3] = (float)len; o[4] = (float)wid; o[5] = (float)psi;
        n_ell[e] = 1;
    }
    return 0;
}

/*
 * Stereo-array workload. For event slot e, attempts a = 0, 1, ... draw
 * E ~ E^-2.5 on [0.03, 100] TeV, a source direction uniform within 2 deg of
 * pointing and a core uniform in an 800 m disc. Telescopes at impact distance
 * d < R(E) = 120 m (E / 0.1 TeV)^0.4 with image size
 * A_type (E / 1 TeV) 1500 pe exp(-d / 150 m) >= 30 pe trigger; the first
 * attempt with at least 2 triggered telescopes is kept (the 40 nearest if more).
 * Gamma images: the major axis points along (T - C) and the centroid sits at
 * source + 0.01 deg/m * min(d, 200 m) along it. Proton-like images
 * (proton_frac > 0): width x U(2,3), 1-3 sub-ellipses, random axes, no source
 * alignment.
 * Outputs: evt_off[n_evt+1] (CSR), img_tel[], ell[], n_ell[], and per event
 * truth[n_evt*8] = (E TeV, src_x, src_y deg, core_x, core_y m, is_proton, m, attempts).
 * max_img bounds the image arrays; returns the image count or -1.
 */
int64_t synth_plan_array(uint64_t seed, int64_t n_evt, double proton_frac, int n_tel, const int32_t* tel_cam,
                         const float* tel_xy, int64_t max_img, int32_t* evt_off, int32_t* img_tel, float* ell,
                         int32_t* n_ell, double* truth) {
    const double G = 2.5, Emin = 0.03, Emax = 100.0;
    int64_t n_img = 0;
    if (n_tel < 1 || n_tel > 128) return -1;
    evt_off[0] = 0;
    for (int64_t e = 0; e < n_evt; ++e) {
        int sel[128];
        double dist[128], sz[128];
        int m = 0;
        double E = 0, sx = 0, sy = 0, cx = 0, cy = 0;
        int proton = 0;
        uint32_t a;
        for (a = 0; a < 1000000u; ++a) {
            rng_t g; rng_init(&g, seed, P_EVENT, (uint32_t)e, (uint32_t)(e >> 32), a);
            double u = rng_uniform(&g);
            double p0 = pow(Emin, 1.0 - G), p1 = pow(Emax, 1.0 - G);
            E = pow(p0 + u * (p1 - p0), 1.0 / (1.0 - G));
            double r = 2.0 * sqrt(rng_uniform(&g)), ang = 2.0 * M_PI * rng_uniform(&g);
            sx = r * cos(ang); sy = r * sin(ang);
            double rc = 800.0 * sqrt(rng_uniform(&g)), ac = 2.0 * M_PI * rng_uniform(&g);
            cx = rc * cos(ac); cy = rc * sin(ac);
            proton = rng_uniform(&g) < proton_frac;
            double R = 120.0 * pow(E / 0.1, 0.4);
            m = 0;
            for (int t = 0; t < n_tel && t < 128; ++t) {
                cam_preset_t c = cam_preset(tel_cam[t]);
                double dx = tel_xy[2 * t] - cx, dy = tel_xy[2 * t + 1] - cy;
                double d = sqrt(dx * dx + dy * dy);
                double s = c.amp * E * 1500.0 * exp(-d / 150.0);
                if (d < R && s >= 30.0) { sel[m] = t; dist[m] = d; sz[m] = s; ++m; }
            }
            if (m >= 2) break;
        }
        if (m < 2) return -1;
        if (m > 40) { /* keep the 40 nearest (selection by distance, ties by index) */
            for (int i = 0; i < 40; ++i) {
                int best = i;
                for (int j = i + 1; j < m; ++j)
                    if (dist[j] < dist[best] || (dist[j] == dist[best] && sel[j] < sel[best])) best = j;
                int ts = sel[i]; sel[i] = sel[best]; sel[best] = ts;
                double td = dist[i]; dist[i] = dist[best]; dist[best] = td;
                double tz = sz[i]; sz[i] = sz[best]; sz[best] = tz;
            }
            m = 40;
            /* restore telescope-index order */
            for (int i = 1; i < m; ++i)
                for (int j = i; j > 0 && sel[j] < sel[j - 1]; --j) {
                    int ts = sel[j]; sel[j] = sel[j - 1]; sel[j - 1] = ts;
                    double td = dist[j]; dist[j] = dist[j - 1]; dist[j - 1] = td;
                    double tz = sz[j]; sz[j] = sz[j - 1]; sz[j - 1] = tz;
                }
        }
        if (n_img + m > max_img) return -1;
        double* tr = truth + e * 8;
        tr[0] = E; tr[1] = sx; tr[2] = sy; tr[3] = cx; tr[4] = cy; tr[5] = proton; tr[6] = m; tr[7] = a;
        for (int i = 0; i < m; ++i) {
            int t = sel[i];
            rng_t g; rng_init(&g, seed, P_IMAGE, (uint32_t)e, (uint32_t)(e >> 32), (uint32_t)t);
            float* o = ell + n_img * ELL_STRIDE;
            memset(o, 0, sizeof(float) * ELL_STRIDE);
            double len = uni(&g, 0.1, 0.4), wid = uni(&g, 0.03, 0.1);
            if (!proton) {
                double ux = tel_xy[2 * t] - cx, uy = tel_xy[2 * t + 1] - cy;
                double d = dist[i];
                double psi = atan2(uy, ux);
                double ex = d > 0 ? ux / d : 1.0, ey = d > 0 ? uy / d : 0.0;
                double off = 0.01 * (d < 200.0 ? d : 200.0);
                o[0] = (float)sz[i]; o[1] = (float)(sx + off * ex); o[2] = (float)(sy + off * ey);
                o[3] = (float)len; o[4] = (float)wid; o[5] = (float)psi;
                n_ell[n_img] = 1;
            } else {
                int ns = 1 + (int)(3.0 * rng_uniform(&g));
                if (ns > 3) ns = 3;
                double rr = 2.0 * sqrt(rng_uniform(&g)), ra = 2.0 * M_PI * rng_uniform(&g);
                double bx = rr * cos(ra), by = rr * sin(ra);
                double wsum = 0, w[3];
                for (int k = 0; k < ns; ++k) { w[k] = 0.2 + rng_uniform(&g); wsum += w[k]; }
                for (int k = 0; k < ns; ++k) {
                    double l2 = k ? uni(&g, 0.1, 0.4) : len, w2 = (k ? uni(&g, 0.03, 0.1) : wid) * uni(&g, 2.0, 3.0);
                    double ps = M_PI * rng_uniform(&g);
                    double jx = k ? 0.4 * (rng_uniform(&g) - 0.5) : 0.0, jy = k ? 0.4 * (rng_uniform(&g) - 0.5) : 0.0;
                    float* q = o + 6 * k;
                    q[0] = (float)(sz[i] * w[k] / wsum); q[1] = (float)(bx + jx); q[2] = (float)(by + jy);
                    q[3] = (float)l2; q[4] = (float)w2; q[5] = (float)ps;
                }
                n_ell[n_img] = ns;
            }
            img_tel[n_img] = t;
            ++n_img;
        }
        evt_off[e + 1] = (int32_t)n_img;
    }
    return n_img;
}

/* ------------------------------------------------------------------ */
/* Waveform rendering                                                   */
/* ------------------------------------------------------------------ */
typedef struct {
    uint64_t seed;
    int64_t n_img;
    const int32_t* img_evt;  /* event slot of each image (stream address) */
    const int32_t* img_tel;
    const int32_t* tel_cam;
    const int64_t* tel_pix_off;
    const double* ped;
    const double* gain;
    const float* ell;
    const int32_t* n_ell;
    const float* const* cam_xy; /* per cam id: 2*P floats */
    const int64_t* wave_off;    /* per image, in samples */
    uint16_t* wave;
    int flags;                  /* bit0: no electronic noise, bit1: no NSB */
    int64_t next;               /* work counter (atomic) */
} render_job_t;

static void render_image(const render_job_t* J, int64_t i, double inv_norm) {
    int tel = J->img_tel[i];
    int cam = J->tel_cam[tel];
    cam_preset_t c = cam_preset(cam);
    const float* xy = J->cam_xy[cam];
    const float* el = J->ell + i * ELL_STRIDE;
    int ne = J->n_ell[i];
    uint16_t* out = J->wave + J->wave_off[i];
    int S = c.n_samp;
    double amp[64];
    uint32_t evt = (uint32_t)J->img_evt[i];
    for (int p = 0; p < c.n_pix; ++p) {
        double x = xy[2 * p], y = xy[2 * p + 1];
        int64_t row = J->tel_pix_off[tel] + p;
        double ped = J->ped[row], gain = J->gain[row];
        nrng_t g; memset(&g, 0, sizeof g);
        rng_init(&g.r, J->seed, P_PIXEL, evt, (uint32_t)tel, (uint32_t)p);
        for (int k = 0; k < S; ++k) amp[k] = ped;
        for (int e = 0; e < ne; ++e) {
            const float* q = el + 6 * e;
            double cs = cos(q[5]), sn = sin(q[5]);
            double dx = x - q[1], dy = y - q[2];
            double l = dx * cs + dy * sn, w = -dx * sn + dy * cs;
            double L = q[3], Wd = q[4];
            double dens = exp(-0.5 * (l * l / (L * L) + w * w / (Wd * Wd))) / (2.0 * M_PI * L * Wd);
            double mu = q[0] * dens * c.area;
            int64_t n = mu > 1e-9 ? rng_poisson(&g.r, mu) : 0;
            if (n == 0) continue;
            double t0 = PULSE_PEAK + TIME_GRAD * l;
            int k0 = (int)floor(t0 - 10.0), k1 = (int)ceil(t0 + 10.0);
            if (k0 < 0) k0 = 0;
            if (k1 > S - 1) k1 = S - 1;
            for (int k = k0; k <= k1; ++k) amp[k] += gain * (double)n * pulse(k - t0, inv_norm);
        }
        if (!(J->flags & 2)) {
            int64_t nn = rng_poisson(&g.r, NSB_MEAN);
            for (int64_t j = 0; j < nn; ++j) {
                double t0 = S * rng_uniform(&g.r);
                int k0 = (int)floor(t0 - 10.0), k1 = (int)ceil(t0 + 10.0);
                if (k0 < 0) k0 = 0;
                if (k1 > S - 1) k1 = S - 1;
                for (int k = k0; k <= k1; ++k) amp[k] += gain * pulse(k - t0, inv_norm);
            }
        }
        for (int k = 0; k < S; ++k) {
            double v = amp[k];
            if (!(J->flags & 1)) v += ENOISE * rng_normal(&g);
            v = floor(v + 0.5);
            if (v < 0.0) v = 0.0;
            if (v > 65535.0) v = 65535.0;
            out[(size_t)p * S + k] = (uint16_t)v;
        }
    }
}

static void* render_worker(void* arg) {
    render_job_t* J = (render_job_t*)arg;
    double inv_norm = 1.0 / pulse_norm();
    for (;;) {
        int64_t i = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (i >= J->n_img) break;
        render_image(J, i, inv_norm);
    }
    return NULL;
}

/*
 * Render uint16 waveforms (wave[wave_off[i] + pix*S + sample]) for n_img images:
 * sample = clamp(floor(ped + gain * sum_pe g(k - t_pe) + N(0, 2) + 0.5), 0, 65535)
 * where signal pe per pixel ~ Poisson(size * ellipse density * pixel area) arrive
 * at t = 6 + 2 * (offset along the major axis, deg) and NSB pe ~ Poisson(0.3) at
 * uniform times. cam_xy is indexed by camera id (entries may be NULL for unused
 * ids). flags: bit0 disables electronic noise, bit1 disables NSB.
 */
int synth_render(uint64_t seed, int64_t n_img, const int32_t* img_evt, const int32_t* img_tel, const int32_t* tel_cam,
                 const int64_t* tel_pix_off, const double* ped, const double* gain, const float* ell,
                 const int32_t* n_ell, const float* const* cam_xy, const int64_t* wave_off, uint16_t* wave,
                 int flags, int n_threads) {
    render_job_t J;
    J.seed = seed; J.n_img = n_img; J.img_evt = img_evt; J.img_tel = img_tel; J.tel_cam = tel_cam;
    J.tel_pix_off = tel_pix_off; J.ped = ped; J.gain = gain; J.ell = ell; J.n_ell = n_ell; J.cam_xy = cam_xy;
    J.wave_off = wave_off; J.wave = wave; J.flags = flags; J.next = 0;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    int started = 0;
    for (int i = 1; i < n_threads; ++i)
        if (pthread_create(&th[started], NULL, render_worker, &J) == 0) ++started;
    render_worker(&J);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    return 0;
}

/* ------------------------------------------------------------------ */
/* DL0 byte stream (the event builder's output; layout in include/rta.h) */
/* ------------------------------------------------------------------ */
static uint16_t crc16_table[256];
static pthread_once_t crc16_once = PTHREAD_ONCE_INIT;

static void crc16_init(void) {
    for (int b = 0; b < 256; ++b) {
        uint16_t r = (uint16_t)(b << 8);
        for (int k = 0; k < 8; ++k) r = (r & 0x8000u) ? (uint16_t)((r << 1) ^ 0x1021u) : (uint16_t)(r << 1);
        crc16_table[b] = r;
    }
}

/* CRC-16-CCITT, polynomial 0x1021, initial value 0xFFFF, no reflection. */
uint16_t synth_crc16(const uint8_t* p, int64_t n) {
    pthread_once(&crc16_once, crc16_init);
    uint16_t r = 0xFFFFu;
    for (int64_t i = 0; i < n; ++i) r = (uint16_t)((r << 8) ^ crc16_table[((r >> 8) ^ p[i]) & 0xFF]);
    return r;
}

static void put16(uint8_t* p, uint32_t v) { p[0] = (uint8_t)(v >> 8); p[1] = (uint8_t)v; }
static void put32(uint8_t* p, uint32_t v) { put16(p, v >> 16); put16(p + 2, v); }

typedef struct {
    int64_t n_pk;
    const int32_t *pk_img, *pk_first, *pk_n, *pk_flags, *pk_count;
    const int64_t* pk_off;
    const uint16_t* wave;
    const int64_t* wave_off;
    const int32_t *img_tel, *img_P, *img_S;
    const uint64_t* img_evnum;
    const int64_t* img_time_ns;
    uint8_t* out;
    int64_t next;
} stream_job_t;

static void* stream_worker(void* arg) {
    stream_job_t* J = (stream_job_t*)arg;
    for (;;) {
        int64_t k = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (k >= J->n_pk) break;
        const int i = J->pk_img[k], P = J->img_P[i], S = J->img_S[i];
        const int first = J->pk_first[k], n = J->pk_n[k];
        const int64_t nbytes = (int64_t)n * S * 2, total = 48 + nbytes;
        uint8_t* p = J->out + J->pk_off[k];
        put16(p, (0u << 13) | (0u << 12) | (1u << 11) | ((uint32_t)J->img_tel[i] & 0x7FFu));
        put16(p + 2, ((uint32_t)J->pk_flags[k] << 14) | ((uint32_t)J->pk_count[k] & 0x3FFFu));
        put16(p + 4, (uint32_t)(total - 7));
        p[6] = 0x10; p[7] = 200; p[8] = 1; p[9] = 0;
        const int64_t t = J->img_time_ns[i];
        const int64_t sec = t / 1000000000, ns = t % 1000000000;
        put32(p + 10, (uint32_t)sec);
        put16(p + 14, (uint32_t)((ns * 65536) / 1000000000));
        put32(p + 16, (uint32_t)(J->img_evnum[i] >> 32));
        put32(p + 20, (uint32_t)J->img_evnum[i]);
        put16(p + 24, (uint32_t)first);
        put16(p + 26, (uint32_t)n);
        put16(p + 28, (uint32_t)P);
        put16(p + 30, (uint32_t)S);
        const uint16_t* src = J->wave + J->wave_off[i] + (int64_t)first * S;
        for (int64_t j = 0; j < (int64_t)n * S; ++j) {      /* little-endian samples */
            p[32 + 2 * j] = (uint8_t)src[j];
            p[33 + 2 * j] = (uint8_t)(src[j] >> 8);
        }
        memset(p + 32 + nbytes, 0, 14);
        put16(p + 46 + nbytes, synth_crc16(p, 46 + nbytes));
    }
    return NULL;
}

/* Write n_pk packets (plan in stream order: image, first pixel, pixel count,
 * sequence flags and count, byte offset) from a bundle into out. */
int synth_write_stream(int64_t n_pk, const int32_t* pk_img, const int32_t* pk_first, const int32_t* pk_n,
                       const int32_t* pk_flags, const int32_t* pk_count, const int64_t* pk_off, const uint16_t* wave,
                       const int64_t* wave_off, const int32_t* img_tel, const int32_t* img_P, const int32_t* img_S,
                       const uint64_t* img_evnum, const int64_t* img_time_ns, uint8_t* out, int n_threads) {
    stream_job_t J = {n_pk, pk_img, pk_first, pk_n, pk_flags, pk_count, pk_off, wave, wave_off, img_tel, img_P,
                      img_S, img_evnum, img_time_ns, out, 0};
    pthread_once(&crc16_once, crc16_init);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    int started = 0;
    for (int i = 1; i < n_threads; ++i)
        if (pthread_create(&th[started], NULL, stream_worker, &J) == 0) ++started;
    stream_worker(&J);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    return 0;
}
