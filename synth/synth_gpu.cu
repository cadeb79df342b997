/*
 * The waveform renderer of synth.c on the GPU, for bulk inputs (the learned
 * surrogate's training and held-out sets of hundreds of thousands of events,
 * which the host renderer would need minutes for).
 *
 * Input generation only, like synth.c: nothing here computes any step of the
 * reconstruction. Same model and the same random streams (Philox-4x32-10 keyed
 * by seed and purpose, addressed by event, telescope and pixel, drawn in the
 * same order), computed in FP32 with the device's fast math functions, so the
 * samples follow the same distributions as the host renderer's but are not
 * equal to them bit for bit. Parity tests use the host renderer; this one only
 * feeds training and statistical evaluation.
 *
 * Per pixel: signal photoelectrons ~ Poisson(size x ellipse density x pixel
 * area) at t = 6 + 2 x (offset along the major axis, deg), night-sky
 * photoelectrons ~ Poisson(0.3) at uniform times, each a point-sampled
 * Gaussian pulse (sigma 1.5 samples, unit sum) times the pixel's gain, on the
 * pedestal, plus N(0, 2) ADC of electronic noise, rounded and clamped to uint16.
 */
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int ELL = 3;            // ellipses per image at most
constexpr int MAX_NSB = 16;       // night-sky photoelectrons kept per pixel (P(> 16 | mean 0.3) ~ 1e-27)
constexpr float PULSE_SIGMA = 1.5f, PULSE_PEAK = 6.f, TIME_GRAD = 2.f, NSB_MEAN = 0.3f, ENOISE = 2.f;

struct Rng {
    uint32_t key[2], ctr[4], buf[4];
    int used;
};

__device__ __forceinline__ void philox(const uint32_t in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = in[0], c1 = in[1], c2 = in[2], c3 = in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

__device__ __forceinline__ uint32_t next_u32(Rng& g) {
    if (g.used == 4) {
        philox(g.ctr, g.key, g.buf);
        g.ctr[0]++;
        g.used = 0;
    }
    return g.buf[g.used++];
}

// uniform in (0, 1): two words as in the host renderer, kept to FP32 resolution
__device__ __forceinline__ float uniform(Rng& g) {
    const uint32_t a = next_u32(g) >> 5, b = next_u32(g) >> 6;
    return (float((uint64_t(a) << 26 | b) >> 29) + 0.5f) * (1.f / 16777216.f);
}

// Poisson deviate: inversion by sequential search below a mean of 10, the
// transformed rejection of Hormann (1993, PTRS) above, as the host renderer.
__device__ int poisson(Rng& g, float mu) {
    if (!(mu > 0.f)) return 0;
    if (mu < 10.f) {
        const float u = uniform(g);
        float p = __expf(-mu), cdf = p;
        int k = 0;
        while (u > cdf && k < 1000) {
            ++k;
            p *= mu / float(k);
            cdf += p;
        }
        return k;
    }
    const float smu = sqrtf(mu), lmu = __logf(mu);
    const float b = 0.931f + 2.53f * smu;
    const float a = -0.059f + 0.02483f * b;
    const float inv_alpha = 1.1239f + 1.1328f / (b - 3.4f);
    const float vr = 0.9277f - 3.6224f / (b - 2.f);
    for (int it = 0; it < 1000; ++it) {
        const float U = uniform(g) - 0.5f, V = uniform(g);
        const float us = 0.5f - fabsf(U);
        const float kf = floorf((2.f * a / us + b) * U + mu + 0.43f);
        if (us >= 0.07f && V <= vr) return int(kf);
        if (kf < 0.f || (us < 0.013f && V > us)) continue;
        if (__logf(V) + __logf(inv_alpha) - __logf(a / (us * us) + b) <= -mu + kf * lmu - lgammaf(kf + 1.f))
            return int(kf);
    }
    return int(mu);
}

}  // namespace

struct RenderGpuArgs {
    uint64_t seed;
    int64_t n_img;
    const int32_t* img_evt;
    const int32_t* img_tel;
    const int32_t* tel_cam;
    const int64_t* tel_pix_off;
    const float* ped;
    const float* gain;
    const float* ell;            // [n_img][ELL * 6]: size, x, y, length, width, angle
    const int32_t* n_ell;
    const float2* cam_xy[16];    // per camera id
    int cam_pix[16], cam_samp[16];
    float cam_area[16];
    const int64_t* wave_off;
    uint16_t* wave;
    float inv_norm;              // 1 / sum_k exp(-k^2 / (2 sigma^2))
};

// One CTA per image, a thread per pixel at a time.
__global__ void __launch_bounds__(256) k_render(const RenderGpuArgs a) {
    for (int64_t i = blockIdx.x; i < a.n_img; i += gridDim.x) {
        const int tel = a.img_tel[i], cam = a.tel_cam[tel];
        const int P = a.cam_pix[cam], S = a.cam_samp[cam];
        const float area = a.cam_area[cam];
        const float* el = a.ell + i * ELL * 6;
        const int ne = min(a.n_ell[i], ELL);
        uint16_t* out = a.wave + a.wave_off[i];
        const uint32_t evt = uint32_t(a.img_evt[i]);
        for (int p = threadIdx.x; p < P; p += blockDim.x) {
            const float2 xy = a.cam_xy[cam][p];
            const int64_t row = a.tel_pix_off[tel] + p;
            const float ped = a.ped[row], gain = a.gain[row];
            Rng g;
            g.key[0] = uint32_t(a.seed);
            g.key[1] = uint32_t(a.seed >> 32) ^ (3u * 0x85EBCA6Bu);      // the pixel purpose
            g.ctr[0] = 0;
            g.ctr[1] = evt;
            g.ctr[2] = uint32_t(tel);
            g.ctr[3] = uint32_t(p);
            g.used = 4;
            float t_sig[ELL], n_sig[ELL];
            for (int e = 0; e < ELL; ++e) t_sig[e] = n_sig[e] = 0.f;
            for (int e = 0; e < ne; ++e) {
                const float* q = el + 6 * e;
                float sn, cs;
                __sincosf(q[5], &sn, &cs);
                const float dx = xy.x - q[1], dy = xy.y - q[2];
                const float l = dx * cs + dy * sn, w = -dx * sn + dy * cs;
                const float L = q[3], Wd = q[4];
                const float dens = __expf(-0.5f * (l * l / (L * L) + w * w / (Wd * Wd))) / (6.2831853f * L * Wd);
                const float mu = q[0] * dens * area;
                n_sig[e] = mu > 1e-9f ? float(poisson(g, mu)) : 0.f;
                t_sig[e] = PULSE_PEAK + TIME_GRAD * l;
            }
            float t_nsb[MAX_NSB];
            const int nn = min(poisson(g, NSB_MEAN), MAX_NSB);
            for (int j = 0; j < nn; ++j) t_nsb[j] = float(S) * uniform(g);
            const float c = -1.f / (2.f * PULSE_SIGMA * PULSE_SIGMA);
            bool has = false;
            float spare = 0.f;
            for (int k = 0; k < S; ++k) {
                float pe = 0.f;
                for (int e = 0; e < ne; ++e)
                    if (n_sig[e] > 0.f && fabsf(k - t_sig[e]) <= 10.f) pe += n_sig[e] * __expf(c * (k - t_sig[e]) * (k - t_sig[e]));
                for (int j = 0; j < nn; ++j)
                    if (fabsf(k - t_nsb[j]) <= 10.f) pe += __expf(c * (k - t_nsb[j]) * (k - t_nsb[j]));
                float v = ped + gain * pe * a.inv_norm;
                // Box-Muller, one value per sample, the pair's partner kept
                float z;
                if (has) {
                    z = spare;
                    has = false;
                } else {
                    const float u1 = uniform(g), u2 = uniform(g);
                    const float rad = sqrtf(-2.f * __logf(u1));
                    float s2, c2;
                    __sincosf(6.2831853f * u2, &s2, &c2);
                    spare = rad * s2;
                    z = rad * c2;
                    has = true;
                }
                v = floorf(v + ENOISE * z + 0.5f);
                out[int64_t(p) * S + k] = uint16_t(fminf(fmaxf(v, 0.f), 65535.f));
            }
        }
    }
}

extern "C" int synth_render_gpu(const RenderGpuArgs* args, int grid, void* stream) {
    k_render<<<grid, 256, 0, (cudaStream_t)stream>>>(*args);
    return int(cudaGetLastError());
}

extern "C" int synth_render_gpu_args_size(void) { return int(sizeof(RenderGpuArgs)); }
