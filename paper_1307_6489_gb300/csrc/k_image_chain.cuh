// Image kernels: calibration + charge integration, tailcut cleaning and Hillas
// moments (the per-telescope part of RT-RECO, Sec. 4.1; signal extraction,
// Sec. 5).
//
// k_image_chain is the hot path. It is a persistent, warp-specialised kernel:
//   warp 0      producer: takes the next image from a global work counter and
//               streams it, chunk by chunk, into a ring of shared-memory stages
//               with bulk copies on the TMA engine (cp.async.bulk, one mbarrier
//               per stage, transaction-count completion); the calibration rows
//               of the chunk's pixels travel with it;
//   warps 1..8  consumers: one thread per pixel of the chunk computes the
//               integer window sum, the single FP32 calibration multiply and the
//               peak time, keeping q and t in shared memory; after the image's
//               last chunk they clean it and reduce the Hillas moments with warp
//               shuffles, while the producer already streams the next image.
// Waveform bytes are read from HBM exactly once; per-pixel values never leave
// the SM. Every mbarrier wait is bounded by the global timer; a wait that runs
// out sets RTA_DEV_TIMEOUT, raises a CTA-wide abort flag and the CTA drains its
// copies in flight before it returns.
#pragma once

#include "rta_launch.cuh"

namespace rta {

constexpr int NCW = 8;             // warps of the block-wide (unfused) kernels
constexpr int NCT = NCW * 32;
constexpr int MAX_STAGES = 8;

enum { HDR_LAST = 1, HDR_BAD = 2, HDR_END = 4 };

struct StageHdr {
    int img;
    int base;      // first pixel of the chunk
    int npix;      // pixels in the chunk
    int flags;     // HDR_*
    int P, S, cam, seg0;  // seg0, seg1: the image's segments of a byte stream
    int64_t pix_off;
    int64_t woff;  // first sample of the image in the waveform buffer
    int64_t row;   // first calibration row of the image's telescope
    int seg1, pad;
};


// ------------------------------------------------------------------ per-pixel integration
template <int S>
__device__ __forceinline__ void load_row(const uint16_t* row, uint32_t (&w)[(S + 1) / 2]) {
    if constexpr ((2 * S) % 16 == 0) {
        const uint4* v = reinterpret_cast<const uint4*>(row);
#pragma unroll
        for (int k = 0; k < S / 8; ++k) {
            uint4 a = v[k];
            w[4 * k] = a.x; w[4 * k + 1] = a.y; w[4 * k + 2] = a.z; w[4 * k + 3] = a.w;
        }
    } else if constexpr (S % 2 == 0) {
        const uint32_t* v = reinterpret_cast<const uint32_t*>(row);
#pragma unroll
        for (int k = 0; k < S / 2; ++k) w[k] = v[k];
    } else {
        const uintptr_t a = reinterpret_cast<uintptr_t>(row);
        const uint32_t* v = reinterpret_cast<const uint32_t*>(a & ~uintptr_t(3));
        const uint32_t sh = (a & 2) ? 16u : 0u;
        uint32_t tmp[(S + 1) / 2 + 1];
#pragma unroll
        for (int k = 0; k < (S + 1) / 2 + 1; ++k) tmp[k] = v[k];
#pragma unroll
        for (int k = 0; k < (S + 1) / 2; ++k) w[k] = __funnelshift_r(tmp[k], tmp[k + 1], sh);
    }
}

template <int S>
__device__ __forceinline__ int sample(const uint32_t (&w)[(S + 1) / 2], int k) {
    return (k & 1) ? int(w[k >> 1] >> 16) : int(w[k >> 1] & 0xFFFFu);
}

// Maximum over a compile-time array as a tree of three-input maxima (no serial
// dependency chain, half the instructions of a pairwise tree).
template <int N>
__device__ __forceinline__ int tree_max(int (&v)[N]) {
#pragma unroll
    for (int step = 1; step < N; step *= 3)
#pragma unroll
        for (int i = 0; i + step < N; i += 3 * step)
            v[i] = (i + 2 * step < N) ? __vimax3_s32(v[i], v[i + step], v[i + 2 * step]) : max(v[i], v[i + step]);
    return v[0];
}

// Window of maximal integer sum, lowest start on ties. Every window start k gets
// the key sum*128 + (127 - k): keys order by sum first and, among equal sums,
// prefer the smaller start. All window sums are independent of each other (built
// from pair sums), so the search has no serial dependency chain.
template <int S, int W>
__device__ __forceinline__ int best_key_x(const int (&x)[S], int one, int k128) {
    static_assert(W == 5 || W == 6, "specialised widths");
    constexpr int NK = S - W + 1;
    int p2[S - 1];
#pragma unroll
    for (int k = 0; k < S - 1; ++k) p2[k] = x[k] * one + x[k + 1];          // IMAD: FMA pipe
    int key[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const int sum = (W == 6) ? p2[k] + p2[k + 2] + p2[k + 4] : p2[k] + p2[k + 2] + x[k + 4];
        key[k] = sum * k128 + (127 - k);                                     // IMAD: FMA pipe
    }
    return tree_max(key);
}

template <int S, int W>
__device__ __forceinline__ int best_key_T(const uint16_t* row, int one, int k128) {
    uint32_t w[(S + 1) / 2];
    load_row<S>(row, w);
    int x[S];
#pragma unroll
    for (int k = 0; k < S; ++k) x[k] = sample<S>(w, k);
    return best_key_x<S, W>(x, one, k128);
}

// Maximum W = 6 window sum of one pixel when every loaded 16-bit sample is below
// 4096 (true for 12-bit digitisers; checked here): two samples per 32-bit word,
// pair sums and window sums formed two lanes at a time with plain 32-bit adds
// (each lane stays below 2^15, so no carry crosses a lane), then the maximum
// over both lanes. Rows that start on an odd 16-bit position are read from the
// word boundary below; the lanes then hold windows k - 1 and k instead of k and
// k + 1, and the windows that would reach outside the row are masked. Returns
// false (nothing computed) when a sample is 4096 or more; the window start is
// not computed here.
template <int S>
__device__ __forceinline__ bool max_window6_packed(const uint16_t* row, int& M) {
    constexpr int NK = S - 6 + 1;                 // window starts 0 .. NK - 1
    constexpr int JQ = NK / 2 + 1;                // packed window words
    constexpr int NW = JQ + 3;                    // loaded words
    const uintptr_t a = reinterpret_cast<uintptr_t>(row);
    const bool odd = (S % 2 == 1) && (a & 2u);
    const uint32_t* v = reinterpret_cast<const uint32_t*>(a & ~uintptr_t(3));
    uint32_t u[NW];
    if constexpr ((2 * S) % 16 == 0) {
#pragma unroll
        for (int k = 0; k < NW / 4; ++k) {
            const uint4 q = reinterpret_cast<const uint4*>(v)[k];
            u[4 * k] = q.x; u[4 * k + 1] = q.y; u[4 * k + 2] = q.z; u[4 * k + 3] = q.w;
        }
#pragma unroll
        for (int k = 4 * (NW / 4); k < NW; ++k) u[k] = v[k];
    } else {
#pragma unroll
        for (int k = 0; k < NW; ++k) u[k] = v[k];
    }
    uint32_t any = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) any |= u[k];
    if (any & 0xF000F000u) return false;
    // pair sums: lanes (hi(u_j) + lo(u_j+1) : lo(u_j) + hi(u_j))
    uint32_t P[NW - 1];
#pragma unroll
    for (int j = 0; j < NW - 1; ++j) P[j] = u[j] + __byte_perm(u[j], u[j + 1], 0x5432);
    // the window words, reduced lane by lane with the three-input 16x2 maximum
    // (both lanes at once; masked lanes are 0 and every sum is >= 0), then the
    // larger of the two lanes
    uint32_t m[JQ];
#pragma unroll
    for (int j = 0; j < JQ; ++j) {
        uint32_t q = P[j] + P[j + 1] + P[j + 2];  // lanes: windows (2j + 1 : 2j), or (2j : 2j - 1) for odd rows
        const bool lo_ok = odd ? (j >= 1 && 2 * j <= NK) : (2 * j <= NK - 1);
        const bool hi_ok = odd ? (2 * j <= NK - 1) : (2 * j + 1 <= NK - 1);
        q &= (hi_ok ? 0xFFFF0000u : 0u) | (lo_ok ? 0xFFFFu : 0u);
        m[j] = q;
    }
#pragma unroll
    for (int step = 1; step < JQ; step *= 3)
#pragma unroll
        for (int i = 0; i + step < JQ; i += 3 * step)
            m[i] = __vimax3_u16x2(m[i], m[i + step], i + 2 * step < JQ ? m[i + 2 * step] : 0u);
    M = int(max(m[0] >> 16, m[0] & 0xFFFFu));
    return true;
}

// Two adjacent pixels of an odd sample count S: their 2S samples are S whole
// 32-bit words from a 4-byte-aligned address (the pair starts at an even pixel),
// so every sample sits at a compile-time word and half -- no funnel shifts.
template <int S, int W>
__device__ __forceinline__ void best_key_pair(const uint16_t* row0, int one, int k128, int& key0, int& key1) {
    static_assert(S % 2 == 1, "pairs are for odd sample counts");
    const uint32_t* v = reinterpret_cast<const uint32_t*>(row0);
    uint32_t w[S];
#pragma unroll
    for (int j = 0; j < S; ++j) w[j] = v[j];
    int x[S];
#pragma unroll
    for (int k = 0; k < S; ++k) x[k] = (k & 1) ? int(w[k >> 1] >> 16) : int(w[k >> 1] & 0xFFFFu);
    key0 = best_key_x<S, W>(x, one, k128);
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const int m = S + k;
        x[k] = (m & 1) ? int(w[m >> 1] >> 16) : int(w[m >> 1] & 0xFFFFu);
    }
    key1 = best_key_x<S, W>(x, one, k128);
}

// Bits 0..15 of v spread to the even bit positions.
__device__ __forceinline__ uint32_t spread_even(uint32_t v) {
    v &= 0xFFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

__device__ __forceinline__ int best_key_generic(const uint16_t* row, int S, int W) {
    int s = 0;
    for (int k = 0; k < W; ++k) s += row[k];
    int key = s * 128 + 127;
    for (int k = 1; k + W <= S; ++k) {
        s += int(row[k + W - 1]) - int(row[k - 1]);
        key = max(key, s * 128 + (127 - k));
    }
    return key;
}

// Window start and integer sum of one pixel whose S samples start at `row`
// (shared memory), for the cameras without a specialised search.
__device__ __forceinline__ void window_sum(const uint16_t* row, int S, const ProcParams& pp, int& sum, int& st) {
    const int W = pp.W;
    if (pp.sliding) {
        const int key = best_key_generic(row, S, W);
        sum = key >> 7;
        st = 127 - (key & 127);
    } else {
        st = pp.start;
        sum = 0;
        for (int k = 0; k < W; ++k) sum += row[st + k];
    }
}

// The calibrated charge: exact integer numerator, one FP32 multiply (never fused).
__device__ __forceinline__ float charge(int sum, int W, int p16, float scale, int& num) {
    num = 16 * sum - W * p16;
    return __fmul_rn(__int2float_rn(num), scale);
}

// The digital-filter-style charge over the chosen window: exact 64-bit integer
// numerator 16 * sum_k c_k s[st+k] - (sum_k c_k) * p16, one rounding to FP32, one
// FP32 multiply (never fused). The weights come from the kernel parameters.
__device__ __forceinline__ float filter_charge(const uint16_t* row, int st, int W, const int* wts, int csum, int p16,
                                               float scale) {
    int64_t acc = 0;
    for (int k = 0; k < W; ++k) acc += int64_t(wts[k]) * row[st + k];
    const int64_t num = 16 * acc - int64_t(csum) * p16;
    return __fmul_rn(__ll2float_rn(num), scale);
}

// Pedestal-subtracted sample centroid of the chosen window.
__device__ __forceinline__ float peak_time(const uint16_t* row, int st, int W, int p16, int num) {
    int sj = 0;
    for (int j = 1; j < W; ++j) sj += j * int(row[st + j]);
    const int numt = 16 * sj - p16 * (W * (W - 1) / 2);
    return num > 0 ? __fadd_rn(float(st), __fdiv_rn(__int2float_rn(numt), __int2float_rn(num)))
                   : float(st) + 0.5f * float(W - 1);
}

// ------------------------------------------------------------------ cleaning + Hillas
// Per-image pixel sets are bitmaps of 32-pixel words (word w holds pixels
// 32w..32w+31): hi = {q >= t_hi}, lo = {q >= t_lo}, core, mask. Cleaning and the
// moment sums visit only the set bits, so pixels below t_lo cost nothing after
// integration. Thread w owns word w and visits its bits in increasing order, and
// partial sums are combined by a fixed tree: the summation order depends only on
// the camera, never on the data or on the rest of the batch.
struct NamedBar {
    __device__ __forceinline__ void operator()() const { named_bar_sync(1, NCT); }
};
struct BlockBar {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct WarpBar {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};

struct ImgBits {
    uint32_t* hi;
    uint32_t* lo;
    uint32_t* core;
    uint32_t* mask;
};

__device__ __forceinline__ int words_of(int P) { return (P + 31) >> 5; }

// Reduce N floats over `nthr` threads (nthr/32 warps): warp shuffle tree, then a
// fixed-order sum over warps.
template <int N, class Bar>
__device__ __forceinline__ void block_reduce(float (&v)[N], float* red, int tid, int nthr, Bar bar) {
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = warp_sum(v[k]);
    if (nthr == 32) return;   // one warp: every lane already holds the totals
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) red[warp * 8 + k] = v[k];
    }
    bar();
#pragma unroll
    for (int k = 0; k < N; ++k) {
        float s = 0.f;
        for (int w = 0; w < nthr / 32; ++w) s += red[w * 8 + k];
        v[k] = s;
    }
}

__device__ __forceinline__ bool bit_of(const uint32_t* bits, int id) { return (bits[id >> 5] >> (id & 31)) & 1u; }

// A neighbour id counts only inside [0, P): -1 pads a list, and an id outside
// the camera (possible in caller-supplied tables) is ignored rather than read
// from another image's bitmap words.
__device__ __forceinline__ bool any_neighbour(const int4 nbr, int K, int P, const uint32_t* bits) {
    const int16_t* n = reinterpret_cast<const int16_t*>(&nbr);
    bool any = false;
#pragma unroll
    for (int j = 0; j < RTA_NB_PAD; ++j) {
        const int id = n[j];
        if (j < K && unsigned(id) < unsigned(P) && bit_of(bits, id)) any = true;
    }
    return any;
}

// Tailcut cleaning on the bitmaps: core = hi (with a hi neighbour if asked),
// mask = core | (lo with a core neighbour). Needs hi and lo filled.
template <class Bar>
__device__ __forceinline__ void clean_bits(const DevCam& C, const ProcParams& pp, const ImgBits& b, int tid,
                                           int nthr, Bar bar) {
    const int nw = words_of(C.P);
    for (int w = tid; w < nw; w += nthr) {
        const uint32_t hb = b.hi[w];
        uint32_t cb = hb;
        if (pp.core_nb) {
            cb = 0;
            for (uint32_t m = hb; m; m &= m - 1) {
                const int bit = __ffs(m) - 1;
                if (any_neighbour(__ldg(C.nb + (w * 32 + bit)), C.K, C.P, b.hi)) cb |= 1u << bit;
            }
        }
        b.core[w] = cb;
    }
    bar();
    for (int w = tid; w < nw; w += nthr) {
        const uint32_t cb = b.core[w];
        uint32_t mb = cb;
        for (uint32_t m = b.lo[w] & ~cb; m; m &= m - 1) {
            const int bit = __ffs(m) - 1;
            if (any_neighbour(__ldg(C.nb + (w * 32 + bit)), C.K, C.P, b.core)) mb |= 1u << bit;
        }
        b.mask[w] = mb;
    }
    bar();
}

// Hillas parameters of the pixels in b.mask. Pass 1: size and centroid; pass 2:
// central second moments and psi; pass 3: projections on the principal axes,
// length^2 = sum q l^2 / size and width^2 = sum q w^2 / size, and the time
// gradient. These equal lambda1 and det/lambda1 of the covariance, but stay well
// conditioned in FP32 for nearly collinear images, where det is a small
// difference of large products. Thread 0 writes the row.
template <class Bar>
__device__ __forceinline__ void hillas_bits(const float* q, const float* t, const DevCam& C, const uint32_t* mask,
                                            float* red, int tid, int nthr, Bar bar, rta_hillas_t* out) {
    const int nw = words_of(C.P);
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    for (int w = tid; w < nw; w += nthr)
        for (uint32_t m = mask[w]; m; m &= m - 1) {
            const int p = w * 32 + __ffs(m) - 1;
            const float qp = q[p];
            const float2 xy = __ldg(C.xy + p);
            a[0] += 1.f;
            a[1] += qp;
            a[2] += qp * xy.x;
            a[3] += qp * xy.y;
        }
    block_reduce<4>(a, red, tid, nthr, bar);
    const int n = int(a[0]);
    const float size = a[1];
    if (n == 0 || !(size > 0.f)) {
        if (tid == 0) {
            rta_hillas_t h = {};
            h.n_pix = n;
            h.flags = RTA_HF_EMPTY | RTA_HF_NO_TIME;
            *out = h;
        }
        return;
    }
    const float cx = __fdiv_rn(a[2], size), cy = __fdiv_rn(a[3], size);
    float b[4] = {0.f, 0.f, 0.f, 0.f};
    for (int w = tid; w < nw; w += nthr)
        for (uint32_t m = mask[w]; m; m &= m - 1) {
            const int p = w * 32 + __ffs(m) - 1;
            const float qp = q[p];
            const float2 xy = __ldg(C.xy + p);
            const float dx = xy.x - cx, dy = xy.y - cy;
            b[0] += qp * dx * dx;
            b[1] += qp * dy * dy;
            b[2] += qp * dx * dy;
            if (t) b[3] += qp * t[p];
        }
    block_reduce<4>(b, red + NCW * 8 * 2, tid, nthr, bar);
    const float psi = 0.5f * atan2f(2.f * b[2], b[0] - b[1]);
    const float tmean = t ? __fdiv_rn(b[3], size) : 0.f;
    float sp, cp;
    sincosf(psi, &sp, &cp);
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    for (int w = tid; w < nw; w += nthr)
        for (uint32_t m = mask[w]; m; m &= m - 1) {
            const int p = w * 32 + __ffs(m) - 1;
            const float qp = q[p];
            const float2 xy = __ldg(C.xy + p);
            const float dx = xy.x - cx, dy = xy.y - cy;
            const float l = dx * cp + dy * sp;
            const float wd = dy * cp - dx * sp;
            c[0] += qp * l * l;
            c[1] += qp * wd * wd;
            if (t) c[2] += qp * l * (t[p] - tmean);
        }
    block_reduce<4>(c, red + NCW * 8 * 1, tid, nthr, bar);
    uint32_t flags = 0;
    float grad = 0.f;
    if (t && n >= 2) grad = c[0] > 0.f ? __fdiv_rn(c[2], c[0]) : 0.f;
    else flags |= RTA_HF_NO_TIME;
    if (tid == 0) {
        rta_hillas_t h;
        h.size = size;
        h.x = cx;
        h.y = cy;
        h.length = sqrtf(__fdiv_rn(c[0], size));
        h.width = sqrtf(__fdiv_rn(c[1], size));
        h.psi = psi;
        h.r = sqrtf(cx * cx + cy * cy);
        h.phi = atan2f(cy, cx);
        h.time_grad = grad;
        h.time_mean = tmean;
        h.n_pix = n;
        h.flags = flags;
        h.reserved[0] = h.reserved[1] = h.reserved[2] = h.reserved[3] = 0.f;
        *out = h;
    }
}

// The cleaning mask of one image as one byte per pixel at rows pix_off[img] ..
// pix_off[img] + P - 1 (the per-pixel output of the general instantiations);
// an image whose rows do not fit n_q is flagged and not written.
__device__ __forceinline__ void write_mask(const ChainArgs& a, const DevCam& C, const uint32_t* mask, int img,
                                           int lane) {
    const int64_t off = a.pix_off[img];
    if (off < 0 || off + C.P > a.n_q) {
        if (lane == 0) atomicOr(a.status, RTA_DEV_BAD_IMAGE);
        return;
    }
    for (int p = lane; p < C.P; p += 32) a.mask_out[off + p] = bit_of(mask, p) ? 1 : 0;
}

__device__ __forceinline__ void write_bad_row(rta_hillas_t* out) {
    rta_hillas_t h = {};
    h.flags = RTA_HF_BAD_INPUT | RTA_HF_EMPTY | RTA_HF_NO_TIME;
    *out = h;
}

// ------------------------------------------------------------------ the fused persistent kernel
// Warp roles: warp 0 producer, warps 1..IW integrators, warp IW+1 the tail warp.
// Tile shape: IW integrator warps, each thread integrating PPT pixels of a chunk
// of IW*32*PPT pixels (thread i takes pixels i, i + IW*32, ...), so the per-chunk
// bookkeeping is shared by PPT pixels and each thread has PPT independent window
// searches in flight. Integrated images go through two shared-memory slots (q, t
// and the hi/lo bitmaps of one image each): the integrators fill one slot while
// the tail warp cleans and parameterises the other.
constexpr int NSLOT = 2;
enum { SLOT_END = 1 };

struct SlotHdr {
    int img, cam, flags, pad;
};

struct ChainSmem {
    uint64_t full[MAX_STAGES];
    uint64_t empty[MAX_STAGES];
    uint64_t slot_full[NSLOT];
    uint64_t slot_free[NSLOT];
    StageHdr hdr[MAX_STAGES];
    SlotHdr shdr[NSLOT];
    uint64_t nb_ready;    // neighbour-peak window: every warp has written this image's keys
    uint64_t nb_free;     // ... and has read them (the next image may overwrite)
    int nb_cnt[2];        // candidates of the current and the next image
    int abort;
    int pad[25];
    float red[8];
    int wts[RTA_MAX_W];   // weights of the digital-filter-style extractor
};

struct SlotView {
    float* q;
    float* t;
    uint32_t* hi;
    uint32_t* lo;
};

__host__ __device__ __forceinline__ size_t slot_bytes(int max_P) {
    return size_t(max_P) * 8 + size_t(8) * ((max_P + 31) / 32);
}

// Pixels of camera S per stage: a multiple of 32 (chunks start on bitmap words)
// that fits the stage's waveform area with 16 bytes of slack for the unaligned
// row loads of odd sample counts.
__host__ __device__ __forceinline__ int chunk_pixels(int chunk, int stage_wave_bytes, int S) {
    const int cp = ((stage_wave_bytes - 16) / (2 * S)) & ~31;
    return cp < chunk ? cp : chunk;
}

// Neighbour-peak window. Per chunk, every pixel's own sliding window and the
// charge q0 it gives go into a 64-bit key ordered by charge, then by earliest
// start (the charge's IEEE bits mapped to an unsigned order; never NaN, the
// calibration scales are finite and positive). After the image's last chunk,
// a candidate pass gives every pixel that needs a charge the start of the
// largest key of its closed neighbourhood and integrates its own samples there,
// re-read from L2 (the image streamed in a moment earlier with an evict-last
// hint).
//
// A pixel's charge in any window is at most q0 (the scales are positive), so a
// pixel with q0 < t_lo cannot pass cleaning whatever its window, and it never
// outranks a neighbour that can: the image chain needs exact starts and final
// charges only where q0 >= t_lo. Those pixels are the candidates; the packed
// maximum gives q0 for the rest, whose stored start is never used. The
// integrate-only outputs need every pixel's charge, so there every start is
// exact and every pixel goes through the candidate pass.
__device__ __forceinline__ uint64_t nb_key(float q, int st) {
    const uint32_t b = __float_as_uint(__fadd_rn(q, 0.0f));          // -0 -> +0
    const uint32_t o = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    return (uint64_t(o) << 32) | uint32_t(0xFFFFFFFFu - uint32_t(st));
}

struct NbShared {
    uint64_t* key;        // [max_P] this image's keys
    int16_t* cand;        // [max_P] candidate pixels (image chain)
    int* n_cand;          // candidates so far in this image
};

template <int S, int W, int IT, int PPT, bool NO_INTEG>
__device__ __forceinline__ void nb_keys_chunk(const ChainArgs& a, const ProcParams& pp, const StageHdr& h,
                                              const unsigned char* buf, const int32_t* cp16, const float* cscale,
                                              const NbShared& nb, const SlotView& v, int ct, int lane) {
    const int Sr = S ? S : h.S;
    const int Wr = W ? W : pp.W;
    const bool integ = !NO_INTEG && a.integrate_only;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int c = ct + k * IT;
        bool cand = false;
        if (c < h.npix) {
            const uint16_t* row = reinterpret_cast<const uint16_t*>(buf) + size_t(c) * Sr;
            int num;
            float q0 = 0.f;
            int st = 0;
            bool exact = true;
            if constexpr (S != 0 && W == 6) {
                int m = 0;
                if (!integ && max_window6_packed<S>(row, m)) {
                    q0 = charge(m, Wr, cp16[c], cscale[c], num);
                    exact = q0 >= pp.t_lo;
                }
            }
            if (exact) {
                int key;
                if constexpr (S != 0) key = best_key_T<S, W>(row, pp.one, pp.k128);
                else key = best_key_generic(row, Sr, Wr);
                q0 = charge(key >> 7, Wr, cp16[c], cscale[c], num);
                st = 127 - (key & 127);
            }
            nb.key[h.base + c] = nb_key(q0, st);
            cand = !integ && q0 >= pp.t_lo;
        }
        if (!integ) {
            // append the candidates (one atomic per warp); the chunk's bitmap words
            // start empty and the candidate pass sets their bits
            const uint32_t bc = __ballot_sync(0xffffffffu, cand);
            int base = 0;
            if (lane == 0 && bc) base = atomicAdd(nb.n_cand, __popc(bc));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (cand) nb.cand[base + __popc(bc & ((1u << lane) - 1u))] = int16_t(h.base + c);
            const int word = (h.base + c) >> 5;
            if (lane == 0 && word < ((h.base + h.npix + 31) >> 5)) {      // only the chunk's own words
                v.hi[word] = 0u;
                v.lo[word] = 0u;
            }
        }
    }
}

// The candidate pass of one image: pixel p takes the start of the largest key
// among itself and its registered neighbours, then its own flat sum there, the
// calibration multiply and the peak time; in the image chain q, t and the
// bitmap bits go to the slot.
template <bool NO_INTEG>
__device__ __forceinline__ void nb_pixel(const ChainArgs& a, const ProcParams& pp, const StageHdr& h, const DevCam& C,
                                         const uint64_t* key, int p, const SlotView& v) {
    uint64_t best = key[p];
    const int4 nbr = C.nb[p];
    const int16_t* ids = reinterpret_cast<const int16_t*>(&nbr);
#pragma unroll
    for (int j = 0; j < RTA_NB_PAD; ++j) {
        const int id = ids[j];
        if (j < C.K && id >= 0 && id < h.P) {
            const uint64_t kn = key[id];
            best = kn > best ? kn : best;
        }
    }
    const int wst = int(0xFFFFFFFFu - uint32_t(best));
    const int Wr = pp.W;
    const uint16_t* row;                                           // global memory (L2)
    if (a.seg) {
        int k = h.seg0;
        while (k + 1 < h.seg1 && p >= a.seg[k].first_pixel + a.seg[k].n_pixels) ++k;
        row = a.wave + a.seg[k].offset / 2 + size_t(p - a.seg[k].first_pixel) * h.S;
    } else {
        row = a.wave + h.woff + size_t(p) * h.S;
    }
    int sum = 0;
    for (int j = 0; j < Wr; ++j) sum += __ldg(row + wst + j);
    const int p16 = __ldg(a.arr.p16 + h.row + p);
    int num;
    const float q = charge(sum, Wr, p16, __ldg(a.arr.scale + h.row + p), num);
    if (!NO_INTEG && a.integrate_only) {
        a.q_out[h.pix_off + p] = q;
        if (a.t_out) a.t_out[h.pix_off + p] = peak_time(row, wst, Wr, p16, num);
    } else {
        v.q[p] = q;
        const uint32_t bit = 1u << (p & 31);
        if (q >= pp.t_hi) atomicOr(&v.hi[p >> 5], bit);
        if (q >= pp.t_lo) {
            atomicOr(&v.lo[p >> 5], bit);
            v.t[p] = peak_time(row, wst, Wr, p16, num);
        }
    }
}

// This thread's pixels of one chunk: window search, the calibration multiply,
// and either the integrate-only outputs or the slot values (q, and t for pixels
// that can survive cleaning) and the hi/lo bitmap words. S and W are
// compile-time for the specialised sliding-window cameras (the camera is the
// same for the whole chunk, so the dispatch happens once per chunk); S == 0 is
// the generic path with run-time S and W.
template <int S, int W, int IT, int PPT, bool NO_INTEG, bool NO_FILTER>
__device__ __forceinline__ void integrate_chunk(const ChainArgs& a, const ProcParams& pp, const StageHdr& h,
                                                const unsigned char* buf, const int32_t* cp16, const float* cscale,
                                                const SlotView& v, int ct, int lane, const int* wts) {
    const int Sr = S ? S : h.S;
    const int Wr = W ? W : pp.W;
    // NO_INTEG / NO_FILTER: instantiations that never see the integrate-only call
    // or the digital filter leave those branches out of their code
    const bool integ = !NO_INTEG && a.integrate_only;
    const bool filt = !NO_FILTER && pp.filter;
    // charge, outputs and thresholds of chunk pixel c with window sum `sum` starting at `wst`
    auto emit = [&](int c, int sum, int wst, const uint16_t* row, bool& hi, bool& lo) {
        const int p16 = cp16[c];
        int num;
        float q = charge(sum, Wr, p16, cscale[c], num);
        if (filt) q = filter_charge(row, wst, Wr, wts, pp.csum, p16, cscale[c]);
        const int p = h.base + c;
        if (integ) {
            a.q_out[h.pix_off + p] = q;
            if (a.t_out) a.t_out[h.pix_off + p] = peak_time(row, wst, Wr, p16, num);
        } else {
            v.q[p] = q;
            hi = q >= pp.t_hi;
            lo = q >= pp.t_lo;
            // only pixels that can survive cleaning need their time
            if (lo) v.t[p] = peak_time(row, wst, Wr, p16, num);
        }
    };
    if constexpr (S != 0 && S % 2 == 1 && PPT == 2) {
        // adjacent pixel pairs 2ct, 2ct + 1 (P is a multiple of 8 for odd S, so
        // chunks hold whole pairs); the warp covers 64 consecutive pixels
        const int c0 = 2 * ct;
        bool hi0 = false, lo0 = false, hi1 = false, lo1 = false;
        if (c0 < h.npix) {
            const uint16_t* row0 = reinterpret_cast<const uint16_t*>(buf) + size_t(c0) * S;
            int key0, key1;
            best_key_pair<S, W>(row0, pp.one, pp.k128, key0, key1);
            emit(c0, key0 >> 7, 127 - (key0 & 127), row0, hi0, lo0);
            emit(c0 + 1, key1 >> 7, 127 - (key1 & 127), row0 + S, hi1, lo1);
        }
        if (!integ) {
            const uint32_t h0 = __ballot_sync(0xffffffffu, hi0), h1 = __ballot_sync(0xffffffffu, hi1);
            const uint32_t l0 = __ballot_sync(0xffffffffu, lo0), l1 = __ballot_sync(0xffffffffu, lo1);
            const int word = (h.base + 64 * (ct >> 5)) >> 5;
            const int nw = (h.base + h.npix + 31) >> 5;      // only the chunk's own words
            if (lane == 0 && word < nw) {
                v.hi[word] = spread_even(h0) | (spread_even(h1) << 1);
                v.lo[word] = spread_even(l0) | (spread_even(l1) << 1);
            }
            if (lane == 0 && word + 1 < nw) {
                v.hi[word + 1] = spread_even(h0 >> 16) | (spread_even(h1 >> 16) << 1);
                v.lo[word + 1] = spread_even(l0 >> 16) | (spread_even(l1 >> 16) << 1);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int c = ct + k * IT;    // pixel within the chunk
            bool hi = false, lo = false;
            if (c < h.npix) {
                const uint16_t* row = reinterpret_cast<const uint16_t*>(buf) + size_t(c) * Sr;
                int sum = 0, wst = 0;
                bool done = false;
                if constexpr (S != 0 && W == 6) {
                    // The charge needs only the maximum; the window start (first
                    // maximum) only for pixels whose peak time is needed. The packed
                    // maximum decides: below t_lo its charge is the pixel's whole
                    // result (no time, no bits); the exact search (one call site)
                    // runs for the pixels that reach t_lo or whose samples are out of
                    // its range.
                    int m = 0;
                    if (!integ && !filt && max_window6_packed<S>(row, m)) {
                        const float q0 = __fmul_rn(__int2float_rn(16 * m - W * cp16[c]), cscale[c]);
                        if (q0 < pp.t_lo) {
                            v.q[h.base + c] = q0;
                            done = true;
                        }
                    }
                    if (!done) {
                        const int key = best_key_T<S, W>(row, pp.one, pp.k128);
                        sum = key >> 7;
                        wst = 127 - (key & 127);
                    }
                } else if constexpr (S != 0) {
                    const int key = best_key_T<S, W>(row, pp.one, pp.k128);
                    sum = key >> 7;
                    wst = 127 - (key & 127);
                } else {
                    window_sum(row, h.S, pp, sum, wst);
                }
                if (!done) emit(c, sum, wst, row, hi, lo);
            }
            if (!integ) {
                const uint32_t bh = __ballot_sync(0xffffffffu, hi), bl = __ballot_sync(0xffffffffu, lo);
                const int word = (h.base + c) >> 5;
                if (lane == 0 && word < ((h.base + h.npix + 31) >> 5)) {      // only the chunk's own words
                    v.hi[word] = bh;
                    v.lo[word] = bl;
                }
            }
        }
    }
}

// The chunk's pixels [base, base + npix) of a byte-stream image from the
// segment(s) that hold them (segment and chunk boundaries are multiples of 8
// samples: 16-byte copies); seg is the segment to start looking at, returned
// for the next chunk. m: the image's record in shared memory.
static __device__ __forceinline__ int stream_chunk_copy(const ChainArgs& a, const StreamImg* m, int seg, int base,
                                                     int npix, int S, unsigned char* buf, uint64_t* bar,
                                                     uint64_t pol) {
    int done = 0;
    while (done < npix) {
        int first, n;
        long long off;
        if (seg < STREAM_INLINE_SEGS) {
            first = m->first[seg];
            n = m->n[seg];
            off = m->off[seg];
        } else {
            const rta_segment_t sg = a.seg[m->seg0 + seg];
            first = sg.first_pixel;
            n = sg.n_pixels;
            off = sg.offset;
        }
        const int p0 = base + done;
        if (p0 >= first + n) {
            ++seg;
            continue;
        }
        const int take = min(npix - done, first + n - p0);
        bulk_g2s(buf + size_t(done) * S * 2, a.wave + off / 2 + size_t(p0 - first) * S,
                 uint32_t(take) * uint32_t(S) * 2u, bar, pol);
        done += take;
    }
    return seg;
}

// NB: the neighbour-peak window (keys and candidates in shared memory, a
// candidate pass after each image). STREAM: a byte-stream bundle (per-image
// records from k_stream_meta, chunks copied from the stream's segments). LEAN:
// the image chain only, without the integrate-only outputs and the digital
// filter; FILT: the image chain with the digital filter, without the
// integrate-only outputs. Each combination is a separate instantiation, so that
// every kernel carries only the code of the calls it serves (branches left in,
// even untaken, cost the hot loop instruction-cache misses and scheduling).
template <int IW, int PPT, int MB, bool NB, bool STREAM = false, bool LEAN = false, bool FILT = false>
__global__ void __launch_bounds__(IW * 32 + 64, MB) k_image_chain(const ChainArgs a) {
    static_assert(!(LEAN && FILT) && !(NB && FILT), "the filter form is of the flat-window chain");
    constexpr bool NO_INTEG = LEAN || STREAM || FILT;     // STREAM: never integrate-only
    const bool integ = !NO_INTEG && a.integrate_only;
    constexpr int IT = IW * 32;          // integrator threads
    constexpr int CHUNK = IT * PPT;      // largest chunk in pixels
    extern __shared__ __align__(128) unsigned char smem_raw[];
    ChainSmem& sm = *reinterpret_cast<ChainSmem*>(smem_raw);
    const size_t head = (sizeof(ChainSmem) + 127) & ~size_t(127);
    const int NST = a.nstage;
    const int calib_bytes = CHUNK * 4;
    const int stage_bytes = a.stage_wave_bytes + 2 * calib_bytes;
    unsigned char* stages = smem_raw + head;
    const int maxP = a.arr.max_P;
    const int maxw = words_of(maxP);
    unsigned char* slots = stages + size_t(NST) * stage_bytes;
    auto slot_view = [&](int s) {
        unsigned char* b = slots + size_t(s) * slot_bytes(maxP);
        SlotView v;
        v.q = reinterpret_cast<float*>(b);
        v.t = v.q + maxP;
        v.hi = reinterpret_cast<uint32_t*>(v.t + maxP);
        v.lo = v.hi + maxw;
        return v;
    };
    uint32_t* core = reinterpret_cast<uint32_t*>(slots + NSLOT * slot_bytes(maxP));
    uint32_t* maskb = core + maxw;
    // neighbour-peak keys and candidates of the image being integrated
    uint64_t* nbk = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(maskb + maxw) + 15) & ~uintptr_t(15));
    int16_t* nbc = reinterpret_cast<int16_t*>(nbk + maxP);
    // byte stream: the records of the image whose chunks the producer issues and of
    // the next one, copied in by cp.async one image ahead (after the keys, if any)
    StreamImg* srec = reinterpret_cast<StreamImg*>(
        (reinterpret_cast<uintptr_t>(NB ? static_cast<void*>(nbc + maxP) : static_cast<void*>(nbk)) + 15) &
        ~uintptr_t(15));
    volatile int* abort_flag = &sm.abort;

    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], IW);
        }
        for (int s = 0; s < NSLOT; ++s) {
            mbar_init(&sm.slot_full[s], IW);
            mbar_init(&sm.slot_free[s], 1);
        }
        if (NB) {
            mbar_init(&sm.nb_ready, IW);
            mbar_init(&sm.nb_free, IW);
            sm.nb_cnt[0] = sm.nb_cnt[1] = 0;
        }
        sm.abort = 0;
        fence_mbar_init();
    }
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < RTA_MAX_W; ++k) sm.wts[k] = a.pp.wts[k];   // constant indices: no copy of the parameters
    }
    __syncthreads();

    if (tid < 32) {
        // ---------------- producer warp: lane 0 issues everything
        if (tid != 0) return;
        // a graph captured at capacity reads the bundle's image count at run time
        const int64_t n_img = a.n_img_dev ? min(*a.n_img_dev, a.n_img) : a.n_img;
        const uint64_t pol_stream = l2_policy_evict_first();
        const uint64_t pol_keep = l2_policy_evict_last();
        int stage = 0;
        uint32_t phase = 0;
        uint32_t pending = 0;          // stages whose copy is issued and not yet seen free again
        uint32_t pend_par[MAX_STAGES];
        bool ok = true;
        auto acquire = [&](int s, uint32_t ph) -> bool {
            if (!mbar_wait(&sm.empty[s], ph ^ 1u, abort_flag)) return false;
            pending &= ~(1u << s);
            return true;
        };
        // the next image is taken, and its table entries loaded, while the current
        // image's chunks are issued: neither the work counter's atomic nor those
        // loads wait at an image boundary
        constexpr bool stream_mode = STREAM;
        int64_t next = atomicAdd(a.counter, 1u);
        int next_tel = -1;
        int64_t next_woff = 0;
        int rec_next = 0;              // byte stream: the record buffer the next image's record goes to
        static_assert(sizeof(StreamImg) % 16 == 0, "records copy in 16-byte pieces");
        auto fetch_next = [&]() {
            if (next >= n_img) return;
            if (stream_mode) {
                const int4* src = reinterpret_cast<const int4*>(a.smeta + next);
                int4* dst = reinterpret_cast<int4*>(srec + rec_next);
#pragma unroll
                for (int k = 0; k < int(sizeof(StreamImg) / 16); ++k) cp_async16(dst + k, src + k);
            } else {
                next_tel = a.img_tel[next];
                next_woff = a.wave_off[next];
            }
        };
        fetch_next();
        for (;;) {
            const int64_t img = next;
            const int tel = next_tel;
            const int64_t woff = next_woff;
            const StreamImg* rec = nullptr;
            if (stream_mode) {
                cp_async_wait_all();       // this image's record (copied one image ago) has landed
                rec = srec + rec_next;
                rec_next ^= 1;
            }
            if (img < n_img) {
                next = atomicAdd(a.counter, 1u);
                fetch_next();
            }
            if (img >= n_img) {
                grid_dependents_launch();    // no image left to take: the next kernel may be scheduled
                if (!acquire(stage, phase)) { ok = false; break; }
                StageHdr h = {};
                h.img = -1;
                h.flags = HDR_END;
                sm.hdr[stage] = h;
                mbar_arrive(&sm.full[stage]);
                break;
            }
            bool bad;
            int P, S, cam;
            int64_t row;
            int64_t poff = 0;
            int seg0 = 0, seg1 = 0;
            if (stream_mode) {
                // checked by k_stream_meta
                bad = rec->ok == 0;
                cam = rec->cam;
                seg0 = rec->seg0;
                seg1 = rec->seg0 + rec->nseg;
                row = rec->row;
                P = rec->P;
                S = rec->S;
            } else {
                bad = tel < 0 || tel >= a.arr.n_tel || woff < 0 || (woff & 7) != 0;
                cam = 0;
                P = S = 0;
                row = 0;
                if (!bad) {
                    cam = a.arr.tel_cam[tel];
                    const DevCam C = a.arr.cams[cam];
                    P = C.P;
                    S = C.S;
                    row = a.arr.tel_row[tel];
                    bad = woff + int64_t(P) * S > a.n_wave;   // never read past the waveform buffer
                }
            }
            if (!bad && integ) {
                poff = a.pix_off[img];
                bad = poff < 0 || poff + P > a.n_q;            // never write past q / t
            }
            if (bad) {
                if (!acquire(stage, phase)) { ok = false; break; }
                StageHdr h = {};
                h.img = int(img);
                h.flags = HDR_BAD | HDR_LAST;
                sm.hdr[stage] = h;
                mbar_arrive(&sm.full[stage]);
                if (++stage == NST) { stage = 0; phase ^= 1u; }
                continue;
            }
            const int CP = chunk_pixels(CHUNK, a.stage_wave_bytes, S);
            const uint16_t* src = a.wave + woff;
            int cur_seg = 0;
            for (int base = 0; base < P; base += CP) {
                if (!acquire(stage, phase)) { ok = false; break; }
                const int npix = min(CP, P - base);
                StageHdr h;
                h.img = int(img);
                h.base = base;
                h.npix = npix;
                h.flags = (base + CP >= P) ? HDR_LAST : 0;
                h.P = P;
                h.S = S;
                h.cam = cam;
                h.seg0 = seg0;
                h.seg1 = seg1;
                h.pad = 0;
                h.pix_off = poff;
                h.woff = woff;
                h.row = row;
                sm.hdr[stage] = h;
                const uint32_t wbytes = uint32_t(npix) * uint32_t(S) * 2u;     // multiple of 16 (P*S % 8 == 0)
                const uint32_t cbytes = (uint32_t(npix) * 4u + 15u) & ~15u;
                unsigned char* buf = stages + size_t(stage) * stage_bytes;
                mbar_arrive_expect_tx(&sm.full[stage], wbytes + 2u * cbytes);
                // the neighbour-peak window reads its candidates' samples once more right
                // after the image: keep the image in L2 until then
                const uint64_t pol = NB ? pol_keep : pol_stream;
                if (stream_mode) {
                    cur_seg = stream_chunk_copy(a, rec, cur_seg, base, npix, S, buf, &sm.full[stage], pol);
                } else {
                    bulk_g2s(buf, src + size_t(base) * S, wbytes, &sm.full[stage], pol);
                }
                bulk_g2s(buf + a.stage_wave_bytes, a.arr.p16 + row + base, cbytes, &sm.full[stage], pol_keep);
                bulk_g2s(buf + a.stage_wave_bytes + calib_bytes, a.arr.scale + row + base, cbytes, &sm.full[stage],
                         pol_keep);
                pending |= 1u << stage;
                pend_par[stage] = phase;
                if (++stage == NST) { stage = 0; phase ^= 1u; }
            }
            if (!ok) break;
        }
        if (!ok) {
            atomicOr(a.status, RTA_DEV_TIMEOUT);
            *abort_flag = 1;
            // drain: every copy still in flight must land before the CTA exits
            for (int s = 0; s < NST; ++s)
                if (pending & (1u << s)) {
                    const uint64_t t0 = global_ns();
                    while (!mbar_try_wait(&sm.full[s], pend_par[s]))
                        if (global_ns() - t0 > RTA_WAIT_TIMEOUT_NS) break;
                }
        }
        if constexpr (STREAM) cp_async_wait_all();   // a record copy after an abort lands first too
        return;
    }

    const int lane = tid & 31;
    const ProcParams pp = a.pp;
    auto give_up = [&]() {
        if (!*abort_flag) atomicOr(a.status, RTA_DEV_TIMEOUT);
        *abort_flag = 1;
    };

    if (tid >= 32 + IT) {
        // ---------------- tail warp: cleaning + Hillas of integrated images
        int slot = 0;
        uint32_t ph = 0;
        for (;;) {
            if (!mbar_wait(&sm.slot_full[slot], ph, abort_flag)) { give_up(); break; }
            const SlotHdr sh = sm.shdr[slot];
            if (sh.flags & SLOT_END) break;
            const SlotView v = slot_view(slot);
            const DevCam C = a.arr.cams[sh.cam];
            const ImgBits ib = {v.hi, v.lo, core, maskb};
            clean_bits(C, pp, ib, lane, 32, WarpBar());
            if constexpr (!NO_INTEG) {
                if (a.mask_out) write_mask(a, C, maskb, sh.img, lane);
            }
            hillas_bits(v.q, v.t, C, maskb, sm.red, lane, 32, WarpBar(), a.out + sh.img);
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.slot_free[slot]);
            if (++slot == NSLOT) { slot = 0; ph ^= 1u; }
        }
        return;
    }

    // ---------------- integrator warps
    const int ct = tid - 32;          // 0 .. IT-1
    int stage = 0, slot = 0;
    uint32_t phase = 0, sphase = 0;
    uint32_t nb_rph = 0, nb_fph = 0;  // neighbour-peak barrier phases
    int nb_img = 0;                   // neighbour-peak images done by this CTA
    SlotView v = slot_view(0);
    for (;;) {
        if (!mbar_wait(&sm.full[stage], phase, abort_flag)) { give_up(); break; }
        const StageHdr h = sm.hdr[stage];
        if (h.flags & HDR_END) {
            // tell the tail warp there is nothing more
            if (!mbar_wait(&sm.slot_free[slot], sphase ^ 1u, abort_flag)) { give_up(); break; }
            if (ct == 0) sm.shdr[slot].flags = SLOT_END;
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.slot_full[slot]);
            break;
        }
        if (h.flags & HDR_BAD) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.empty[stage]);
            if (ct == 0) {
                atomicOr(a.status, RTA_DEV_BAD_IMAGE);
                if (!integ) write_bad_row(a.out + h.img);
            }
            if (++stage == NST) { stage = 0; phase ^= 1u; }
            continue;
        }
        if (NB && h.base == 0 && nb_img > 0) {
            // this image's keys and candidates overwrite the previous image's:
            // every warp must be done with those
            if (!mbar_wait(&sm.nb_free, nb_fph, abort_flag)) { give_up(); break; }
            nb_fph ^= 1u;
        }
        if (h.base == 0 && !integ) {
            // the slot must be free: the tail warp is done with the image two back
            if (!mbar_wait(&sm.slot_free[slot], sphase ^ 1u, abort_flag)) { give_up(); break; }
        }
        const unsigned char* buf = stages + size_t(stage) * stage_bytes;
        const int32_t* cp16 = reinterpret_cast<const int32_t*>(buf + a.stage_wave_bytes);
        const float* cscale = reinterpret_cast<const float*>(buf + a.stage_wave_bytes + calib_bytes);
        if constexpr (NB) {
            // per image two counters in turn: the one of the image before is reset
            // during this image's candidate pass, after every warp has passed nb_free
            const NbShared nb = {nbk, nbc, &sm.nb_cnt[nb_img & 1]};
            if (pp.W == 6 && h.S == 40)
                nb_keys_chunk<40, 6, IT, PPT, NO_INTEG>(a, pp, h, buf, cp16, cscale, nb, v, ct, lane);
            else if (pp.W == 6 && h.S == 30)
                nb_keys_chunk<30, 6, IT, PPT, NO_INTEG>(a, pp, h, buf, cp16, cscale, nb, v, ct, lane);
            else if (pp.W == 6 && h.S == 25)
                nb_keys_chunk<25, 6, IT, PPT, NO_INTEG>(a, pp, h, buf, cp16, cscale, nb, v, ct, lane);
            else
                nb_keys_chunk<0, 0, IT, PPT, NO_INTEG>(a, pp, h, buf, cp16, cscale, nb, v, ct, lane);
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.empty[stage]);
            if (++stage == NST) { stage = 0; phase ^= 1u; }
            if (h.flags & HDR_LAST) {
                // every key, candidate and bitmap word of the image is written...
                if (lane == 0) mbar_arrive(&sm.nb_ready);
                if (!mbar_wait(&sm.nb_ready, nb_rph, abort_flag)) { give_up(); break; }
                nb_rph ^= 1u;
                // ...so the candidate pass can look at any pixel's neighbours
                const DevCam C = a.arr.cams[h.cam];
                if (integ) {
                    for (int p = ct; p < h.P; p += IT) nb_pixel<NO_INTEG>(a, pp, h, C, nbk, p, v);
                } else {
                    const int n = *nb.n_cand;
                    for (int j = ct; j < n; j += IT) nb_pixel<NO_INTEG>(a, pp, h, C, nbk, nbc[j], v);
                }
                if (ct == 0) sm.nb_cnt[(nb_img + 1) & 1] = 0;
                ++nb_img;
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.nb_free);
            }
        } else {
            if (pp.sliding && pp.W == 6 && h.S == 40)
                integrate_chunk<40, 6, IT, PPT, NO_INTEG, LEAN>(a, pp, h, buf, cp16, cscale, v, ct, lane, sm.wts);
            else if (pp.sliding && pp.W == 6 && h.S == 30)
                integrate_chunk<30, 6, IT, PPT, NO_INTEG, LEAN>(a, pp, h, buf, cp16, cscale, v, ct, lane, sm.wts);
            else if (pp.sliding && pp.W == 6 && h.S == 25)
                integrate_chunk<25, 6, IT, PPT, NO_INTEG, LEAN>(a, pp, h, buf, cp16, cscale, v, ct, lane, sm.wts);
            else if (pp.sliding && pp.W == 5 && h.S == 16)
                integrate_chunk<16, 5, IT, PPT, NO_INTEG, LEAN>(a, pp, h, buf, cp16, cscale, v, ct, lane, sm.wts);
            else
                integrate_chunk<0, 0, IT, PPT, NO_INTEG, LEAN>(a, pp, h, buf, cp16, cscale, v, ct, lane, sm.wts);
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.empty[stage]);
            if (++stage == NST) { stage = 0; phase ^= 1u; }
        }
        if ((h.flags & HDR_LAST) && !integ) {
            if (ct == 0) {
                SlotHdr sh;
                sh.img = h.img;
                sh.cam = h.cam;
                sh.flags = 0;
                sh.pad = 0;
                sm.shdr[slot] = sh;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.slot_full[slot]);
            if (++slot == NSLOT) { slot = 0; sphase ^= 1u; }
            v = slot_view(slot);
        }
    }
}

}  // namespace rta
