// Inference of the deep-sets surrogate (energy, direction offset and
// gamma/hadron score next to the geometric direction, Sec. 4.1), in two kernels:
//
//   k_tel    one warp per four events, no block barrier after the weights are
//            staged: per-event baseline and used images (eight lanes per
//            event), per-image features, the per-telescope network
//            16 -> 128 -> 128 (ReLU) on the tensor cores (mma.sync m16n8k16,
//            BF16 operands, FP32 accumulators) sixteen image rows at a time --
//            the first layer's accumulators become the second layer's A
//            fragments in registers, the weights reach the MMA from shared
//            memory by ldmatrix.trans -- and the sum / mean pooling in
//            registers. Writes the pooled vectors, baselines and used counts.
//   k_event  one persistent CTA per SM walks tiles of up to 32 events: the
//            event network 256 -> 256 (ReLU, weights staged once per CTA) and
//            256 -> 4 on the tensor cores, then the outputs and the fallback
//            list for the geometric intersection. The next tile's pooled rows
//            arrive by cp.async while the current one computes.
//
// Every stage evaluates the same expressions in the same order as the
// layer-by-layer kernels of the training path (k_features, k_gemm, k_pool,
// k_head in k_mlp.cu): the features and the eight-lane event reductions, the
// k-order of each MMA accumulation, the image order of the pooling sums (an
// unused image adds +0 here where the pooling kernel skips it, which leaves a
// sum unchanged). The outputs therefore equal those of the training-path
// forward bit for bit.
#include <algorithm>

#include "rta_mlp_dev.cuh"

namespace rta {
namespace {

constexpr int FE = 32;              // events per k_event tile at most
constexpr int NT = 256;             // threads per CTA (both kernels)
constexpr int EPW = 32 / SUR_EVT_LANES;   // events per k_tel warp iteration
constexpr int LDX = 24;             // feature row stride (16 + 8: conflict-free fragment loads)
constexpr int LDH = SUR_H + 8;      // hidden row stride (conflict-free ldmatrix / fragment loads)
constexpr int LDV = SUR_G + 8;      // pooled / event-network row stride

// k_tel shared memory: weights, then per warp a 16-row feature tile and a
// 16-row hidden tile
constexpr size_t TS_W1 = 0;                                      // bf16 [16][LDH]
constexpr size_t TS_W2 = TS_W1 + size_t(SUR_XPAD) * LDH * 2;     // bf16 [128][LDH]
constexpr size_t TS_B = TS_W2 + size_t(SUR_H) * LDH * 2;         // f32 b1[128], b2[128]
constexpr size_t TS_WARP = TS_B + 2 * SUR_H * 4;
constexpr size_t TS_X_BYTES = 16 * LDX * 2;
constexpr size_t TS_H_BYTES = 16 * LDH * 2;
constexpr size_t TS_TOTAL = TS_WARP + (NT / 32) * (TS_X_BYTES + TS_H_BYTES);
static_assert(2 * TS_TOTAL <= 227 * 1024, "two k_tel CTAs per SM");
static_assert(EPW == 4, "k_tel assigns rows to four events per warp");

// k_event shared memory
constexpr size_t SM_V1 = 0;                                      // bf16 [256 k][LDV]: V1 as stored
constexpr size_t SM_P = SM_V1 + size_t(SUR_G) * LDV * 2;         // bf16 [2][32][LDV] pooled rows, double-buffered
constexpr size_t SM_G = SM_P + 2 * size_t(FE) * LDV * 2;         // bf16 [32][LDV]
constexpr size_t SM_V2 = SM_G + size_t(FE) * LDV * 2;            // bf16 [256][4]
constexpr size_t SM_Y = SM_V2 + size_t(SUR_G) * 4 * 2;           // f32 [32][4]
constexpr size_t SM_TOTAL = SM_Y + size_t(FE) * 4 * 4;
static_assert(SM_TOTAL <= 227 * 1024, "shared memory per CTA");

__device__ __forceinline__ uint32_t lds32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// A fragments of two m16 row blocks at rows r0.., k-columns k0..k0+15 of a row-major BF16 tile.
__device__ __forceinline__ void load_a(uint32_t (&af)[2][4], const __nv_bfloat16* base, int ld, int r0, int k0,
                                       int gq, int tq) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const __nv_bfloat16* p = base + (r0 + 16 * i + gq) * ld + k0 + 2 * tq;
        af[i][0] = lds32(p);
        af[i][1] = lds32(p + 8 * ld);
        af[i][2] = lds32(p + 8);
        af[i][3] = lds32(p + 8 * ld + 8);
    }
}

// ReLU(acc + bias) rounded to BF16 into a row-major tile (rows r0.., columns c0..).
__device__ __forceinline__ void store_relu(const float (&acc)[2][4][4], const float (&bias)[4][2], __nv_bfloat16* dst,
                                           int ld, int r0, int c0, int gq, int tq) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = r0 + 16 * i + gq + 8 * h, n = c0 + 8 * j + 2 * tq;
                const float v0 = fmaxf(acc[i][j][2 * h] + bias[j][0], 0.f);
                const float v1 = fmaxf(acc[i][j][2 * h + 1] + bias[j][1], 0.f);
                *reinterpret_cast<__nv_bfloat162*>(dst + m * ld + n) = __floats2bfloat162_rn(v0, v1);
            }
}

// B fragments of two n8 tiles (columns n0..n0+15) at k-rows k0..k0+15 of a
// k-major BF16 matrix in shared memory: b[0..1] for n0, b[2..3] for n0 + 8.
__device__ __forceinline__ void ldsm_b_trans(uint32_t (&b)[4], const __nv_bfloat16* base, int ld, int k0, int n0,
                                             int lane) {
    const __nv_bfloat16* p = base + (k0 + (lane & 15)) * ld + n0 + (lane >> 4) * 8;
    const uint32_t addr = static_cast<uint32_t>(__cvta_generic_to_shared(p));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3])
                 : "r"(addr));
}

template <typename T>
__device__ __forceinline__ T sel4(int g, T v0, T v1, T v2, T v3) {
    return g == 0 ? v0 : g == 1 ? v1 : g == 2 ? v2 : v3;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void zero_acc(float (&acc)[2][4][4]) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
}

}  // namespace


// ------------------------------------------------------------------ k_tel
__global__ void __launch_bounds__(NT, 2) k_tel(const InferArgs a) {
    extern __shared__ __align__(128) unsigned char sm[];
    __nv_bfloat16* W1s = reinterpret_cast<__nv_bfloat16*>(sm + TS_W1);
    __nv_bfloat16* W2s = reinterpret_cast<__nv_bfloat16*>(sm + TS_W2);
    float* b1s = reinterpret_cast<float*>(sm + TS_B);
    float* b2s = b1s + SUR_H;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
    __nv_bfloat16* Xw = reinterpret_cast<__nv_bfloat16*>(sm + TS_WARP + warp * (TS_X_BYTES + TS_H_BYTES));
    __nv_bfloat16* Hw = reinterpret_cast<__nv_bfloat16*>(sm + TS_WARP + warp * (TS_X_BYTES + TS_H_BYTES) + TS_X_BYTES);
    {
        const uint4* w1 = reinterpret_cast<const uint4*>(a.pb + OFF_W1);
        const uint4* w2 = reinterpret_cast<const uint4*>(a.pb + OFF_W2);
        for (int i = tid; i < SUR_XPAD * SUR_H / 8; i += NT)
            *reinterpret_cast<uint4*>(W1s + (i / (SUR_H / 8)) * LDH + 8 * (i % (SUR_H / 8))) = w1[i];
        for (int i = tid; i < SUR_H * SUR_H / 8; i += NT)
            *reinterpret_cast<uint4*>(W2s + (i / (SUR_H / 8)) * LDH + 8 * (i % (SUR_H / 8))) = w2[i];
        for (int i = tid; i < SUR_H; i += NT) {
            b1s[i] = a.p[OFF_B1 + i];
            b2s[i] = a.p[OFF_B2 + i];
        }
    }
    __syncthreads();
    const FeatArgs& f = a.f;
    const int64_t n_evt = f.n_evt, n_img = f.n_img;
    const int sub = lane % SUR_EVT_LANES, grp = lane / SUR_EVT_LANES;
    const int64_t nwarps = (int64_t(gridDim.x) * NT) >> 5;
    for (int64_t e0 = (int64_t(blockIdx.x) * (NT / 32) + warp) * EPW; e0 < n_evt; e0 += nwarps * EPW) {
        // ---- per-event prologue, eight lanes per event (as k_features)
        const int64_t e = e0 + grp;
        int i0 = 0, n = 0;
        bool ok = false;
        if (e < n_evt) {
            i0 = f.evt_off[e];
            const int i1 = f.evt_off[e + 1];
            ok = !(i0 < 0 || i1 < i0 || i1 > n_img);
            n = ok ? i1 - i0 : 0;
        }
        float bx, by;
        int cnt;
        sur_event_baseline(f.h, i0, n, sub, nullptr, bx, by, cnt);
        if (e < n_evt && sub == 0) {
            f.base[e] = make_float2(bx, by);
            f.n_used[e] = ok ? cnt : -1;
        }
        // the four events' rows, in order
        int off[EPW + 1], ig[EPW], cg[EPW];
        float bxg[EPW], byg[EPW];
        off[0] = 0;
#pragma unroll
        for (int g = 0; g < EPW; ++g) {
            off[g + 1] = off[g] + __shfl_sync(0xffffffffu, n, SUR_EVT_LANES * g);
            ig[g] = __shfl_sync(0xffffffffu, i0, SUR_EVT_LANES * g);
            cg[g] = __shfl_sync(0xffffffffu, ok ? cnt : 0, SUR_EVT_LANES * g);
            bxg[g] = __shfl_sync(0xffffffffu, bx, SUR_EVT_LANES * g);
            byg[g] = __shfl_sync(0xffffffffu, by, SUR_EVT_LANES * g);
        }
        const int R = off[EPW];
        float pacc[EPW][4];
#pragma unroll
        for (int g = 0; g < EPW; ++g) pacc[g][0] = pacc[g][1] = pacc[g][2] = pacc[g][3] = 0.f;

        for (int rb = 0; rb < R; rb += 16) {
            // ---- features of rows rb .. rb + 15 (lanes 0..15)
            bool urow = false;
            if (lane < 16) {
                const int r = rb + lane;
                __nv_bfloat162 x[SUR_XPAD / 2];
                if (r < R) {
                    const int g = (r >= off[1]) + (r >= off[2]) + (r >= off[3]);
                    const int img = sel4(g, ig[0], ig[1], ig[2], ig[3]) + (r - sel4(g, off[0], off[1], off[2], off[3]));
                    const rta_hillas_t h = f.h[img];
                    urow = sur_used(h);
                    sur_image_features(h, f.img_tel[img], f.tel_cam, f.tel_xy, f.cam_code, f.n_tel,
                                       sel4(g, bxg[0], bxg[1], bxg[2], bxg[3]),
                                       sel4(g, byg[0], byg[1], byg[2], byg[3]), x);
                } else {
#pragma unroll
                    for (int j = 0; j < SUR_XPAD / 2; ++j) x[j] = __floats2bfloat162_rn(0.f, 0.f);
                }
                uint4* xr = reinterpret_cast<uint4*>(Xw + lane * LDX);
                xr[0] = make_uint4(bf2_bits(x[0]), bf2_bits(x[1]), bf2_bits(x[2]), bf2_bits(x[3]));
                xr[1] = make_uint4(bf2_bits(x[4]), bf2_bits(x[5]), bf2_bits(x[6]), bf2_bits(x[7]));
            }
            const unsigned umask = __ballot_sync(0xffffffffu, urow);
            __syncwarp();
            const bool ua = (umask >> gq) & 1u, ub = (umask >> (gq + 8)) & 1u;
            // ---- layer 1: 16 n8 tiles, one k-step
            uint32_t ax[4];
            {
                const __nv_bfloat16* p = Xw + gq * LDX + 2 * tq;
                ax[0] = lds32(p);
                ax[1] = lds32(p + 8 * LDX);
                ax[2] = lds32(p + 8);
                ax[3] = lds32(p + 8 * LDX + 8);
            }
            uint32_t ah[8][4];
            {
                float acc1[16][4];
#pragma unroll
                for (int j = 0; j < 16; ++j) acc1[j][0] = acc1[j][1] = acc1[j][2] = acc1[j][3] = 0.f;
#pragma unroll
                for (int jp = 0; jp < 8; ++jp) {
                    uint32_t b[4];
                    ldsm_b_trans(b, W1s, LDH, 0, 16 * jp, lane);
                    const uint32_t b0[2] = {b[0], b[1]}, b1[2] = {b[2], b[3]};
                    mma_bf16(acc1[2 * jp], ax, b0);
                    mma_bf16(acc1[2 * jp + 1], ax, b1);
                }
                // ReLU(acc + b1) in BF16, rearranged as the A fragments of layer 2
#pragma unroll
                for (int ks = 0; ks < 8; ++ks) {
                    const int n0 = 16 * ks + 2 * tq, n1 = n0 + 8;
                    const float* c0 = acc1[2 * ks];
                    const float* c1 = acc1[2 * ks + 1];
                    ah[ks][0] = bf2_bits(__floats2bfloat162_rn(fmaxf(c0[0] + b1s[n0], 0.f), fmaxf(c0[1] + b1s[n0 + 1], 0.f)));
                    ah[ks][1] = bf2_bits(__floats2bfloat162_rn(fmaxf(c0[2] + b1s[n0], 0.f), fmaxf(c0[3] + b1s[n0 + 1], 0.f)));
                    ah[ks][2] = bf2_bits(__floats2bfloat162_rn(fmaxf(c1[0] + b1s[n1], 0.f), fmaxf(c1[1] + b1s[n1 + 1], 0.f)));
                    ah[ks][3] = bf2_bits(__floats2bfloat162_rn(fmaxf(c1[2] + b1s[n1], 0.f), fmaxf(c1[3] + b1s[n1 + 1], 0.f)));
                }
            }
            // ---- layer 2 in two halves of 64 columns; 8 k-steps in ascending order per tile
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float acc2[8][4];
#pragma unroll
                for (int j = 0; j < 8; ++j) acc2[j][0] = acc2[j][1] = acc2[j][2] = acc2[j][3] = 0.f;
#pragma unroll
                for (int ks = 0; ks < 8; ++ks) {
#pragma unroll
                    for (int jp = 0; jp < 4; ++jp) {
                        uint32_t b[4];
                        ldsm_b_trans(b, W2s, LDH, 16 * ks, 64 * half + 16 * jp, lane);
                        const uint32_t b0[2] = {b[0], b[1]}, b1[2] = {b[2], b[3]};
                        mma_bf16(acc2[2 * jp], ah[ks], b0);
                        mma_bf16(acc2[2 * jp + 1], ah[ks], b1);
                    }
                }
                // ReLU(acc + b2) in BF16; an unused image gets a +0 row
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int n = 64 * half + 8 * j + 2 * tq;
                    *reinterpret_cast<__nv_bfloat162*>(Hw + gq * LDH + n) = __floats2bfloat162_rn(
                        ua ? fmaxf(acc2[j][0] + b2s[n], 0.f) : 0.f, ua ? fmaxf(acc2[j][1] + b2s[n + 1], 0.f) : 0.f);
                    *reinterpret_cast<__nv_bfloat162*>(Hw + (gq + 8) * LDH + n) = __floats2bfloat162_rn(
                        ub ? fmaxf(acc2[j][2] + b2s[n], 0.f) : 0.f, ub ? fmaxf(acc2[j][3] + b2s[n + 1], 0.f) : 0.f);
                }
            }
            __syncwarp();
            // ---- pooling: lane = 4 channels; rows in image order, each into its event
            const int rend = min(R, rb + 16);
            for (int r = rb; r < rend; ++r) {
                const int g = (r >= off[1]) + (r >= off[2]) + (r >= off[3]);
                const uint2 v = *reinterpret_cast<const uint2*>(Hw + (r - rb) * LDH + 4 * lane);
                const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.x));
                const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.y));
#pragma unroll
                for (int gg = 0; gg < EPW; ++gg)
                    if (g == gg) {
                        pacc[gg][0] += lo.x;
                        pacc[gg][1] += lo.y;
                        pacc[gg][2] += hi.x;
                        pacc[gg][3] += hi.y;
                    }
            }
            __syncwarp();
        }
        // ---- pooled vectors [sum / 40, sum / max(1, n_used)] in BF16
#pragma unroll
        for (int g = 0; g < EPW; ++g) {
            const int64_t eg = e0 + g;
            if (eg >= n_evt) break;
            const float d = fmaxf(1.f, float(cg[g]));
            __nv_bfloat16* pr = a.P + eg * SUR_G + 4 * lane;
            const __nv_bfloat162 s0 = __floats2bfloat162_rn(pacc[g][0] * (1.f / SUR_POOL_DIV), pacc[g][1] * (1.f / SUR_POOL_DIV));
            const __nv_bfloat162 s1 = __floats2bfloat162_rn(pacc[g][2] * (1.f / SUR_POOL_DIV), pacc[g][3] * (1.f / SUR_POOL_DIV));
            const __nv_bfloat162 m0 = __floats2bfloat162_rn(pacc[g][0] / d, pacc[g][1] / d);
            const __nv_bfloat162 m1 = __floats2bfloat162_rn(pacc[g][2] / d, pacc[g][3] / d);
            *reinterpret_cast<uint2*>(pr) = make_uint2(bf2_bits(s0), bf2_bits(s1));
            *reinterpret_cast<uint2*>(pr + SUR_H) = make_uint2(bf2_bits(m0), bf2_bits(m1));
        }
    }
}

// ------------------------------------------------------------------ k_event
// Pooled rows of events [e0, e0 + ne) into a shared-memory tile (zeros past ne).
__device__ __forceinline__ void stage_pooled(__nv_bfloat16* Pt, const __nv_bfloat16* P, int64_t e0, int ne, int tid) {
    for (int i = tid; i < FE * (SUR_G / 8); i += NT) {
        const int el = i / (SUR_G / 8), c = i % (SUR_G / 8);
        __nv_bfloat16* dst = Pt + el * LDV + 8 * c;
        if (el < ne) cp_async16(dst, P + (e0 + el) * SUR_G + 8 * c);
        else *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
    cp_async_commit();
}

__global__ void __launch_bounds__(NT, 1) k_event(const InferArgs a) {
    extern __shared__ __align__(128) unsigned char sm[];
    __nv_bfloat16* V1s = reinterpret_cast<__nv_bfloat16*>(sm + SM_V1);
    __nv_bfloat16* Pbuf = reinterpret_cast<__nv_bfloat16*>(sm + SM_P);
    __nv_bfloat16* Gs = reinterpret_cast<__nv_bfloat16*>(sm + SM_G);
    __nv_bfloat16* V2s = reinterpret_cast<__nv_bfloat16*>(sm + SM_V2);
    float* Ys = reinterpret_cast<float*>(sm + SM_Y);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
    const int64_t n_evt = a.f.n_evt;
    const int TE = a.tile_events;
    int64_t t = blockIdx.x;
    if (t < a.n_tiles) stage_pooled(Pbuf, a.P, t * TE, int(TE < n_evt - t * TE ? TE : n_evt - t * TE), tid);
    // weights: V1 copied as stored (k-major rows, padded), V2 as stored
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.pb + OFF_V1);
        for (int i = tid; i < SUR_G * SUR_G / 8; i += NT)
            *reinterpret_cast<uint4*>(V1s + (i / (SUR_G / 8)) * LDV + 8 * (i % (SUR_G / 8))) = src[i];
        for (int i = tid; i < SUR_G * 4; i += NT) V2s[i] = a.pb[OFF_V2 + i];
    }
    const int wn2 = warp * 32;
    float c1r[4][2];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int c = 0; c < 2; ++c) c1r[j][c] = a.p[OFF_C1 + wn2 + 8 * j + 2 * tq + c];

    for (int buf = 0; t < a.n_tiles; t += gridDim.x, buf ^= 1) {
        const int64_t e0 = t * TE;
        const int ne = int(TE < n_evt - e0 ? TE : n_evt - e0);
        __nv_bfloat16* Ps = Pbuf + buf * (FE * LDV);
        cp_async_wait_all();
        __syncthreads();
        const int64_t tn = t + gridDim.x;
        if (tn < a.n_tiles)
            stage_pooled(Pbuf + (buf ^ 1) * (FE * LDV), a.P, tn * TE, int(TE < n_evt - tn * TE ? TE : n_evt - tn * TE), tid);
        // ---- event network 256 -> 256 (columns wn2..wn2+31 per warp)
        {
            float acc[2][4][4];
            uint32_t af[2][4], bfr[2][4];
            zero_acc(acc);
#pragma unroll 4
            for (int ks = 0; ks < SUR_G / 16; ++ks) {
                load_a(af, Ps, LDV, 0, 16 * ks, gq, tq);
                ldsm_b_trans(bfr[0], V1s, LDV, 16 * ks, wn2, lane);
                ldsm_b_trans(bfr[1], V1s, LDV, 16 * ks, wn2 + 16, lane);
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint32_t b[2] = {bfr[j >> 1][2 * (j & 1)], bfr[j >> 1][2 * (j & 1) + 1]};
                        mma_bf16(acc[i][j], af[i], b);
                    }
            }
            store_relu(acc, c1r, Gs, LDV, 0, wn2, gq, tq);
        }
        __syncthreads();
        // ---- 256 -> 4 on the tensor cores, one warp per 16 events
        if (warp < 2) {
            const int r0 = 16 * warp;
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
            for (int ks = 0; ks < SUR_G / 16; ++ks) {
                const __nv_bfloat16* p = Gs + (r0 + gq) * LDV + 16 * ks + 2 * tq;
                const uint32_t af[4] = {lds32(p), lds32(p + 8 * LDV), lds32(p + 8), lds32(p + 8 * LDV + 8)};
                uint32_t bf[2];
                head_b_fragment(V2s, ks, gq, tq, bf);
                mma_bf16(acc, af, bf);
            }
            if (tq < 2) {
                const int c = 2 * tq;
                const float c2a = a.p[OFF_C2 + c], c2b = a.p[OFF_C2 + c + 1];
                Ys[(r0 + gq) * 4 + c] = acc[0] + c2a;
                Ys[(r0 + gq) * 4 + c + 1] = acc[1] + c2b;
                Ys[(r0 + gq + 8) * 4 + c] = acc[2] + c2a;
                Ys[(r0 + gq + 8) * 4 + c + 1] = acc[3] + c2b;
            }
        }
        __syncthreads();
        // ---- outputs
        if (tid < ne) {
            const int64_t e = e0 + tid;
            const float y[4] = {Ys[tid * 4 + 0], Ys[tid * 4 + 1], Ys[tid * 4 + 2], Ys[tid * 4 + 3]};
            sur_emit_event(a.o, e, y, a.f.base[e], a.f.n_used[e]);
        }
    }
    cp_async_wait_all();
}

cudaError_t launch_infer(const InferArgs& a, int n_sm, cudaStream_t s) {
    if (a.tile_events < 1 || a.tile_events > FE) return cudaErrorInvalidValue;
    if (a.f.n_evt <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_tel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(TS_TOTAL));
    if (e != cudaSuccess) return e;
    const int64_t warps = (a.f.n_evt + EPW - 1) / EPW;
    const int64_t g = std::min<int64_t>((warps + NT / 32 - 1) / (NT / 32), int64_t(n_sm) * 2);
    k_tel<<<int(g), NT, TS_TOTAL, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_event, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SM_TOTAL))) != cudaSuccess)
        return e;
    k_event<<<int(std::min<int64_t>(a.n_tiles, n_sm)), NT, SM_TOTAL, s>>>(a);
    return cudaGetLastError();
}

}  // namespace rta
