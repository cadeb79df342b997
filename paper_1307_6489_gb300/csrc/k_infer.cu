// Inference of the deep-sets surrogate (energy, direction offset and
// gamma/hadron score next to the geometric direction, Sec. 4.1), in two
// kernels, both on the fifth-generation tensor cores (tcgen05: operands in
// shared memory as canonical K-major core matrices, FP32 accumulators in
// tensor memory, one thread issuing the MMAs and committing them to an
// mbarrier that the CTA waits on with a time limit):
//
//   k_tel    tiles of up to 32 events: per-event baseline and used images (eight
//            lanes per event), then, 128 image rows at a time, the features,
//            the per-telescope network 16 -> 128 -> 128 (ReLU; BF16
//            activations re-staged as the next layer's operand) and the sum /
//            mean pooling in image order. Writes the pooled vectors, baselines
//            and used counts.
//   k_event  tiles of 128 events: the event network 256 -> 256 (ReLU), then
//            the 256 -> 4 output layer in FP32 from the BF16-rounded
//            activations, the outputs, and the fallback list for the
//            geometric intersection.
//
// The features and the eight-lane event reductions are the training path's
// own expressions (rta_mlp_dev.cuh), so the baselines and used counts equal
// those of k_features bit for bit. The network layers sum their exact BF16
// products in FP32 in the tensor core's order rather than mma.sync's, so the
// outputs agree with the training-path forward to accumulation-order effects.
#include <algorithm>

#include "rta_mlp_dev.cuh"
#include "rta_tc.cuh"

namespace rta {
namespace {

constexpr int NT = 256;             // threads per CTA (both kernels)
constexpr int TM = 128;             // MMA M: image rows per k_tel block, events per k_event tile
constexpr int TE = 32;              // events per k_tel tile at most
constexpr int LDH = SUR_H + 8;      // row stride of the row-major hidden tile used for pooling

// k_tel shared memory (two CTAs per SM)
constexpr size_t TS_W1 = 0;                                      // bf16 W1^T canonical [128 n][16 k]
constexpr size_t TS_W2 = TS_W1 + size_t(SUR_H) * SUR_XPAD * 2;   // bf16 W2^T canonical [128 n][128 k]
constexpr size_t TS_X = TS_W2 + size_t(SUR_H) * SUR_H * 2;       // bf16 features, canonical [128][16]
constexpr size_t TS_H = TS_X + size_t(TM) * SUR_XPAD * 2;        // bf16 H1 canonical [128][128]; then H2 row-major [128][LDH]
constexpr size_t TS_PACC = TS_H + size_t(TM) * LDH * 2;          // f32 [32][128] pooling sums
constexpr size_t TS_B = TS_PACC + size_t(TE) * SUR_H * 4;        // f32 b1[128], b2[128]
constexpr size_t TS_ROWB = TS_B + 2 * SUR_H * 4;                 // int64 [33] first row of each event
constexpr size_t TS_BASE = TS_ROWB + size_t(TE + 1) * 8;         // float2 [32]
constexpr size_t TS_LO = TS_BASE + size_t(TE) * 8;               // int [32] first image
constexpr size_t TS_CNT = TS_LO + size_t(TE) * 4;                // int [32] rows
constexpr size_t TS_NU = TS_CNT + size_t(TE) * 4;                // int [32] used images (0 if malformed)
constexpr size_t TS_USED = TS_NU + size_t(TE) * 4;               // u8 [128]
constexpr size_t TS_TCAM = TS_USED + TM;                         // int [1024] camera of each telescope
constexpr size_t TS_TXY = TS_TCAM + size_t(RTA_MAX_TEL) * 4;     // float2 [1024] telescope positions
constexpr size_t TS_CODE = TS_TXY + size_t(RTA_MAX_TEL) * 8;     // f32 [16] camera codes
constexpr size_t TS_BAR = TS_CODE + size_t(RTA_MAX_CAMS) * 4;    // MMA mbarrier, load mbarrier, TMEM address, abort flag
constexpr size_t TS_TOTAL = TS_BAR + 32;
static_assert(TS_H % 16 == 0 && TS_X % 16 == 0 && TS_W2 % 16 == 0, "16-byte aligned operand tiles");
static_assert(TS_BAR % 8 == 0 && TS_ROWB % 8 == 0 && TS_TXY % 8 == 0, "aligned barriers and tables");
static_assert(TS_W2 == TS_W1 + size_t(PK_W2T - PK_W1T) * 2, "W1^T and W2^T are one contiguous copy");
static_assert(2 * TS_TOTAL <= 227 * 1024, "two k_tel CTAs per SM");

// k_event shared memory
constexpr size_t SM_V1 = 0;                                      // bf16 V1^T, canonical K-major [256 n][256 k]
constexpr size_t SM_P = SM_V1 + size_t(SUR_G) * SUR_G * 2;       // bf16 pooled tile, canonical [128][256]
constexpr size_t SM_V2 = SM_P + size_t(TM) * SUR_G * 2;          // f32 [256][4]
constexpr size_t SM_C1 = SM_V2 + size_t(SUR_G) * 4 * 4;          // f32 [256]
constexpr size_t SM_YP = SM_C1 + size_t(SUR_G) * 4;              // f32 [128][4] second-half partial outputs
constexpr size_t SM_BAR = SM_YP + size_t(TM) * 4 * 4;            // MMA mbarrier, load mbarrier, TMEM address, abort flag
constexpr size_t SM_TOTAL = SM_BAR + 32;
static_assert(SM_TOTAL <= 227 * 1024, "shared memory per CTA");

// One thread: copy `bytes` (a multiple of 16) from global to shared memory with
// the bulk-copy engine in pieces of at most 32 KB, all completing on bar.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t policy) {
    for (uint32_t o = 0; o < bytes; o += 32768u)
        bulk_g2s(static_cast<char*>(dst) + o, static_cast<const char*>(src) + o, min(32768u, bytes - o), bar, policy);
}

// Wait for the MMAs committed to bar (phase `phase`); on a timeout flag the
// status word and the CTA's abort flag. Every thread calls it; returns false
// for every thread once any thread gave up.
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t phase, volatile int* abort_s, unsigned int* status) {
    if (!mbar_wait(bar, phase, abort_s)) {
        *abort_s = 1;
        atomicOr(status, RTA_DEV_TIMEOUT);
    }
    __syncthreads();
    if (*abort_s) return false;
    tc_fence_after();
    return true;
}

// Release the CTA's tensor memory. After an abort, one more bounded wait on
// each barrier lets MMAs and copies still in flight finish first (mma_parity /
// ld_parity: the parity of the phase that may be pending; a completed or never
// started phase returns at once).
__device__ __forceinline__ void tc_teardown(uint64_t* bar, uint32_t mma_parity, uint64_t* bar_ld, uint32_t ld_parity,
                                            volatile int* abort_s, uint32_t tmem, uint32_t ncols) {
    tc_fence_before();
    __syncthreads();
    if (*abort_s && threadIdx.x == 0) {
        volatile int none = 0;
        mbar_wait(bar, mma_parity, &none);
        mbar_wait(bar_ld, ld_parity, &none);
    }
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tc_dealloc(tmem, ncols);
}

}  // namespace

// ------------------------------------------------------------------ k_tel
__global__ void __launch_bounds__(NT, 2) k_tel(const InferArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __nv_bfloat16* W1s = reinterpret_cast<__nv_bfloat16*>(sm + TS_W1);
    __nv_bfloat16* W2s = reinterpret_cast<__nv_bfloat16*>(sm + TS_W2);
    __nv_bfloat16* Xs = reinterpret_cast<__nv_bfloat16*>(sm + TS_X);
    __nv_bfloat16* Hs = reinterpret_cast<__nv_bfloat16*>(sm + TS_H);
    float* Pacc = reinterpret_cast<float*>(sm + TS_PACC);
    float* b1s = reinterpret_cast<float*>(sm + TS_B);
    float* b2s = b1s + SUR_H;
    int64_t* rowb = reinterpret_cast<int64_t*>(sm + TS_ROWB);
    float2* base_s = reinterpret_cast<float2*>(sm + TS_BASE);
    int* lo_s = reinterpret_cast<int*>(sm + TS_LO);
    int* cnt_s = reinterpret_cast<int*>(sm + TS_CNT);
    int* nu_s = reinterpret_cast<int*>(sm + TS_NU);
    uint8_t* used_s = sm + TS_USED;
    int* tcam_s = reinterpret_cast<int*>(sm + TS_TCAM);
    float2* txy_s = reinterpret_cast<float2*>(sm + TS_TXY);
    float* code_s = reinterpret_cast<float*>(sm + TS_CODE);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + TS_BAR);       // MMA completion
    uint64_t* bar_ld = bar + 1;                                       // weight copy
    uint32_t* tmem_s = reinterpret_cast<uint32_t*>(sm + TS_BAR + 16);
    volatile int* abort_s = reinterpret_cast<volatile int*>(sm + TS_BAR + 20);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const FeatArgs& f = a.f;
    const int64_t n_evt = f.n_evt, n_img = f.n_img;
    const int n_tel = min(f.n_tel, RTA_MAX_TEL);

    if (warp == 0) {
        tc_alloc(tmem_s, 256);               // columns 0-127: layer 1, 128-255: layer 2
        tc_relinquish();
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(bar_ld, 1);
        fence_mbar_init();
        *abort_s = 0;
        // W1^T and W2^T (canonical operands) by the bulk-copy engine
        constexpr uint32_t bytes = uint32_t(PK_V1T - PK_W1T) * 2;
        mbar_arrive_expect_tx(bar_ld, bytes);
        bulk_copy(W1s, a.pk + PK_W1T, bytes, bar_ld, l2_policy_evict_last());
    }
    {
        // telescope tables and biases: all loads issued before any store
        int tc[RTA_MAX_TEL / NT];
        float2 txy[RTA_MAX_TEL / NT];
#pragma unroll
        for (int k = 0; k < RTA_MAX_TEL / NT; ++k) {
            const int i = tid + k * NT;
            tc[k] = i < n_tel ? f.tel_cam[i] : 0;
            txy[k] = i < n_tel ? f.tel_xy[i] : make_float2(0.f, 0.f);
        }
        const float code = tid < RTA_MAX_CAMS ? f.cam_code[tid] : 0.f;
        const float bb1 = tid < SUR_H ? a.p[OFF_B1 + tid] : 0.f, bb2 = tid < SUR_H ? a.p[OFF_B2 + tid] : 0.f;
#pragma unroll
        for (int k = 0; k < RTA_MAX_TEL / NT; ++k) {
            const int i = tid + k * NT;
            if (i < n_tel) {
                tcam_s[i] = tc[k];
                txy_s[i] = txy[k];
            }
        }
        if (tid < RTA_MAX_CAMS) code_s[tid] = code;
        if (tid < SUR_H) {
            b1s[tid] = bb1;
            b2s[tid] = bb2;
        }
    }
    __syncthreads();
    bool alive = tc_wait(bar_ld, 0, abort_s, a.o.status);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_s;
    const uint32_t idesc = tc_idesc_bf16(TM, SUR_H);
    const uint32_t x_addr = smem_addr(Xs), h_addr = smem_addr(Hs), w1_addr = smem_addr(W1s), w2_addr = smem_addr(W2s);
    const int q = warp & 3, c_half = (warp >> 2) * (SUR_H / 2), row = 32 * q + lane;
    const uint32_t t_lane = uint32_t(32 * q) << 16;
    const int sub = lane % SUR_EVT_LANES, grp = lane / SUR_EVT_LANES;
    uint32_t phase = 0;
    const int te = a.tel_tile_events;
    const int64_t n_tiles = (n_evt + te - 1) / te;

    for (int64_t t = alive ? int64_t(blockIdx.x) : n_tiles; t < n_tiles; t += gridDim.x) {
        const int64_t e0 = t * te;
        const int ne = int(te < n_evt - e0 ? te : n_evt - e0);
        // ---- per-event prologue, eight lanes per event (as k_features)
        {
            const int el = (32 / SUR_EVT_LANES) * warp + grp;
            const int64_t e = e0 + el;
            int i0 = 0, n = 0;
            bool ok = false;
            if (el < ne) {
                i0 = f.evt_off[e];
                const int i1 = f.evt_off[e + 1];
                ok = !(i0 < 0 || i1 < i0 || i1 > n_img);
                n = ok ? i1 - i0 : 0;
            }
            float bx, by;
            int cnt;
            sur_event_baseline(f.h, i0, n, sub, nullptr, bx, by, cnt);
            if (sub == 0) {
                if (el < ne) {
                    f.base[e] = make_float2(bx, by);
                    f.n_used[e] = ok ? cnt : -1;
                }
                base_s[el] = make_float2(bx, by);
                lo_s[el] = i0;
                cnt_s[el] = n;
                nu_s[el] = ok ? cnt : 0;
            }
        }
        for (int i = tid; i < TE * SUR_H; i += NT) Pacc[i] = 0.f;
        __syncthreads();
        if (warp == 0) {
            int64_t v = cnt_s[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            rowb[lane + 1] = v;
            if (lane == 0) rowb[0] = 0;
        }
        __syncthreads();
        const int64_t R = rowb[TE];

        for (int64_t rb = 0; rb < R; rb += TM) {
            // ---- features of rows rb .. rb + 127, one thread per row
            if (tid < TM) {
                const int64_t r = rb + tid;
                __nv_bfloat162 x[SUR_XPAD / 2];
                bool used = false;
                if (r < R) {
                    int lo = 0, hi = TE - 1;              // last event whose first row is <= r
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (rowb[mid] <= r) lo = mid;
                        else hi = mid - 1;
                    }
                    const int64_t img = int64_t(lo_s[lo]) + (r - rowb[lo]);
                    const rta_hillas_t h = f.h[img];
                    used = sur_used(h);
                    const float2 b = base_s[lo];
                    sur_image_features(h, f.img_tel[img], tcam_s, txy_s, code_s, n_tel, b.x, b.y, x);
                } else {
#pragma unroll
                    for (int j = 0; j < SUR_XPAD / 2; ++j) x[j] = __floats2bfloat162_rn(0.f, 0.f);
                }
                *reinterpret_cast<uint4*>(Xs + canon_off(tid, 0, SUR_XPAD)) =
                    make_uint4(bf2_bits(x[0]), bf2_bits(x[1]), bf2_bits(x[2]), bf2_bits(x[3]));
                *reinterpret_cast<uint4*>(Xs + canon_off(tid, 8, SUR_XPAD)) =
                    make_uint4(bf2_bits(x[4]), bf2_bits(x[5]), bf2_bits(x[6]), bf2_bits(x[7]));
                used_s[tid] = used;
            }
            fence_proxy_async_smem();
            __syncthreads();
            // ---- layer 1: D1 = X W1 (one K-step)
            if (tid == 0) {
                tc_fence_after();
                tc_mma(tmem, tc_desc(x_addr, 128u, 16u * SUR_XPAD), tc_desc(w1_addr, 128u, 16u * SUR_XPAD), idesc, false);
                tc_commit(bar);
            }
            alive = tc_wait(bar, phase, abort_s, a.o.status);
            phase ^= 1u;
            if (!alive) break;
            // ReLU(D1 + b1) in BF16 -> canonical operand of layer 2 (this thread: one row, 64 columns)
#pragma unroll 1
            for (int cb = 0; cb < SUR_H / 2; cb += 16) {
                const int c0 = c_half + cb;
                uint32_t v[16];
                tc_ld16(tmem + t_lane + uint32_t(c0), v);
                uint32_t w[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    w[i] = bf2_bits(__floats2bfloat162_rn(fmaxf(__uint_as_float(v[2 * i]) + b1s[c0 + 2 * i], 0.f),
                                                          fmaxf(__uint_as_float(v[2 * i + 1]) + b1s[c0 + 2 * i + 1], 0.f)));
                *reinterpret_cast<uint4*>(Hs + canon_off(row, c0, SUR_H)) = make_uint4(w[0], w[1], w[2], w[3]);
                *reinterpret_cast<uint4*>(Hs + canon_off(row, c0 + 8, SUR_H)) = make_uint4(w[4], w[5], w[6], w[7]);
            }
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            // ---- layer 2: D2 = H1 W2 (eight K-steps)
            if (tid == 0) {
                tc_fence_after();
#pragma unroll 1
                for (int ks = 0; ks < SUR_H / 16; ++ks)
                    tc_mma(tmem + SUR_H, tc_desc(h_addr + 256u * ks, 128u, 16u * SUR_H),
                           tc_desc(w2_addr + 256u * ks, 128u, 16u * SUR_H), idesc, ks > 0);
                tc_commit(bar);
            }
            alive = tc_wait(bar, phase, abort_s, a.o.status);
            phase ^= 1u;
            if (!alive) break;
            // ReLU(D2 + b2) in BF16, +0 rows for unused images -> row-major tile for pooling
            const bool urow = used_s[row];
#pragma unroll 1
            for (int cb = 0; cb < SUR_H / 2; cb += 16) {
                const int c0 = c_half + cb;
                uint32_t v[16];
                tc_ld16(tmem + SUR_H + t_lane + uint32_t(c0), v);
                uint32_t w[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    w[i] = bf2_bits(__floats2bfloat162_rn(
                        urow ? fmaxf(__uint_as_float(v[2 * i]) + b2s[c0 + 2 * i], 0.f) : 0.f,
                        urow ? fmaxf(__uint_as_float(v[2 * i + 1]) + b2s[c0 + 2 * i + 1], 0.f) : 0.f));
                uint4* hr = reinterpret_cast<uint4*>(Hs + row * LDH + c0);
                hr[0] = make_uint4(w[0], w[1], w[2], w[3]);
                hr[1] = make_uint4(w[4], w[5], w[6], w[7]);
            }
            tc_fence_before();
            __syncthreads();
            // ---- pooling: thread = (channel, event parity); image order within each event
            {
                const int c = tid & (SUR_H - 1);
                const int64_t rend = min(R, rb + TM);
                for (int el = tid >> 7; el < ne; el += NT / SUR_H) {
                    const int64_t lo = max(rowb[el], rb), hi = min(rowb[el + 1], rend);
                    if (lo >= hi) continue;
                    float s = Pacc[el * SUR_H + c];
                    for (int64_t r = lo; r < hi; ++r) s += __bfloat162float(Hs[(r - rb) * LDH + c]);
                    Pacc[el * SUR_H + c] = s;
                }
            }
            __syncthreads();
        }
        if (!alive) break;
        // ---- pooled vectors [sum / 40, sum / max(1, n_used)] in BF16
        for (int idx = tid; idx < ne * (SUR_H / 4); idx += NT) {
            const int el = idx / (SUR_H / 4), c4 = idx % (SUR_H / 4);
            const float4 s = reinterpret_cast<const float4*>(Pacc + el * SUR_H)[c4];
            const float d = fmaxf(1.f, float(nu_s[el]));
            const int64_t e = e0 + el, et = e / a.ev_tile_events, er = e % a.ev_tile_events;
            __nv_bfloat16* blk = a.P + et * (TM * SUR_G);
            *reinterpret_cast<uint2*>(blk + canon_off(er, 4 * c4, SUR_G)) =
                make_uint2(bf2_bits(__floats2bfloat162_rn(s.x * (1.f / SUR_POOL_DIV), s.y * (1.f / SUR_POOL_DIV))),
                           bf2_bits(__floats2bfloat162_rn(s.z * (1.f / SUR_POOL_DIV), s.w * (1.f / SUR_POOL_DIV))));
            *reinterpret_cast<uint2*>(blk + canon_off(er, SUR_H + 4 * c4, SUR_G)) =
                make_uint2(bf2_bits(__floats2bfloat162_rn(s.x / d, s.y / d)),
                           bf2_bits(__floats2bfloat162_rn(s.z / d, s.w / d)));
        }
        __syncthreads();
    }
    tc_teardown(bar, phase ^ 1u, bar_ld, 0u, abort_s, tmem, 256);
}

// ------------------------------------------------------------------ k_event
// Event network on tcgen05: per tile of 128 events, G = ReLU(P V1 + c1) with
// P (128 x 256) and V1^T (256 x 256) in shared memory as canonical K-major
// operands and G (FP32, 128 lanes x 256 columns) in tensor memory; one thread
// issues the sixteen K-steps and commits them to an mbarrier. Then each thread
// reads one event's row of G (warps 0-3 columns 0-127, warps 4-7 columns
// 128-255), rounds it to BF16 as the training path stores it, and forms the
// 256 -> 4 output layer in FP32; the outputs and fallback list follow.
__global__ void __launch_bounds__(NT, 1) k_event(const InferArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __nv_bfloat16* V1s = reinterpret_cast<__nv_bfloat16*>(sm + SM_V1);
    __nv_bfloat16* Pt = reinterpret_cast<__nv_bfloat16*>(sm + SM_P);
    float* V2f = reinterpret_cast<float*>(sm + SM_V2);
    float* c1s = reinterpret_cast<float*>(sm + SM_C1);
    float* yp = reinterpret_cast<float*>(sm + SM_YP);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + SM_BAR);       // MMA completion
    uint64_t* bar_ld = bar + 1;                                       // operand copies
    uint32_t* tmem_s = reinterpret_cast<uint32_t*>(sm + SM_BAR + 16);
    volatile int* abort_s = reinterpret_cast<volatile int*>(sm + SM_BAR + 20);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t n_evt = a.f.n_evt;
    const int te = a.ev_tile_events;
    const int64_t n_tiles = (n_evt + te - 1) / te;
    // bytes of the pooled rows of tile t: whole 8-row core-matrix groups
    auto tile_bytes = [&](int64_t t) {
        const int64_t ne = te < n_evt - t * te ? te : n_evt - t * te;
        return uint32_t((ne + 7) / 8) * uint32_t(8 * SUR_G * 2);
    };

    if (warp == 0) {
        tc_alloc(tmem_s, 256);
        tc_relinquish();
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(bar_ld, 1);
        fence_mbar_init();
        *abort_s = 0;
        // V1^T and the first tile's pooled rows by the bulk-copy engine
        const int64_t t0 = blockIdx.x;
        const uint32_t pbytes = t0 < n_tiles ? tile_bytes(t0) : 0u;
        mbar_arrive_expect_tx(bar_ld, uint32_t(SUR_G * SUR_G * 2) + pbytes);
        bulk_copy(V1s, a.pk + PK_V1T, uint32_t(SUR_G * SUR_G * 2), bar_ld, l2_policy_evict_last());
        if (pbytes) bulk_copy(Pt, a.P + t0 * (TM * SUR_G), pbytes, bar_ld, l2_policy_evict_first());
    }
    {
        float v2[SUR_G * 4 / NT];
#pragma unroll
        for (int k = 0; k < SUR_G * 4 / NT; ++k) v2[k] = __bfloat162float(a.pb[OFF_V2 + tid + k * NT]);
        const float c1 = a.p[OFF_C1 + tid];
#pragma unroll
        for (int k = 0; k < SUR_G * 4 / NT; ++k) V2f[tid + k * NT] = v2[k];
        c1s[tid] = c1;
    }
    __syncthreads();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_s;
    const uint32_t idesc = tc_idesc_bf16(TM, SUR_G);
    const uint32_t p_addr = smem_addr(Pt), v_addr = smem_addr(V1s);
    const int q = warp & 3, hcol = (warp >> 2) * (SUR_G / 2);
    const int row = 32 * q + lane;
    const float c2[4] = {a.p[OFF_C2 + 0], a.p[OFF_C2 + 1], a.p[OFF_C2 + 2], a.p[OFF_C2 + 3]};
    uint32_t phase = 0, ld_phase = 0;

    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int64_t e0 = t * te;
        const int ne = int(te < n_evt - e0 ? te : n_evt - e0);
        if (t != blockIdx.x && tid == 0) {            // later tiles: pooled rows only
            const uint32_t pbytes = tile_bytes(t);
            mbar_arrive_expect_tx(bar_ld, pbytes);
            bulk_copy(Pt, a.P + t * (TM * SUR_G), pbytes, bar_ld, l2_policy_evict_first());
        }
        bool alive = tc_wait(bar_ld, ld_phase, abort_s, a.o.status);
        ld_phase ^= 1u;
        if (!alive) break;
        if (tid == 0) {
#pragma unroll 1
            for (int ks = 0; ks < SUR_G / 16; ++ks)
                tc_mma(tmem, tc_desc(p_addr + 256u * ks, 128u, 16u * SUR_G), tc_desc(v_addr + 256u * ks, 128u, 16u * SUR_G),
                       idesc, ks > 0);
            tc_commit(bar);
        }
        alive = tc_wait(bar, phase, abort_s, a.o.status);
        phase ^= 1u;
        if (!alive) break;
        // this thread's event row, half of the columns
        float y[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
        for (int cb = 0; cb < SUR_G / 2; cb += 16) {
            uint32_t r[16];
            tc_ld16(tmem + (uint32_t(32 * q) << 16) + uint32_t(hcol + cb), r);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int col = hcol + cb + i;
                const float g = __bfloat162float(__float2bfloat16(fmaxf(__uint_as_float(r[i]) + c1s[col], 0.f)));
#pragma unroll
                for (int o = 0; o < 4; ++o) y[o] = fmaf(g, V2f[col * 4 + o], y[o]);
            }
        }
        if (hcol != 0) {
#pragma unroll
            for (int o = 0; o < 4; ++o) yp[row * 4 + o] = y[o];
        }
        tc_fence_before();
        __syncthreads();
        if (hcol == 0 && row < ne) {
            float yo[4];
#pragma unroll
            for (int o = 0; o < 4; ++o) yo[o] = (y[o] + yp[row * 4 + o]) + c2[o];
            const int64_t e = e0 + row;
            sur_emit_event(a.o, e, yo, a.f.base[e], a.f.n_used[e]);
        }
    }
    tc_teardown(bar, phase ^ 1u, bar_ld, ld_phase ^ 1u, abort_s, tmem, 256);
}

// BF16 twin -> transposed canonical K-major layout of the tensor-core layers.
__global__ void k_pack_tc(const __nv_bfloat16* __restrict__ pb, __nv_bfloat16* __restrict__ pk) {
    const int64_t n1 = SUR_H * SUR_XPAD, n2 = SUR_H * SUR_H, n3 = SUR_G * SUR_G;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n1 + n2 + n3;
         i += int64_t(gridDim.x) * blockDim.x) {
        if (i < n1) {                                 // W1 [16 k][128 n] -> [128 n][16 k]
            const int64_t k = i / SUR_H, n = i % SUR_H;
            pk[PK_W1T + canon_off(n, k, SUR_XPAD)] = pb[OFF_W1 + i];
        } else if (i < n1 + n2) {                     // W2 [128 k][128 n]
            const int64_t j = i - n1, k = j / SUR_H, n = j % SUR_H;
            pk[PK_W2T + canon_off(n, k, SUR_H)] = pb[OFF_W2 + j];
        } else {                                      // V1 [256 k][256 n]
            const int64_t j = i - n1 - n2, k = j / SUR_G, n = j % SUR_G;
            pk[PK_V1T + canon_off(n, k, SUR_G)] = pb[OFF_V1 + j];
        }
    }
}

cudaError_t launch_pack_tc(const __nv_bfloat16* pb, __nv_bfloat16* pk, cudaStream_t s) {
    k_pack_tc<<<64, 256, 0, s>>>(pb, pk);
    return cudaGetLastError();
}

cudaError_t launch_infer(const InferArgs& a, int n_sm, cudaStream_t s) {
    if (a.f.n_evt <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_tel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(TS_TOTAL));
    if (e != cudaSuccess) return e;
    if (a.tel_tile_events < 1 || a.tel_tile_events > TE) return cudaErrorInvalidValue;
    const int64_t tel_tiles = (a.f.n_evt + a.tel_tile_events - 1) / a.tel_tile_events;
    k_tel<<<int(std::min<int64_t>(tel_tiles, int64_t(n_sm) * 2)), NT, TS_TOTAL, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_event, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SM_TOTAL))) != cudaSuccess)
        return e;
    if (a.ev_tile_events < 1 || a.ev_tile_events > TM) return cudaErrorInvalidValue;
    const int64_t tiles = (a.f.n_evt + a.ev_tile_events - 1) / a.ev_tile_events;
    k_event<<<int(std::min<int64_t>(tiles, n_sm)), NT, SM_TOTAL, s>>>(a);
    return cudaGetLastError();
}

}  // namespace rta
