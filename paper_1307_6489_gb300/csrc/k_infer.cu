// Inference of the deep-sets surrogate (energy, direction offset and
// gamma/hadron score next to the geometric direction, Sec. 4.1), after
// k_features (per-event baseline, per-image BF16 features and used flags,
// shared with training):
//
//   k_phi    image-parallel per-telescope network, 16 -> 128 -> 128 (ReLU) on
//            the tensor cores (mma.sync m16n8k16, BF16 operands, FP32
//            accumulators). One warp owns 16 image rows: the first layer's
//            accumulators become the second layer's A fragments in registers;
//            the weights sit in shared memory and reach the MMA by
//            ldmatrix.trans. No block barrier after the weights are staged.
//            Unused images get +0 rows.
//   k_event  one persistent CTA per SM walks tiles of up to 32 consecutive
//            events: it stages the tile's rows of the per-telescope output in
//            shared memory, pools them (sum / 40 and mean), runs the event
//            network 256 -> 256 (ReLU, weights staged once per CTA) and
//            256 -> 4 on the tensor cores, and writes the outputs and the
//            fallback list for the geometric intersection.
//
// Every stage evaluates the same expressions in the same order as the
// layer-by-layer kernels of the training path (k_mlp.cu): the k-order of each
// MMA accumulation, the image order of the pooling sums (a +0 row leaves a sum
// unchanged where the pooling kernel skips the image), the output head. The
// outputs therefore equal those of the training-path forward bit for bit.
#include <algorithm>

#include "rta_mlp_dev.cuh"

namespace rta {
namespace {

constexpr int FE = 32;              // events per tile at most (one warp-wide scan)
constexpr int RT = 128;             // staged per-telescope rows per pass
constexpr int NT = 256;             // threads per k_event CTA
constexpr int PHI_WARPS = 4;        // warps per k_phi CTA
constexpr int LDH = SUR_H + 8;      // hidden row stride (conflict-free ldmatrix / fragment loads)
constexpr int LDV = SUR_G + 8;      // pooled / event-network row stride

constexpr size_t SM_V1 = 0;                                      // bf16 [256 k][LDV]: V1 as stored
constexpr size_t SM_H = SM_V1 + size_t(SUR_G) * LDV * 2;         // bf16 [RT][LDH] staged rows; P, G later
constexpr size_t SM_PACC = SM_H + size_t(RT) * LDH * 2;          // f32 [32][128] pooling sums
constexpr size_t SM_V2 = SM_PACC + size_t(FE) * SUR_H * 4;       // bf16 [256][4]
constexpr size_t SM_Y = SM_V2 + size_t(SUR_G) * 4 * 2;           // f32 [32][4]
constexpr size_t SM_ROWB = SM_Y + size_t(FE) * 4 * 4;            // int64 [33] first row of each event
constexpr size_t SM_LO = SM_ROWB + size_t(FE + 1) * 8;           // int [32] first image
constexpr size_t SM_TOTAL = SM_LO + size_t(FE) * 4;
constexpr size_t SM_G_OFF = size_t(FE) * LDV * 2;                // G follows P inside the staged-row buffer
static_assert(2 * size_t(FE) * LDV * 2 <= size_t(RT) * LDH * 2, "P and G must fit the staged-row buffer");
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

__device__ __forceinline__ void zero_acc(float (&acc)[2][4][4]) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
}

}  // namespace

// ------------------------------------------------------------------ k_phi
__global__ void __launch_bounds__(PHI_WARPS * 32, 3) k_phi(const InferArgs a) {
    __shared__ __align__(16) __nv_bfloat16 W1s[SUR_XPAD][LDH];
    __shared__ __align__(16) __nv_bfloat16 W2s[SUR_H][LDH];
    __shared__ float b1s[SUR_H], b2s[SUR_H];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
    {
        const uint4* w1 = reinterpret_cast<const uint4*>(a.pb + OFF_W1);
        const uint4* w2 = reinterpret_cast<const uint4*>(a.pb + OFF_W2);
        for (int i = tid; i < SUR_XPAD * SUR_H / 8; i += PHI_WARPS * 32)
            *reinterpret_cast<uint4*>(&W1s[i / (SUR_H / 8)][8 * (i % (SUR_H / 8))]) = w1[i];
        for (int i = tid; i < SUR_H * SUR_H / 8; i += PHI_WARPS * 32)
            *reinterpret_cast<uint4*>(&W2s[i / (SUR_H / 8)][8 * (i % (SUR_H / 8))]) = w2[i];
        for (int i = tid; i < SUR_H; i += PHI_WARPS * 32) {
            b1s[i] = a.p[OFF_B1 + i];
            b2s[i] = a.p[OFF_B2 + i];
        }
    }
    __syncthreads();
    const int64_t n_img = a.f.n_img;
    const int64_t n_units = (n_img + 15) / 16;
    for (int64_t u = int64_t(blockIdx.x) * PHI_WARPS + warp; u < n_units; u += int64_t(gridDim.x) * PHI_WARPS) {
        const int64_t ra = u * 16 + gq, rb = ra + 8;
        const bool va = ra < n_img, vb = rb < n_img;
        // A fragment of the features (one k-step)
        uint32_t ax[4];
        {
            const uint32_t* xa = reinterpret_cast<const uint32_t*>(a.f.X + ra * SUR_XPAD) + tq;
            const uint32_t* xb = reinterpret_cast<const uint32_t*>(a.f.X + rb * SUR_XPAD) + tq;
            ax[0] = va ? xa[0] : 0u;
            ax[1] = vb ? xb[0] : 0u;
            ax[2] = va ? xa[4] : 0u;
            ax[3] = vb ? xb[4] : 0u;
        }
        const bool ua = va && a.f.used[ra], ub = vb && a.f.used[rb];
        // layer 1: 16 n8 tiles
        float acc1[16][4];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc1[j][0] = acc1[j][1] = acc1[j][2] = acc1[j][3] = 0.f;
#pragma unroll
        for (int jp = 0; jp < 8; ++jp) {
            uint32_t b[4];
            ldsm_b_trans(b, &W1s[0][0], LDH, 0, 16 * jp, lane);
            const uint32_t b0[2] = {b[0], b[1]}, b1[2] = {b[2], b[3]};
            mma_bf16(acc1[2 * jp], ax, b0);
            mma_bf16(acc1[2 * jp + 1], ax, b1);
        }
        // ReLU(acc + b1) in BF16, rearranged as the A fragments of layer 2
        uint32_t ah[8][4];
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
        // layer 2: 8 k-steps in ascending order for every n8 tile
        float acc2[16][4];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc2[j][0] = acc2[j][1] = acc2[j][2] = acc2[j][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 8; ++ks) {
#pragma unroll
            for (int jp = 0; jp < 8; ++jp) {
                uint32_t b[4];
                ldsm_b_trans(b, &W2s[0][0], LDH, 16 * ks, 16 * jp, lane);
                const uint32_t b0[2] = {b[0], b[1]}, b1[2] = {b[2], b[3]};
                mma_bf16(acc2[2 * jp], ah[ks], b0);
                mma_bf16(acc2[2 * jp + 1], ah[ks], b1);
            }
        }
        // ReLU(acc + b2) in BF16; an unused image gets a +0 row
        __nv_bfloat16* ha = a.H2 + ra * SUR_H + 2 * tq;
        __nv_bfloat16* hb = a.H2 + rb * SUR_H + 2 * tq;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int n = 8 * j + 2 * tq;
            if (va)
                *reinterpret_cast<__nv_bfloat162*>(ha + 8 * j) = __floats2bfloat162_rn(
                    ua ? fmaxf(acc2[j][0] + b2s[n], 0.f) : 0.f, ua ? fmaxf(acc2[j][1] + b2s[n + 1], 0.f) : 0.f);
            if (vb)
                *reinterpret_cast<__nv_bfloat162*>(hb + 8 * j) = __floats2bfloat162_rn(
                    ub ? fmaxf(acc2[j][2] + b2s[n], 0.f) : 0.f, ub ? fmaxf(acc2[j][3] + b2s[n + 1], 0.f) : 0.f);
        }
    }
}

// ------------------------------------------------------------------ k_event
__global__ void __launch_bounds__(NT, 1) k_event(const InferArgs a) {
    extern __shared__ __align__(128) unsigned char sm[];
    __nv_bfloat16* V1s = reinterpret_cast<__nv_bfloat16*>(sm + SM_V1);
    __nv_bfloat16* Hs = reinterpret_cast<__nv_bfloat16*>(sm + SM_H);
    __nv_bfloat16* Ps = Hs;
    __nv_bfloat16* Gs = reinterpret_cast<__nv_bfloat16*>(sm + SM_H + SM_G_OFF);
    float* Pacc = reinterpret_cast<float*>(sm + SM_PACC);
    __nv_bfloat16* V2s = reinterpret_cast<__nv_bfloat16*>(sm + SM_V2);
    float* Ys = reinterpret_cast<float*>(sm + SM_Y);
    int64_t* rowb = reinterpret_cast<int64_t*>(sm + SM_ROWB);
    int* lo_s = reinterpret_cast<int*>(sm + SM_LO);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
    const FeatArgs& f = a.f;
    const int64_t n_evt = f.n_evt;
    const int TE = a.tile_events;
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
    __syncthreads();

    for (int64_t t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        const int64_t e0 = t * TE;
        const int ne = int(TE < n_evt - e0 ? TE : n_evt - e0);
        // rows of the tile: the images of its well-formed events, in order
        if (warp == 0) {
            int64_t v = 0;
            if (lane < ne) {
                const int64_t e = e0 + lane;
                const int i0 = f.evt_off[e];
                lo_s[lane] = i0;
                v = f.n_used[e] >= 0 ? int64_t(f.evt_off[e + 1]) - i0 : 0;
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            rowb[lane + 1] = v;
            if (lane == 0) rowb[0] = 0;
        }
        for (int i = tid; i < FE * SUR_H; i += NT) Pacc[i] = 0.f;
        __syncthreads();
        const int64_t R = rowb[ne];

        // ---- pooling over the staged rows, RT rows at a time
        for (int64_t c0 = 0; c0 < R; c0 += RT) {
            const int64_t c1 = min(R, c0 + RT);
            for (int i = tid; i < RT * (SUR_H / 8); i += NT) {
                const int row = i / (SUR_H / 8), part = i % (SUR_H / 8);
                const int64_t r = c0 + row;
                if (r >= c1) break;
                int lo = 0, hi = ne - 1;                // last event whose first row is <= r
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (rowb[mid] <= r) lo = mid;
                    else hi = mid - 1;
                }
                const int64_t img = int64_t(lo_s[lo]) + (r - rowb[lo]);
                *reinterpret_cast<uint4*>(Hs + row * LDH + 8 * part) =
                    reinterpret_cast<const uint4*>(a.H2 + img * SUR_H)[part];
            }
            __syncthreads();
            // thread = (channel pair, event group); image order within each event
            const int cp = tid & 63;
            for (int el = tid >> 6; el < ne; el += NT / 64) {
                const int64_t lo = max(rowb[el], c0), hi = min(rowb[el + 1], c1);
                if (lo >= hi) continue;
                float2 s = reinterpret_cast<float2*>(Pacc + el * SUR_H)[cp];
                for (int64_t r = lo; r < hi; ++r) {
                    const float2 h =
                        __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(Hs + (r - c0) * LDH)[cp]);
                    s.x += h.x;
                    s.y += h.y;
                }
                reinterpret_cast<float2*>(Pacc + el * SUR_H)[cp] = s;
            }
            __syncthreads();
        }

        // ---- pooled vector [sum / 40, sum / max(1, n_used)] in BF16
        for (int idx = tid; idx < FE * (SUR_H / 4); idx += NT) {
            const int el = idx / (SUR_H / 4), c4 = idx % (SUR_H / 4);
            const float4 s = reinterpret_cast<const float4*>(Pacc + el * SUR_H)[c4];
            const int nu = el < ne ? f.n_used[e0 + el] : 0;
            const float d = fmaxf(1.f, float(nu > 0 ? nu : 0));
            __nv_bfloat162* pr = reinterpret_cast<__nv_bfloat162*>(Ps + el * LDV + 4 * c4);
            pr[0] = __floats2bfloat162_rn(s.x * (1.f / SUR_POOL_DIV), s.y * (1.f / SUR_POOL_DIV));
            pr[1] = __floats2bfloat162_rn(s.z * (1.f / SUR_POOL_DIV), s.w * (1.f / SUR_POOL_DIV));
            pr[SUR_H / 2] = __floats2bfloat162_rn(s.x / d, s.y / d);
            pr[SUR_H / 2 + 1] = __floats2bfloat162_rn(s.z / d, s.w / d);
        }
        __syncthreads();

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
            sur_emit_event(a.o, e, y, f.base[e], f.n_used[e]);
        }
        __syncthreads();
    }
}

cudaError_t launch_infer(const InferArgs& a, int n_sm, cudaStream_t s) {
    if (a.tile_events < 1 || a.tile_events > FE) return cudaErrorInvalidValue;
    const int64_t units = (a.f.n_img + 15) / 16;
    if (units > 0) {
        const int64_t g = std::min<int64_t>((units + PHI_WARPS - 1) / PHI_WARPS, int64_t(n_sm) * 3);
        k_phi<<<int(g), PHI_WARPS * 32, 0, s>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaFuncSetAttribute(k_event, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SM_TOTAL));
    if (e != cudaSuccess) return e;
    k_event<<<int(std::min<int64_t>(a.n_tiles, n_sm)), NT, SM_TOTAL, s>>>(a);
    return cudaGetLastError();
}

}  // namespace rta
