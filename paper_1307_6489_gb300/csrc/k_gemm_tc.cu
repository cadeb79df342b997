// The dense contractions of the surrogate's training (forward layers, input
// gradients and weight gradients) on the fifth-generation tensor cores:
// D[M x N] = op(A) op(B), BF16 operands, FP32 accumulation in tensor memory,
// the layer's epilogue fused into the read-back.
//
// A CTA of four warps takes work items (a tile of 128 rows of D, one K-range of
// a split reduction) in a grid-stride loop and streams each item's K-chunks of
// A and B through a four-stage ring of shared-memory buffers filled by 16-byte
// asynchronous copies. One thread issues the chunk's MMAs (M = 128, N = the full
// width, K-steps of 16) into the item's TMEM accumulator and commits them to the
// stage's mbarrier; a stage is refilled once the MMAs that read it are done.
// After an item's last chunk every warp reads its 32 TMEM lanes (rows) and
// applies the epilogue.
//
// Operand staging. An operand stored with K contiguous ("K-major": A as
// [M x K], B as [N x K]) goes to the canonical K-major core-matrix layout of
// rta_tc.cuh. One stored with its rows along K ("MN-major": A as [K x M], B as
// [K x N], the activations and gradients of a weight gradient and the weights
// of a forward layer) goes to the canonical MN-major layout: core matrices of 8
// K-rows x 8 MN-values (16 contiguous bytes per K-row), core matrices adjacent
// in K 128 bytes apart (LBO), groups of 8 MN-values KC x 16 bytes apart (SBO),
// and the instruction descriptor marks the operand as MN-major. Either way a
// 16-byte piece of a stored row lands as one 16-byte piece in shared memory.
#include <algorithm>

#include "rta_mlp_dev.cuh"
#include "rta_tc.cuh"

namespace rta {
namespace {

constexpr int TC_BM = 128;   // rows of a tile = TMEM lanes
constexpr int TC_NS = 4;     // pipeline stages
constexpr int TC_NT = 128;   // four warps, one per TMEM lane quarter

// element offset of (row r, k) in an MN-major chunk of KC K-rows
__device__ __forceinline__ int mn_off(int r, int k, int KC) {
    return (r >> 3) * (8 * KC) + (k >> 3) * 64 + (k & 7) * 8 + (r & 7);
}

// 16 bytes global -> shared, zero-filled when !valid (src is not read then)
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Rows [r0, r0 + R) x K-range [k0, k0 + KC) of a stored operand into a stage.
// Rows at or beyond r_end and K at or beyond k_end read as zero.
template <bool MN, int KC>
__device__ __forceinline__ void stage_chunk(uint32_t s, const __nv_bfloat16* X, int64_t ld, int64_t r0, int R,
                                            int64_t r_end, int64_t k0, int64_t k_end, int tid) {
    if (!MN) {   // stored [rows x K]: 16-byte pieces (row, 8 K-values)
        constexpr int KP = KC / 8;
        for (int p = tid; p < R * KP; p += TC_NT) {
            const int r = p / KP, j = p % KP;
            const int64_t row = r0 + r, k = k0 + 8 * j;
            const bool ok = row < r_end && k < k_end;
            cp_async16(s + 2 * uint32_t(canon_off(r, 8 * j, KC)), ok ? X + row * ld + k : X, ok);
        }
    } else {     // stored [K x rows]: 16-byte pieces (K-row, 8 row values)
        const int RP = R / 8;
        for (int p = tid; p < KC * RP; p += TC_NT) {
            const int kk = p / RP, j = p % RP;
            const int64_t k = k0 + kk, row = r0 + 8 * j;
            const bool ok = k < k_end && row < r_end;
            cp_async16(s + 2 * uint32_t(mn_off(8 * j, kk, KC)), ok ? X + k * ld + row : X, ok);
        }
    }
}

// Position in a CTA's sequence of (item, chunk).
struct ChunkIt {
    int64_t item, c, nk, kbeg, m0;
    int z;
    bool valid;
};

__device__ __forceinline__ void it_begin(ChunkIt& t, int64_t item, int64_t n_items, int64_t n_tiles, int64_t kchunk,
                                         int64_t K, int KC) {
    t.item = item;
    t.valid = item < n_items;
    t.c = 0;
    if (!t.valid) return;
    t.m0 = (item % n_tiles) * TC_BM;
    t.z = int(item / n_tiles);
    t.kbeg = int64_t(t.z) * kchunk;
    const int64_t kend = min(K, t.kbeg + kchunk);
    t.nk = (kend - t.kbeg + KC - 1) / KC;   // >= 1: the host makes every split non-empty
}

__device__ __forceinline__ void it_next(ChunkIt& t, int64_t n_items, int64_t n_tiles, int64_t kchunk, int64_t K,
                                        int KC) {
    if (++t.c == t.nk) it_begin(t, t.item + gridDim.x, n_items, n_tiles, kchunk, K, KC);
}

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
    return pack_bf16(__float2bfloat16(lo), __float2bfloat16(hi));
}

// Epilogue of 16 columns [c0, c0 + 16) of row m.
__device__ __forceinline__ void epilogue16(const GemmArgs& g, int64_t m, int64_t M, int c0, int z,
                                           const uint32_t (&r)[16]) {
    float v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
    if (g.epi == EPI_F32_SPLIT) {    // partial sums of split z: [splits][M x N]
        float4* o = reinterpret_cast<float4*>(g.Cf + (int64_t(z) * M + m) * g.N + c0);
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        return;
    }
    if (g.epi == EPI_F32_BIAS) {    // the first n_store columns, plus bias
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (c0 + i < g.n_store) g.Cf[m * g.ldc + c0 + i] = v[i] + g.bias[c0 + i];
        return;
    }
    if (g.epi == EPI_BIAS_RELU_BF16) {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i] + g.bias[c0 + i], 0.f);
    } else if (g.epi == EPI_MASK_BF16) {
        const uint4* mk = reinterpret_cast<const uint4*>(g.mask + m * g.ldmask + c0);
        const uint4 q0 = mk[0], q1 = mk[1];
        const uint32_t w[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const uint16_t h = uint16_t(w[i / 2] >> (16 * (i & 1)));
            if (!(__bfloat162float(__ushort_as_bfloat16(h)) > 0.f)) v[i] = 0.f;
        }
    }
    uint4* o = reinterpret_cast<uint4*>(g.Cb + m * g.ldc + c0);
    o[0] = make_uint4(bf16x2(v[0], v[1]), bf16x2(v[2], v[3]), bf16x2(v[4], v[5]), bf16x2(v[6], v[7]));
    o[1] = make_uint4(bf16x2(v[8], v[9]), bf16x2(v[10], v[11]), bf16x2(v[12], v[13]), bf16x2(v[14], v[15]));
}

template <bool A_MN, bool B_MN, int KC>
__global__ void __launch_bounds__(TC_NT) k_gemm_tc(const GemmArgs g, int64_t n_tiles, int64_t n_items, int64_t kchunk,
                                                   uint32_t tmem_cols) {
    extern __shared__ __align__(128) uint8_t sm[];
    const int N = int(g.N);
    const uint32_t a_bytes = uint32_t(TC_BM * KC * 2), b_bytes = uint32_t(N * KC * 2);
    const uint32_t stage_bytes = a_bytes + b_bytes;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + TC_NS * stage_bytes);
    uint32_t* tmem_s = reinterpret_cast<uint32_t*>(bar + TC_NS);
    volatile int* abort_s = reinterpret_cast<volatile int*>(tmem_s + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t M = g.M, K = g.K;
    if (int64_t(blockIdx.x) >= n_items) return;

    if (warp == 0) {
        tc_alloc(tmem_s, tmem_cols);
        tc_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < TC_NS; ++i) mbar_init(&bar[i], 1);
        fence_mbar_init();
        *abort_s = 0;
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_s;
    const uint32_t s0 = smem_addr(sm);
    const uint32_t idesc = tc_idesc_bf16(TC_BM, N) | (uint32_t(A_MN) << 15) | (uint32_t(B_MN) << 16);
    // LBO: core matrices adjacent in K; SBO: groups of 8 rows (K-major) or 8 MN-values (MN-major)
    const uint32_t sbo = uint32_t(16 * KC);

    ChunkIt prod, cons;
    it_begin(prod, blockIdx.x, n_items, n_tiles, kchunk, K, KC);
    cons = prod;
    auto issue = [&](int stage) {
        const uint32_t sa = s0 + uint32_t(stage) * stage_bytes, sb = sa + a_bytes;
        const int64_t k0 = prod.kbeg + prod.c * KC;
        const int64_t k_end = min(K, prod.kbeg + kchunk);
        stage_chunk<A_MN, KC>(sa, g.A, g.lda, prod.m0, TC_BM, M, k0, k_end, tid);
        stage_chunk<B_MN, KC>(sb, g.B, g.ldb, 0, N, N, k0, k_end, tid);
        it_next(prod, n_items, n_tiles, kchunk, K, KC);
    };
#pragma unroll 1
    for (int s = 0; s < TC_NS - 1; ++s) {
        if (prod.valid) issue(s);
        cp_async_commit();
    }
    int64_t q = 0;
#pragma unroll 1
    while (cons.valid) {
        const int st = int(q % TC_NS);
        cp_async_wait<TC_NS - 2>();        // this thread's pieces of chunk q have landed
        fence_proxy_async_smem();
        if (__syncthreads_or(*abort_s)) break;   // ... and everyone's; one decision for the CTA
        if (tid == 0) {
            tc_fence_after();
            const uint32_t sa = s0 + uint32_t(st) * stage_bytes, sb = sa + a_bytes;
#pragma unroll 1
            for (int kk = 0; kk < KC; kk += 16) {
                const uint64_t da = tc_desc(sa + uint32_t(kk) * 16, 128, sbo);
                const uint64_t db = tc_desc(sb + uint32_t(kk) * 16, 128, sbo);
                tc_mma(tmem, da, db, idesc, cons.c > 0 || kk > 0);
            }
            tc_commit(&bar[st]);
        }
        // refill the stage chunk q - 1 used, once its MMAs are done
        if (q >= 1 && !mbar_wait(&bar[(q - 1) % TC_NS], uint32_t(((q - 1) / TC_NS) & 1), abort_s)) {
            atomicOr(g.status, RTA_DEV_TIMEOUT);
            *abort_s = 1;
        }
        if (prod.valid) issue(int((q + TC_NS - 1) % TC_NS));
        cp_async_commit();
        if (cons.c + 1 == cons.nk) {        // the item's last chunk: epilogue
            if (!mbar_wait(&bar[st], uint32_t((q / TC_NS) & 1), abort_s)) {
                atomicOr(g.status, RTA_DEV_TIMEOUT);
                *abort_s = 1;
            }
            tc_fence_after();
            const int64_t m = cons.m0 + 32 * warp + lane;
            const uint32_t t_row = tmem + (uint32_t(32 * warp) << 16);
#pragma unroll 1
            for (int c0 = 0; c0 < N; c0 += 16) {
                uint32_t r[16];
                tc_ld16(t_row + uint32_t(c0), r);
                if (m < M) epilogue16(g, m, M, c0, cons.z, r);
            }
            tc_fence_before();             // the next item's MMAs follow the next barrier
        }
        it_next(cons, n_items, n_tiles, kchunk, K, KC);
        ++q;
    }
    // teardown: no copy and no MMA of this CTA may still be in flight
    cp_async_wait<0>();
    if (q >= 1 && !mbar_wait(&bar[(q - 1) % TC_NS], uint32_t(((q - 1) / TC_NS) & 1), abort_s))
        atomicOr(g.status, RTA_DEV_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, tmem_cols);
}

template <bool A_MN, bool B_MN, int KC>
cudaError_t launch_t(const GemmArgs& g, int splits, int n_sm, cudaStream_t s) {
    const int64_t n_tiles = (g.M + TC_BM - 1) / TC_BM;
    const int64_t chunks = (g.K + KC - 1) / KC;
    const int64_t per = (chunks + splits - 1) / splits;
    const int64_t kchunk = per * KC;
    const int64_t n_items = n_tiles * ((chunks + per - 1) / per);
    const size_t smem = size_t(TC_NS) * (TC_BM + g.N) * KC * 2 + TC_NS * 8 + 16;
    uint32_t cols = 32;
    while (cols < uint32_t(g.N)) cols <<= 1;
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<A_MN, B_MN, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return e;
    // resident CTAs per SM: shared memory and the 512 TMEM columns
    const int per_sm = int(std::max<size_t>(1, std::min<size_t>(size_t(200) * 1024 / smem, 512 / cols)));
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(n_items, int64_t(n_sm) * per_sm));
    k_gemm_tc<A_MN, B_MN, KC><<<unsigned(grid), TC_NT, smem, s>>>(g, n_tiles, n_items, kchunk, cols);
    return cudaGetLastError();
}

}  // namespace

int gemm_tc_splits(int64_t K, int splits) {
    const int KC = K <= 16 ? 16 : 64;
    const int64_t chunks = (K + KC - 1) / KC;
    const int64_t per = (chunks + splits - 1) / splits;
    return int((chunks + per - 1) / per);
}

cudaError_t launch_gemm(const GemmArgs& g, bool a_mn, bool b_mn, int splits, int n_sm, cudaStream_t s) {
    if (g.M <= 0) return cudaSuccess;
    if (g.N < 16 || g.N > 256 || g.N % 16 || g.K < 1 || splits < 1) return cudaErrorInvalidValue;
    // whole 16-byte pieces: MN-major row counts and K-major reductions in multiples of 8
    if ((a_mn ? g.M : g.K) % 8 || (b_mn ? g.N : g.K) % 8) return cudaErrorInvalidValue;
    const bool f32 = g.epi == EPI_F32_SPLIT || g.epi == EPI_F32_BIAS;
    if ((uintptr_t(g.A) | uintptr_t(g.B) | uintptr_t(f32 ? (const void*)g.Cf : (const void*)g.Cb)) % 16 ||
        (g.lda | g.ldb) % 8 || (!f32 && g.ldc % 8) || (g.epi == EPI_F32_SPLIT && g.ldc != g.N) ||
        (g.epi == EPI_MASK_BF16 && (uintptr_t(g.mask) % 16 || g.ldmask % 8)))
        return cudaErrorInvalidValue;
    if (g.K <= 16) {
        if (a_mn && b_mn) return launch_t<true, true, 16>(g, splits, n_sm, s);
        if (a_mn) return launch_t<true, false, 16>(g, splits, n_sm, s);
        if (b_mn) return launch_t<false, true, 16>(g, splits, n_sm, s);
        return launch_t<false, false, 16>(g, splits, n_sm, s);
    }
    if (a_mn && b_mn) return launch_t<true, true, 64>(g, splits, n_sm, s);
    if (a_mn) return launch_t<true, false, 64>(g, splits, n_sm, s);
    if (b_mn) return launch_t<false, true, 64>(g, splits, n_sm, s);
    return launch_t<false, false, 64>(g, splits, n_sm, s);
}

}  // namespace rta
