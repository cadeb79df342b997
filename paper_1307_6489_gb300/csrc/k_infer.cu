// Inference of the deep-sets surrogate (energy, direction offset and
// gamma/hadron score next to the geometric direction, Sec. 4.1) in ONE
// persistent kernel on the fifth-generation tensor cores: a CTA of 512 threads
// per SM takes an equal share of the bundle's image rows (a range of whole
// events) and carries it from the Hillas rows to the event rows, geometric
// fallback included, in tiles of at most 128 events:
//
//   1. the tile's Hillas rows arrive by one bulk copy; per event (four lanes)
//      the used images and the two-image baseline;
//   2. per pass of up to 512 image rows: the features of every row, then the
//      first layer (16 -> 128) of all four 128-row blocks in one batch of MMAs
//      (TMEM columns 128 j for block j), then per block the second layer
//      (128 -> 128) and the sum over each event's used images. The blocks are
//      pipelined: while the second layer of block j + 1 runs on the tensor
//      core, the CTA converts and pools block j; block j + 1's first-layer
//      activations are converted in the same step as block j's second-layer
//      ones;
//   3. the pooled vectors [sum / 40, mean] as the A operand of the event
//      network 256 -> 256 (ReLU) on the tensor core; the 256 -> 4 output layer
//      on the CUDA cores, straight from the event network's BF16-rounded
//      activations in registers (exact BF16 products summed in FP32, each
//      thread over its 64 columns, the four partial sums then in fixed order);
//   4. the events whose learned offset exceeds the fallback bound get the
//      stereo intersection of their images, computed with the stereo kernel's
//      own pieces and grouping (rta_stereo_dev.cuh), so their direction equals
//      rta_stereo's bit for bit.
//
// tcgen05 usage: operands in shared memory as canonical K-major core matrices
// (rta_tc.cuh), FP32 accumulators in tensor memory (all 512 columns: four
// blocks of the per-telescope layers, later the event network), one thread
// issuing the MMAs and committing them to an mbarrier that the CTA waits on
// with a time limit; four warps share each TMEM lane quarter, each taking a
// slice of the columns. Weights arrive by bulk copies; the event network's
// 128 KB V1^T shares its shared memory with the per-telescope stage (its head
// follows the last second-layer MMA, its tail the last pooling).
//
// The kernel is launched with programmatic dependent launch. Before
// griddepcontrol.wait it allocates tensor memory, sets up barriers and loads
// the registered telescope tables; when the caller declares the inputs settled
// (the fused image-kernel + inference call, whose preceding kernel is the image
// kernel), the event offsets, telescope ids and weights are read before the
// wait as well, so that the CTA's event range and its first tile's layout are
// ready when the image kernel's rows become visible.
//
// The features and the per-event reductions are the training path's own
// expressions (rta_mlp_dev.cuh), so baselines and used counts equal those of
// k_features bit for bit (the same lanes per event); every event's pooled sums
// run over its rows in image order whatever the tile and block boundaries, so
// an event's outputs do not depend on the events around it.
#include <algorithm>

#include "rta_mlp_dev.cuh"
#include "rta_stereo_dev.cuh"
#include "rta_tc.cuh"

namespace rta {
namespace {

constexpr int NT = 512;             // threads per CTA (sixteen warps: four per TMEM lane quarter)
constexpr int NW = NT / 32;
constexpr int NSLICE = NW / 4;      // column slices of a TMEM row (warps sharing a lane quarter)
constexpr int ST_NTC = 256;         // threads of the CTA-wide stereo (as in the stereo kernel)
constexpr int TM = 128;             // MMA M: image rows per block, events per tile at most
constexpr int NBLK = 4;             // blocks per pass: their accumulators fill the 512 TMEM columns
constexpr int SB = NBLK * TM;       // image rows per pass
constexpr uint32_t TMEM_COLS = NBLK * SUR_H;
constexpr int LDH = SUR_H + 8;      // row stride of the row-major second-layer tile used for pooling
static_assert(TMEM_COLS == 512 && SUR_G <= int(TMEM_COLS), "tensor memory plan");

// Shared memory. Region U holds, during the per-telescope stage, W1^T and W2^T,
// the pass's features, the first-layer activations of one block, and the
// tile's staged Hillas rows, whose place the second-layer tile takes once the
// features are formed; during the event stage V1^T; the fallback's staged
// images after that.
constexpr size_t W_BYTES = size_t(PK_V1T - PK_W1T) * 2;          // 36,864
constexpr size_t U_W = 0;                                         // bf16 W1^T [128][16], W2^T [128][128]
constexpr size_t U_X = U_W + W_BYTES;                             // bf16 features: four canonical [128][16] blocks
constexpr size_t U_H1 = U_X + size_t(SB) * SUR_XPAD * 2;          // bf16 first-layer activations, canonical [128][128]
constexpr size_t U_ROWS = U_H1 + size_t(TM) * SUR_H * 2;          // staged rows; then bf16 H2 row-major [128][LDH]
constexpr size_t V1_BYTES = size_t(SUR_G) * SUR_G * 2;            // 131,072
constexpr size_t U_SIZE = V1_BYTES;
constexpr int MAX_STAGED_ROWS = SB;                               // a staged tile is one pass
static_assert(U_ROWS + size_t(MAX_STAGED_ROWS) * sizeof(rta_hillas_t) <= U_SIZE, "staged rows fit");
static_assert(U_ROWS + size_t(TM) * LDH * 2 <= U_SIZE, "second-layer tile fits");
constexpr int PSTRIDE = SUR_H + 4;                                // pooling-sum row stride (floats)
constexpr size_t S_P = U_SIZE;                                    // f32 pooling sums [128][PSTRIDE], then bf16 P
                                                                  // [128][256], then f32 output partials
constexpr size_t S_P_BYTES = size_t(TM) * PSTRIDE * 4;
constexpr size_t S_TCAM = S_P + S_P_BYTES;                        // int [1024] camera of each telescope
constexpr size_t S_TXY = S_TCAM + size_t(RTA_MAX_TEL) * 4;        // float2 [1024] telescope positions
constexpr size_t S_CODE = S_TXY + size_t(RTA_MAX_TEL) * 8;        // f32 [16] camera codes
constexpr size_t S_B1 = S_CODE + size_t(RTA_MAX_CAMS) * 4;        // f32 [128]
constexpr size_t S_B2 = S_B1 + SUR_H * 4;                         // f32 [128]
constexpr size_t S_C1 = S_B2 + SUR_H * 4;                         // f32 [256]
constexpr size_t S_C2 = S_C1 + SUR_G * 4;                         // f32 [4]
constexpr size_t S_V2 = S_C2 + 16;                                // f32 [256][4]: the output layer's BF16 weights
constexpr size_t S_ROWB = S_V2 + size_t(SUR_G) * 4 * 4;           // int64 [129] first row of each event
constexpr size_t S_BASE = S_ROWB + size_t(TM + 1) * 8;            // float2 [128]
constexpr size_t S_EOFF = S_BASE + size_t(TM) * 8;                // int [129 + pad] the tile's event offsets
constexpr size_t S_LO = S_EOFF + size_t(TM + 4) * 4;              // int [128] first image
constexpr size_t S_CNT = S_LO + size_t(TM) * 4;                   // int [128] images (0 if malformed)
constexpr size_t S_NU = S_CNT + size_t(TM) * 4;                   // int [128] used images (-1 if malformed)
constexpr size_t S_INV = S_NU + size_t(TM) * 4;                   // f32 [128] 1 / max(1, used images)
constexpr size_t S_FB = S_INV + size_t(TM) * 4;                   // int [128] fallback list; [128] its count
constexpr size_t S_FBB = S_FB + size_t(TM + 4) * 4;               // int [128] fallback events for the CTA; [128] count
constexpr size_t S_RED = S_FBB + size_t(TM + 4) * 4;              // DW [8][5], int [8][2]: CTA-wide stereo sums
constexpr size_t S_TEL = S_RED + size_t(ST_NTC / 32) * (5 * sizeof(DW) + 2 * 4);    // int [512] staged rows' telescopes
constexpr size_t S_USED = S_TEL + size_t(MAX_STAGED_ROWS) * 4;    // u8 [SB] row takes part
constexpr size_t S_EVR = S_USED + SB;                             // u8 [SB] the row's event in the tile
constexpr size_t S_OK = S_EVR + SB;                               // u8 [128] event offsets well formed
constexpr size_t S_BAR = S_OK + TM;                               // 5 mbarriers, TMEM address, abort flag
constexpr size_t S_TOTAL = S_BAR + 64;
static_assert(U_X % 16 == 0 && U_H1 % 16 == 0 && U_ROWS % 16 == 0 && S_V2 % 16 == 0, "U layout");
static_assert(S_P % 16 == 0 && S_P_BYTES >= size_t(TM) * SUR_G * 2 && S_P_BYTES >= size_t(NSLICE) * TM * 16,
              "pooling region holds the P operand and the output partials");
static_assert(S_TXY % 8 == 0 && S_ROWB % 8 == 0 && S_BASE % 8 == 0 && S_RED % 8 == 0 && S_BAR % 8 == 0,
              "aligned tables");
constexpr size_t U_FBROWS = size_t(NW) * RTA_STEREO_MAX_M * sizeof(StereoImg);   // the tile's rows again, for the fallback
static_assert(U_FBROWS % 16 == 0 && U_FBROWS + size_t(MAX_STAGED_ROWS) * sizeof(rta_hillas_t) <= U_SIZE,
              "fallback staging and the rows it reads fit U");
static_assert(S_TOTAL <= 227 * 1024, "one CTA per SM");
static_assert(TM <= 255, "a row's event index fits a byte");
static_assert(SB == NT, "one feature row per thread and pass");
constexpr int ISSUER = NT - 32;     // lane 0 of the last warp issues the pipelined second-layer MMAs
constexpr int NPOOL = 7 * 64;       // pooling threads: seven event groups of 64 channel pairs
static_assert(ISSUER >= NPOOL, "the issuing warp does not pool");

// One thread: copy `bytes` (a multiple of 16) from global to shared memory with
// the bulk-copy engine in pieces of at most 32 KB, all completing on bar.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t policy) {
    for (uint32_t o = 0; o < bytes; o += 32768u)
        bulk_g2s(static_cast<char*>(dst) + o, static_cast<const char*>(src) + o, min(32768u, bytes - o), bar, policy);
}

// Wait for the phase `phase` of bar (MMAs or copies); on a timeout flag the
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

// The CTA's events: CTA b of G takes [B_b, max(B_b, B_b+1)) with B_0 = 0,
// B_G = n_evt and B_j the first event whose first image is at or past the j-th
// G-quantile of the images, so that every CTA gets about the same number of image
// rows (events have 2-40 images). Each B_j is found by a sampled search (128
// threads per bound, a round of loads per 128-fold narrowing) that depends only
// on j and the offsets, so neighbouring CTAs agree on their common bound; for
// offsets that are not ascending the bounds are still in [0, n_evt], and the
// max() rule still gives every event to some CTA. scratch: 2 ints of shared memory.
__device__ __forceinline__ void event_range(const int32_t* evt_off, int64_t n_evt, int* scratch, int64_t& begin,
                                            int64_t& end) {
    const int tid = threadIdx.x, half = (tid >> 7) & 1, k = tid & 127;
    const bool act = tid < 256;                         // threads past 256 only join the barriers
    const int64_t G = gridDim.x, b = blockIdx.x;
    const int32_t first = evt_off[0], last = evt_off[n_evt];
    const int64_t j = b + half;                         // bound B_b (half 0) and B_b+1 (half 1)
    int64_t lo = 0, hi = n_evt;                         // the bound lies in [lo, hi]
    if (j == 0 || !act) hi = 0;
    if (j == G) lo = n_evt;
    for (;;) {
        const bool open = act && lo < hi;
        if (!__syncthreads_or(open)) break;
        if (act && k == 0) scratch[half] = 128;
        __syncthreads();
        const int64_t step = open ? max(int64_t(1), (hi - lo + 127) / 128) : 1;
        const int64_t pk = lo + k * step;
        const int64_t v = open && pk < hi ? int64_t(evt_off[pk]) : 0;
        // the target after the sample's load: the first round's loads overlap
        const int64_t total = max(int64_t(0), int64_t(last) - first);
        const int64_t target = first + (total * j) / G;
        if (open && pk < hi && v >= target) atomicMin(&scratch[half], k);
        __syncthreads();
        if (open) {
            const int kk = scratch[half];
            if (kk == 128) {
                lo = lo + ((hi - lo - 1) / step) * step + 1;   // past the last sample
            } else {
                const int64_t hk = lo + kk * step;
                lo = kk == 0 ? lo : lo + (kk - 1) * step + 1;
                hi = hk;
            }
        }
    }
    if (act && k == 0) scratch[half] = int(lo);
    __syncthreads();
    begin = scratch[0];
    end = max(begin, int64_t(scratch[1]));
    __syncthreads();
}

}  // namespace

namespace {

// ReLU(acc + bias) of 32 TMEM columns of this thread's row, rounded to BF16
// pairs (the activation as the next layer sees it).
__device__ __forceinline__ void relu_bf16_32(uint32_t taddr, const float* __restrict__ bias, uint32_t (&w)[16],
                                             bool keep) {
    uint32_t v[32];
    tc_ld32(taddr, v);
#pragma unroll
    for (int i = 0; i < 16; ++i)
        w[i] = bf2_bits(__floats2bfloat162_rn(keep ? fmaxf(__uint_as_float(v[2 * i]) + bias[2 * i], 0.f) : 0.f,
                                              keep ? fmaxf(__uint_as_float(v[2 * i + 1]) + bias[2 * i + 1], 0.f)
                                                   : 0.f));
}

// Shared-memory accesses by 32-bit shared-window address.
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ float2 lds_f2(uint32_t a) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts_f2(uint32_t a, float2 v) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
// A BF16 pair (low half first) as two floats: exact.
__device__ __forceinline__ float2 bf2_to_f2(uint32_t v) {
    return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xFFFF0000u));
}

// Sums of the second-layer tile's rows [lo, up) (relative to the block) of one
// event, channel pair cp (h2: the pair's shared address in row 0; acc: the
// event's running sums of the pair), added in row order.
__device__ __forceinline__ void pool_rows(uint32_t h2, uint32_t acc, int lo, int up) {
    constexpr uint32_t RS = LDH * 2;         // bytes per row
    float2 s = lds_f2(acc);
    int r = lo;
    for (; r + 4 <= up; r += 4) {
        const uint32_t base = h2 + uint32_t(r) * RS;
        const uint32_t v0 = lds_u32(base), v1 = lds_u32(base + RS), v2 = lds_u32(base + 2 * RS),
                       v3 = lds_u32(base + 3 * RS);
        const float2 a0 = bf2_to_f2(v0), a1 = bf2_to_f2(v1), a2 = bf2_to_f2(v2), a3 = bf2_to_f2(v3);
        s.x += a0.x;
        s.y += a0.y;
        s.x += a1.x;
        s.y += a1.y;
        s.x += a2.x;
        s.y += a2.y;
        s.x += a3.x;
        s.y += a3.y;
    }
    for (; r < up; ++r) {
        const float2 a0 = bf2_to_f2(lds_u32(h2 + uint32_t(r) * RS));
        s.x += a0.x;
        s.y += a0.y;
    }
    sts_f2(acc, s);
}

}  // namespace

// ------------------------------------------------------------------ the kernel
__global__ void __launch_bounds__(NT, 1) k_deepsets_infer(const InferArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __nv_bfloat16* Ws = reinterpret_cast<__nv_bfloat16*>(sm + U_W);
    __nv_bfloat16* Xs = reinterpret_cast<__nv_bfloat16*>(sm + U_X);
    __nv_bfloat16* H1s = reinterpret_cast<__nv_bfloat16*>(sm + U_H1);
    __nv_bfloat16* H2s = reinterpret_cast<__nv_bfloat16*>(sm + U_ROWS);
    rta_hillas_t* rows_s = reinterpret_cast<rta_hillas_t*>(sm + U_ROWS);
    float* Pacc = reinterpret_cast<float*>(sm + S_P);
    __nv_bfloat16* Ps = reinterpret_cast<__nv_bfloat16*>(sm + S_P);
    float* outp = reinterpret_cast<float*>(sm + S_P);
    int* tcam_s = reinterpret_cast<int*>(sm + S_TCAM);
    float2* txy_s = reinterpret_cast<float2*>(sm + S_TXY);
    float* code_s = reinterpret_cast<float*>(sm + S_CODE);
    float* b1s = reinterpret_cast<float*>(sm + S_B1);
    float* b2s = reinterpret_cast<float*>(sm + S_B2);
    float* c1s = reinterpret_cast<float*>(sm + S_C1);
    float* c2s = reinterpret_cast<float*>(sm + S_C2);
    float* V2f = reinterpret_cast<float*>(sm + S_V2);
    int64_t* rowb = reinterpret_cast<int64_t*>(sm + S_ROWB);
    float2* base_s = reinterpret_cast<float2*>(sm + S_BASE);
    int* eoff_s = reinterpret_cast<int*>(sm + S_EOFF);
    int* lo_s = reinterpret_cast<int*>(sm + S_LO);
    int* cnt_s = reinterpret_cast<int*>(sm + S_CNT);
    int* nu_s = reinterpret_cast<int*>(sm + S_NU);
    float* inv_s = reinterpret_cast<float*>(sm + S_INV);
    int* fb_s = reinterpret_cast<int*>(sm + S_FB);
    int* fb_n = fb_s + TM;
    int* fbb_s = reinterpret_cast<int*>(sm + S_FBB);
    int* fbb_n = fbb_s + TM;
    DW* red_s = reinterpret_cast<DW*>(sm + S_RED);
    int* redi_s = reinterpret_cast<int*>(sm + S_RED + size_t(ST_NTC / 32) * 5 * sizeof(DW));
    int* tel_s = reinterpret_cast<int*>(sm + S_TEL);
    uint8_t* used_s = sm + S_USED;
    uint8_t* evr_s = sm + S_EVR;
    uint8_t* ok_s = sm + S_OK;
    uint64_t* bar_mma = reinterpret_cast<uint64_t*>(sm + S_BAR);    // MMA completion
    uint64_t* bar_w = bar_mma + 1;                                    // W1^T, W2^T copy
    uint64_t* bar_rows = bar_mma + 2;                                 // the tile's Hillas rows
    uint64_t* bar_vt = bar_mma + 3;                                   // V1^T tail copy
    uint64_t* bar_vh = bar_mma + 4;                                   // V1^T head copy
    uint32_t* tmem_s = reinterpret_cast<uint32_t*>(sm + S_BAR + 48);
    volatile int* abort_s = reinterpret_cast<volatile int*>(sm + S_BAR + 52);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const FeatArgs& f = a.f;
    const int n_tel = min(f.n_tel, RTA_MAX_TEL);
    const bool settled = a.settled != 0;

    // ---- set-up that reads nothing earlier stream work may write
    if (warp == 0) {
        tc_alloc(tmem_s, TMEM_COLS);
        tc_relinquish();
    }
    if (tid == 0) {
        mbar_init(bar_mma, 1);
        mbar_init(bar_w, 1);
        mbar_init(bar_rows, 1);
        mbar_init(bar_vt, 1);
        mbar_init(bar_vh, 1);
        fence_mbar_init();
        *abort_s = 0;
    }
    // ---- the set-up's inputs: the registered telescope tables (registration copies,
    // complete before any launch), then, once they may be read (before the wait only when the
    // caller declared them settled), the weights and the CTA's event range. Every load is
    // issued before the first store, so that their latencies overlap the range search.
    int tc[RTA_MAX_TEL / NT];
    float2 txy[RTA_MAX_TEL / NT];
#pragma unroll
    for (int k = 0; k < RTA_MAX_TEL / NT; ++k) {
        const int i = tid + k * NT;
        tc[k] = i < n_tel ? f.tel_cam[i] : 0;
        txy[k] = i < n_tel ? f.tel_xy[i] : make_float2(0.f, 0.f);
    }
    const float code = tid < RTA_MAX_CAMS ? f.cam_code[tid] : 0.f;
    if (!settled) grid_dependency_wait();
    // a batch gathered on the device gives its counts at run time (capacities in f)
    const int64_t n_evt = f.n_evt_dev ? min(*f.n_evt_dev, f.n_evt) : f.n_evt;
    const int64_t n_img = f.n_img_dev ? min(*f.n_img_dev, f.n_img) : f.n_img;
    if (tid == 0) {
        mbar_arrive_expect_tx(bar_w, uint32_t(W_BYTES));
        bulk_copy(Ws, a.pk + PK_W1T, uint32_t(W_BYTES), bar_w, l2_policy_evict_last());
    }
    const float bb1 = tid < SUR_H ? a.p[OFF_B1 + tid] : 0.f, bb2 = tid < SUR_H ? a.p[OFF_B2 + tid] : 0.f;
    const float c1 = tid < SUR_G ? a.p[OFF_C1 + tid] : 0.f, c2 = tid < 4 ? a.p[OFF_C2 + tid] : 0.f;
    float v2[SUR_G * 4 / NT];
#pragma unroll
    for (int k = 0; k < SUR_G * 4 / NT; ++k) v2[k] = __bfloat162float(a.pb[OFF_V2 + tid + k * NT]);
    int64_t ev_begin, ev_end;
    event_range(f.evt_off, n_evt, fb_s, ev_begin, ev_end);
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
    if (tid < SUR_G) c1s[tid] = c1;
    if (tid < 4) c2s[tid] = c2;
#pragma unroll
    for (int k = 0; k < SUR_G * 4 / NT; ++k) V2f[tid + k * NT] = v2[k];   // [k][o], o fastest
    for (int i = tid; i < TM * PSTRIDE; i += NT) Pacc[i] = 0.f;           // the first tile's pooling sums
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_s;
    const uint32_t idesc_h = tc_idesc_bf16(TM, SUR_H), idesc_g = tc_idesc_bf16(TM, SUR_G);
    const uint32_t x_addr = smem_addr(Xs), h1_addr = smem_addr(H1s), w1_addr = smem_addr(Ws),
                   w2_addr = smem_addr(Ws + SUR_H * SUR_XPAD), p_addr = smem_addr(Ps), v_addr = smem_addr(sm);
    const int q = warp & 3, row = 32 * q + lane, slice = warp >> 2;
    const int c_off = slice * (SUR_H / NSLICE), g_off = slice * (SUR_G / NSLICE);
    const uint32_t t_lane = uint32_t(32 * q) << 16;
    const int sub = lane % SUR_EVT_LANES, grp = lane / SUR_EVT_LANES;
    uint32_t ph_mma = 0, ph_w = 0, ph_rows = 0, ph_vt = 0, ph_vh = 0;
    bool alive = true;
    // what thread 0 has issued and the CTA has not yet waited for (drained before exit)
    bool mma_fly = false, w_fly = (tid == 0), rows_fly = false, vt_fly = false, vh_fly = false;

    bool first_tile = true;
    for (int64_t e0 = ev_begin; e0 < ev_end; e0 += TM) {
        const int ne = int(min(int64_t(TM), ev_end - e0));
        if (!first_tile) {
            // the event stage overwrote W1^T / W2^T and the pooling sums
            if (tid == 0) {
                mbar_arrive_expect_tx(bar_w, uint32_t(W_BYTES));
                bulk_copy(Ws, a.pk + PK_W1T, uint32_t(W_BYTES), bar_w, l2_policy_evict_last());
                w_fly = true;
            }
            for (int i = tid; i < TM * PSTRIDE; i += NT) Pacc[i] = 0.f;
        }
        // ---- the tile's layout from its event offsets (inputs: before the wait when settled)
        const int eo = tid <= ne ? f.evt_off[e0 + tid] : 0;
        if (tid <= ne) eoff_s[tid] = eo;
        if (tid == 0) *fb_n = *fbb_n = 0;
        __syncthreads();
        // the tile's Hillas rows are staged when its offsets are well formed (ascending,
        // inside [0, n_img]) and they fit one pass; else every row is read from global memory
        const bool ordered = tid >= ne || (eoff_s[tid] <= eoff_s[tid + 1] && eoff_s[tid] >= 0 && eoff_s[tid + 1] <= n_img);
        const bool wellformed = __syncthreads_and(ordered);
        const int R0 = wellformed ? eoff_s[ne] - eoff_s[0] : 0;
        const bool staged = wellformed && a.rows_aligned && R0 > 0 && R0 <= MAX_STAGED_ROWS;
        const int row_first = staged ? eoff_s[0] : 0;
        if (wellformed && tid <= ne) rowb[tid] = int64_t(eoff_s[tid]) - eoff_s[0];   // the tile's rows in order
        if (tid < ne) {
            const int i0 = eoff_s[tid], i1 = eoff_s[tid + 1];
            const bool ok = !(i0 < 0 || i1 < i0 || i1 > n_img);
            lo_s[tid] = i0;
            cnt_s[tid] = ok ? i1 - i0 : 0;
            ok_s[tid] = ok;
        }
        if (staged)
            for (int k = tid; k < R0; k += NT) tel_s[k] = f.img_tel[row_first + k];
        __syncthreads();
        if (!wellformed && warp == 0) {
            // first row of each event in the tile: a scan of the row counts (0 for a
            // malformed event), four per lane
            int64_t v[4], run = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int el = 4 * lane + k;
                run += el < ne ? cnt_s[el] : 0;
                v[k] = run;
            }
            int64_t x = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t u = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += u;
            }
            const int64_t before = x - run;
#pragma unroll
            for (int k = 0; k < 4; ++k) rowb[4 * lane + k + 1] = before + v[k];
            if (lane == 0) rowb[0] = 0;
        }
        // ---- from here on the preceding kernel's Hillas rows are read
        if (first_tile && settled) grid_dependency_wait();
        if (staged) {
            if (tid == 0) {
                const uint32_t bytes = uint32_t(R0) * uint32_t(sizeof(rta_hillas_t));
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar_rows, bytes);
                bulk_copy(rows_s, f.h + row_first, bytes, bar_rows, l2_policy_evict_first());
                rows_fly = true;
            }
            alive = tc_wait(bar_rows, ph_rows, abort_s, a.o.status);
            if (!alive) break;
            ph_rows ^= 1u;
            rows_fly = false;
        } else {
            __syncthreads();
        }
        const rta_hillas_t* hrows = staged ? rows_s : f.h;
        // ---- per-event prologue, SUR_EVT_LANES lanes per event (as k_features)
        for (int p0 = 0; p0 < ne; p0 += NT / SUR_EVT_LANES) {
            const int el = p0 + (32 / SUR_EVT_LANES) * warp + grp;
            const int i0 = el < ne ? lo_s[el] : 0, n = el < ne ? cnt_s[el] : 0;
            float bx, by;
            int cnt;
            sur_event_baseline(hrows, i0 - row_first, n, sub, nullptr, bx, by, cnt);
            if (sub == 0 && el < ne) {
                const bool ok = ok_s[el];
                base_s[el] = make_float2(bx, by);
                nu_s[el] = ok ? cnt : -1;
                inv_s[el] = __frcp_rn(fmaxf(1.f, float(ok ? cnt : 0)));   // = 1.f / n (both round to nearest)
            }
        }
        __syncthreads();
        const int64_t R = rowb[ne];
        bool w_pending = true;                          // this tile's W1^T, W2^T not yet waited for

        for (int64_t pb = 0; pb < R; pb += SB) {
            const int nbk = int((min(int64_t(SB), R - pb) + TM - 1) / TM);   // blocks in this pass
            const bool last_pass = pb + SB >= R;
            // ---- features of rows pb .. pb + SB - 1 (one per thread); rows past R are zero
            {
                const int qr = tid;
                const int64_t r = pb + qr;
                __nv_bfloat162 x[SUR_XPAD / 2];
                bool used = false;
                int ev = 0;
                if (r < R) {
                    int lo = 0, hi = ne - 1;              // last event whose first row is <= r
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (rowb[mid] <= r) lo = mid;
                        else hi = mid - 1;
                    }
                    ev = lo;
                    const int64_t img = int64_t(lo_s[lo]) + (r - rowb[lo]);
                    const rta_hillas_t h = hrows[img - row_first];
                    const int tel = staged ? tel_s[img - row_first] : f.img_tel[img];
                    used = sur_used(h);
                    const float2 b = base_s[lo];
                    sur_image_features(h, tel, tcam_s, txy_s, code_s, n_tel, b.x, b.y, x);
                } else {
#pragma unroll
                    for (int j = 0; j < SUR_XPAD / 2; ++j) x[j] = __floats2bfloat162_rn(0.f, 0.f);
                }
                __nv_bfloat16* xt = Xs + (qr / TM) * (TM * SUR_XPAD);
                *reinterpret_cast<uint4*>(xt + canon_off(qr % TM, 0, SUR_XPAD)) =
                    make_uint4(bf2_bits(x[0]), bf2_bits(x[1]), bf2_bits(x[2]), bf2_bits(x[3]));
                *reinterpret_cast<uint4*>(xt + canon_off(qr % TM, 8, SUR_XPAD)) =
                    make_uint4(bf2_bits(x[4]), bf2_bits(x[5]), bf2_bits(x[6]), bf2_bits(x[7]));
                used_s[qr] = used;
                evr_s[qr] = uint8_t(ev);
            }
            fence_proxy_async_smem();
            __syncthreads();
            if (w_pending) {                            // W1^T, W2^T of this tile
                alive = tc_wait(bar_w, ph_w, abort_s, a.o.status);
                if (!alive) break;
                ph_w ^= 1u;
                w_pending = w_fly = false;
            }
            // ---- first layer of every block of the pass: D1(j) = X_j W1 into TMEM columns 128 j
            if (tid == 0) {
                tc_fence_after();
                for (int j = 0; j < nbk; ++j)
                    tc_mma(tmem + uint32_t(SUR_H * j), tc_desc(x_addr + uint32_t(j * TM * SUR_XPAD * 2), 128u, 16u * SUR_XPAD),
                           tc_desc(w1_addr, 128u, 16u * SUR_XPAD), idesc_h, false);
                tc_commit(bar_mma);
                mma_fly = true;
            }
            alive = tc_wait(bar_mma, ph_mma, abort_s, a.o.status);
            if (!alive) break;
            ph_mma ^= 1u;
            mma_fly = false;
            // block 0's activations -> canonical operand of its second layer (this thread: one row,
            // 32 columns)
            if (32 * q < int(min(int64_t(TM), R - pb))) {
                uint32_t w[16];
                relu_bf16_32(tmem + t_lane + uint32_t(c_off), b1s + c_off, w, true);
#pragma unroll
                for (int q8 = 0; q8 < 4; ++q8)
                    *reinterpret_cast<uint4*>(H1s + canon_off(row, c_off + 8 * q8, SUR_H)) =
                        make_uint4(w[4 * q8], w[4 * q8 + 1], w[4 * q8 + 2], w[4 * q8 + 3]);
            }
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {                             // second layer of block 0 (eight K-steps)
                tc_fence_after();
#pragma unroll 1
                for (int ks = 0; ks < SUR_H / 16; ++ks)
                    tc_mma(tmem, tc_desc(h1_addr + 256u * ks, 128u, 16u * SUR_H),
                           tc_desc(w2_addr + 256u * ks, 128u, 16u * SUR_H), idesc_h, ks > 0);
                tc_commit(bar_mma);
                mma_fly = true;
            }
            // ---- the blocks, pipelined: block j's second layer completes; block j + 1's first-layer
            // activations and block j's second-layer activations are converted together; block
            // j + 1's second layer then runs on the tensor core while the CTA pools block j
            for (int j = 0; j < nbk; ++j) {
                alive = tc_wait(bar_mma, ph_mma, abort_s, a.o.status);
                if (!alive) break;
                ph_mma ^= 1u;
                mma_fly = false;
                const bool more = j + 1 < nbk;
                const bool last_block = last_pass && !more;
                // rows of blocks j and j + 1; a warp whose 32 rows lie past them converts nothing
                // (those accumulator rows are never read)
                const int nr_j = int(min(int64_t(TM), R - pb - int64_t(TM) * j));
                const int nr_k = more ? int(min(int64_t(TM), R - pb - int64_t(TM) * (j + 1))) : 0;
                if (last_block && tid == 0) {
                    // the tensor core is done with W, X and H1: the head of V1^T may land there
                    mbar_arrive_expect_tx(bar_vh, uint32_t(U_ROWS));
                    bulk_copy(sm, a.pk + PK_V1T, uint32_t(U_ROWS), bar_vh, l2_policy_evict_last());
                    vh_fly = true;
                }
                if (32 * q < nr_k) {
                    uint32_t w[16];
                    relu_bf16_32(tmem + t_lane + uint32_t(SUR_H * (j + 1) + c_off), b1s + c_off, w, true);
#pragma unroll
                    for (int q8 = 0; q8 < 4; ++q8)
                        *reinterpret_cast<uint4*>(H1s + canon_off(row, c_off + 8 * q8, SUR_H)) =
                            make_uint4(w[4 * q8], w[4 * q8 + 1], w[4 * q8 + 2], w[4 * q8 + 3]);
                }
                if (32 * q < nr_j) {
                    // ReLU(D2 + b2) in BF16, zero rows for unused images -> row-major tile for pooling
                    uint32_t w[16];
                    relu_bf16_32(tmem + t_lane + uint32_t(SUR_H * j + c_off), b2s + c_off, w, used_s[j * TM + row] != 0);
                    uint4* hr = reinterpret_cast<uint4*>(H2s + row * LDH + c_off);
#pragma unroll
                    for (int q8 = 0; q8 < 4; ++q8) hr[q8] = make_uint4(w[4 * q8], w[4 * q8 + 1], w[4 * q8 + 2], w[4 * q8 + 3]);
                }
                fence_proxy_async_smem();
                tc_fence_before();
                __syncthreads();
                if (more && tid == ISSUER) {            // second layer of block j + 1
                    tc_fence_after();
                    const uint32_t d = tmem + uint32_t(SUR_H * (j + 1));
#pragma unroll 1
                    for (int ks = 0; ks < SUR_H / 16; ++ks)
                        tc_mma(d, tc_desc(h1_addr + 256u * ks, 128u, 16u * SUR_H),
                               tc_desc(w2_addr + 256u * ks, 128u, 16u * SUR_H), idesc_h, ks > 0);
                    tc_commit(bar_mma);
                    mma_fly = true;
                }
                // ---- pooling of block j: thread = (channel pair, event group) of the first NPOOL
                // threads (the issuing warp, held up while its MMAs are accepted, takes no part); each
                // event's sums run over its rows in image order, continuing from the blocks before
                if (tid < NPOOL) {
                    const int64_t r0 = pb + int64_t(TM) * j;
                    const int nr = int(min(int64_t(TM), R - r0));
                    const int e_first = evr_s[j * TM], e_last = evr_s[j * TM + nr - 1];
                    const int cp = tid & 63, g8 = tid >> 6;
                    const uint32_t h2a = smem_addr(H2s) + uint32_t(cp) * 4u, pacc_a = smem_addr(Pacc);
                    for (int el = e_first + g8; el <= e_last; el += NPOOL / 64) {
                        const int lo = int(max(rowb[el], r0) - r0), up = int(min(rowb[el + 1], r0 + nr) - r0);
                        if (lo < up) pool_rows(h2a, pacc_a + uint32_t(el * PSTRIDE * 4 + cp * 8), lo, up);
                    }
                }
                fence_proxy_async_smem();               // the V1^T tail copy may overwrite the tile next
                __syncthreads();
            }
            if (!alive) break;
        }
        if (!alive) break;
        if (w_pending) {                                // a tile without image rows: the copy must still land
            alive = tc_wait(bar_w, ph_w, abort_s, a.o.status);
            if (!alive) break;
            ph_w ^= 1u;
            w_fly = false;
        }
        // ---- the per-telescope stage is done with region U: the rest of V1^T follows in
        if (tid == 0) {
            fence_proxy_async_smem();
            if (R == 0) {
                mbar_arrive_expect_tx(bar_vh, uint32_t(U_ROWS));
                bulk_copy(sm, a.pk + PK_V1T, uint32_t(U_ROWS), bar_vh, l2_policy_evict_last());
                vh_fly = true;
            }
            mbar_arrive_expect_tx(bar_vt, uint32_t(U_SIZE - U_ROWS));
            bulk_copy(sm + U_ROWS, a.pk + PK_V1T + U_ROWS / 2, uint32_t(U_SIZE - U_ROWS), bar_vt, l2_policy_evict_last());
            vt_fly = true;
        }
        // ---- pooled vectors [sum / 40, sum * RN(1 / max(1, n_used))] in BF16, in place of the sums.
        // Item i of this thread: event 8 (k / 128) + k % 8 and channels 8 ((k / 8) % 16) .. + 7,
        // k = tid + 512 i; every sum is read before any operand is written.
        {
            constexpr int NIT = TM * (SUR_H / 8) / NT;       // items per thread
            float sv[NIT][8];
#pragma unroll
            for (int it = 0; it < NIT; ++it) {
                const int k = tid + NT * it;
                const int el = 8 * (k >> 7) + (k & 7), ch = 8 * ((k >> 3) & 15);
                const bool live = el < ne;
                const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 u0 = live ? *reinterpret_cast<const float4*>(Pacc + el * PSTRIDE + ch) : z;
                const float4 u1 = live ? *reinterpret_cast<const float4*>(Pacc + el * PSTRIDE + ch + 4) : z;
                sv[it][0] = u0.x; sv[it][1] = u0.y; sv[it][2] = u0.z; sv[it][3] = u0.w;
                sv[it][4] = u1.x; sv[it][5] = u1.y; sv[it][6] = u1.z; sv[it][7] = u1.w;
            }
            __syncthreads();
#pragma unroll
            for (int it = 0; it < NIT; ++it) {
                const int k = tid + NT * it;
                const int el = 8 * (k >> 7) + (k & 7), ch = 8 * ((k >> 3) & 15);
                const bool live = el < ne;
                const float rd = live ? inv_s[el] : 0.f;
                uint32_t ws[4], wm[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float a0 = live ? sv[it][2 * i] : 0.f, a1 = live ? sv[it][2 * i + 1] : 0.f;
                    ws[i] = bf2_bits(__floats2bfloat162_rn(a0 * (1.f / SUR_POOL_DIV), a1 * (1.f / SUR_POOL_DIV)));
                    // the mean as the training path forms it: the sum times the reciprocal count
                    wm[i] = bf2_bits(__floats2bfloat162_rn(a0 * rd, a1 * rd));
                }
                *reinterpret_cast<uint4*>(Ps + canon_off(el, ch, SUR_G)) = make_uint4(ws[0], ws[1], ws[2], ws[3]);
                *reinterpret_cast<uint4*>(Ps + canon_off(el, SUR_H + ch, SUR_G)) = make_uint4(wm[0], wm[1], wm[2], wm[3]);
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        alive = tc_wait(bar_vh, ph_vh, abort_s, a.o.status);
        if (!alive) break;
        ph_vh ^= 1u;
        vh_fly = false;
        alive = tc_wait(bar_vt, ph_vt, abort_s, a.o.status);
        if (!alive) break;
        ph_vt ^= 1u;
        vt_fly = false;
        // ---- event network: G = P V1 (sixteen K-steps) into TMEM columns 0-255
        if (tid == 0) {
            tc_fence_after();
#pragma unroll 1
            for (int ks = 0; ks < SUR_G / 16; ++ks)
                tc_mma(tmem, tc_desc(p_addr + 256u * ks, 128u, 16u * SUR_G), tc_desc(v_addr + 256u * ks, 128u, 16u * SUR_G),
                       idesc_g, ks > 0);
            tc_commit(bar_mma);
            mma_fly = true;
        }
        alive = tc_wait(bar_mma, ph_mma, abort_s, a.o.status);
        if (!alive) break;
        ph_mma ^= 1u;
        mma_fly = false;
        if (staged && tid == 0) {
            // V1^T is consumed: the tile's rows come back for the geometric fallback
            const uint32_t bytes = uint32_t(R0) * uint32_t(sizeof(rta_hillas_t));
            mbar_arrive_expect_tx(bar_rows, bytes);
            bulk_copy(sm + U_FBROWS, f.h + row_first, bytes, bar_rows, l2_policy_evict_first());
            rows_fly = true;
        }
        // ---- output layer on the CUDA cores: this thread's event row, its 64 columns of
        // G = BF16(ReLU(acc + c1)) times V2 (exact BF16 products, summed in FP32 in column order);
        // the four slices' partial sums go to shared memory (over the consumed P operand)
        if (32 * q < ne) {            // a warp whose 32 rows lie past the tile's events skips it
            float y0 = 0.f, y1 = 0.f, y2 = 0.f, y3 = 0.f;
            const float4* v2 = reinterpret_cast<const float4*>(V2f);
#pragma unroll 1
            for (int cb = 0; cb < SUR_G / NSLICE; cb += 32) {
                const int c0 = g_off + cb;
                uint32_t rr[32];
                tc_ld32(tmem + t_lane + uint32_t(c0), rr);
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const float g = __bfloat162float(__float2bfloat16_rn(fmaxf(__uint_as_float(rr[k]) + c1s[c0 + k], 0.f)));
                    const float4 v = v2[c0 + k];
                    y0 = __fmaf_rn(g, v.x, y0);
                    y1 = __fmaf_rn(g, v.y, y1);
                    y2 = __fmaf_rn(g, v.z, y2);
                    y3 = __fmaf_rn(g, v.w, y3);
                }
            }
            reinterpret_cast<float4*>(outp)[slice * TM + row] = make_float4(y0, y1, y2, y3);
        }
        tc_fence_before();
        __syncthreads();
        if (slice == 0 && row < ne) {
            float yo[4];
            {
                const float4* op = reinterpret_cast<const float4*>(outp);
                float4 s = op[row];
#pragma unroll
                for (int k = 1; k < NSLICE; ++k) {
                    const float4 u = op[k * TM + row];
                    s.x += u.x;
                    s.y += u.y;
                    s.z += u.z;
                    s.w += u.w;
                }
                yo[0] = s.x + c2s[0];
                yo[1] = s.y + c2s[1];
                yo[2] = s.z + c2s[2];
                yo[3] = s.w + c2s[3];
            }
            const int64_t e = e0 + row;
            const float2 b = base_s[row];
            const int nu = nu_s[row];
            rta_event_t r = {};
            r.log_energy = yo[0];
            r.dir_x = b.x + yo[1];
            r.dir_y = b.y + yo[2];
            r.gammaness = 1.f / (1.f + expf(-yo[3]));
            r.n_used = nu;
            r.base_x = b.x;
            r.base_y = b.y;
            if (nu < 2) {
                r.flags |= RTA_EF_NO_DIRECTION;        // the geometric method is undefined as well
            } else if (sqrtf(yo[1] * yo[1] + yo[2] * yo[2]) > a.o.fallback_deg) {
                r.flags |= RTA_EF_FALLBACK;
                if (cnt_s[row] > STEREO_WARP_M) fbb_s[atomicAdd(fbb_n, 1)] = row;   // for the CTA-wide pass
                else fb_s[atomicAdd(fb_n, 1)] = row;
            }
            a.o.out[e] = r;
        }
        __syncthreads();
        if (staged) {
            alive = tc_wait(bar_rows, ph_rows, abort_s, a.o.status);
            if (!alive) break;
            ph_rows ^= 1u;
            rows_fly = false;
        }
        const rta_hillas_t* fr_s = reinterpret_cast<const rta_hillas_t*>(sm + U_FBROWS);
        auto frow = [&](int64_t img) -> const rta_hillas_t& { return staged ? fr_s[img - row_first] : f.h[img]; };
        // the telescope of an image and the positions: the shared-memory copies
        auto ftel = [&](int64_t img) { return staged ? tel_s[img - row_first] : f.img_tel[img]; };
        // ---- geometric fallback with the stereo kernel's grouping: up to STEREO_SMALL_M
        // images eight lanes, up to STEREO_WARP_M a warp (one event per warp at a time),
        // larger events ST_NTC threads (warps 0-7, one event after another) while the
        // other warps take the smaller ones
        {
            const int nsmall = *fb_n, nbig = *fbb_n;
            if (nbig > 0 && warp < ST_NTC / 32) {
                StereoImg* imc = reinterpret_cast<StereoImg*>(sm);
                for (int j = 0; j < nbig; ++j) {
                    const int el = fbb_s[j];
                    const int i0 = lo_s[el], m = min(cnt_s[el], RTA_STEREO_MAX_M);
                    int nvalid = 0;
                    if (tid < m)
                        nvalid = stereo_stage(frow(int64_t(i0) + tid), ftel(int64_t(i0) + tid), n_tel, txy_s, a.o.status, imc + tid);
                    stereo_bar<ST_NTC>();
                    CSum acc[5];
                    const int npair = pair_sums<ST_NTC>(imc, m, tid, acc);
                    const rta_stereo_t sr = cta_result<ST_NTC>(acc, npair, nvalid, red_s, redi_s);
                    if (tid == 0) {
                        rta_event_t* o = a.o.out + e0 + el;
                        if (!(sr.flags & RTA_SF_INVALID)) {
                            o->dir_x = sr.dir_x;
                            o->dir_y = sr.dir_y;
                        } else {
                            o->flags |= RTA_EF_NO_DIRECTION;
                        }
                    }
                }
            } else {
                const int w0 = nbig > 0 ? ST_NTC / 32 : 0;
                StereoImg* im = reinterpret_cast<StereoImg*>(sm) + warp * RTA_STEREO_MAX_M;
                for (int j = warp - w0; j < nsmall; j += NW - w0) {
                    const int el = fb_s[j];
                    const int i0 = lo_s[el], m = min(cnt_s[el], RTA_STEREO_MAX_M);
                    int nvalid = 0;
                    for (int k = lane; k < m; k += 32)
                        nvalid += stereo_stage(frow(int64_t(i0) + k), ftel(int64_t(i0) + k), n_tel, txy_s, a.o.status, im + k);
                    __syncwarp();
                    rta_stereo_t sr;
                    if (m <= STEREO_SMALL_M) {
                        // lanes 0-7 hold the event (eight-lane group 0); the other groups are empty
                        CSum acc[5];
                        const int npair = pair_sums<8>(im, lane < 8 ? m : 0, lane & 7, acc);
                        sr = group_result<8>(acc, npair, nvalid);
                    } else {
                        CSum acc[5];
                        const int npair = pair_sums<32>(im, m, lane, acc);
                        sr = group_result<32>(acc, npair, nvalid);
                    }
                    if (lane == 0) {
                        rta_event_t* o = a.o.out + e0 + el;
                        if (!(sr.flags & RTA_SF_INVALID)) {
                            o->dir_x = sr.dir_x;
                            o->dir_y = sr.dir_y;
                        } else {
                            o->flags |= RTA_EF_NO_DIRECTION;
                        }
                    }
                    __syncwarp();
                }
            }
        }
        fence_proxy_async_smem();      // the staged images precede the next tile's bulk copies into U
        __syncthreads();
        first_tile = false;
    }
    // ---- release the tensor memory; MMAs and copies still in flight (after an
    // abort) get one more bounded wait each, so none lands after the CTA is gone
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        volatile int none = 0;
        if (mma_fly) mbar_wait(bar_mma, ph_mma, &none);
        if (w_fly) mbar_wait(bar_w, ph_w, &none);
        if (rows_fly) mbar_wait(bar_rows, ph_rows, &none);
        if (vt_fly) mbar_wait(bar_vt, ph_vt, &none);
        if (vh_fly) mbar_wait(bar_vh, ph_vh, &none);
    }
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, TMEM_COLS);
}

// BF16 twin -> transposed canonical K-major layout of the inference kernel's
// tensor-core layers, and the padded output layer of the training path.
__global__ void k_pack_tc(const __nv_bfloat16* __restrict__ pb, __nv_bfloat16* __restrict__ pk) {
    const int64_t n1 = SUR_H * SUR_XPAD, n2 = SUR_H * SUR_H, n3 = SUR_G * SUR_G, n4 = SUR_G * 16;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n1 + n2 + n3 + n4;
         i += int64_t(gridDim.x) * blockDim.x) {
        if (i < n1) {                                 // W1 [16 k][128 n] -> [128 n][16 k]
            const int64_t k = i / SUR_H, n = i % SUR_H;
            pk[PK_W1T + canon_off(n, k, SUR_XPAD)] = pb[OFF_W1 + i];
        } else if (i < n1 + n2) {                     // W2 [128 k][128 n]
            const int64_t j = i - n1, k = j / SUR_H, n = j % SUR_H;
            pk[PK_W2T + canon_off(n, k, SUR_H)] = pb[OFF_W2 + j];
        } else if (i < n1 + n2 + n3) {                // V1 [256 k][256 n]
            const int64_t j = i - n1 - n2, k = j / SUR_G, n = j % SUR_G;
            pk[PK_V1T + canon_off(n, k, SUR_G)] = pb[OFF_V1 + j];
        } else {                                      // V2 [256 k][4 n] -> [256 k][16 n], zero columns 4..15
            const int64_t j = i - n1 - n2 - n3, k = j / 16, n = j % 16;
            pk[PK_V2P + j] = n < 4 ? pb[OFF_V2 + k * 4 + n] : __float2bfloat16(0.f);
        }
    }
}

cudaError_t launch_pack_tc(const __nv_bfloat16* pb, __nv_bfloat16* pk, cudaStream_t s) {
    k_pack_tc<<<64, 256, 0, s>>>(pb, pk);
    return cudaGetLastError();
}

cudaError_t launch_infer(const InferArgs& a, int n_sm, cudaStream_t s) {
    if (a.f.n_evt <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_deepsets_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, int(S_TOTAL));
    if (e != cudaSuccess) return e;
    // one CTA per SM, with at least 16 events each on average
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(n_sm, a.f.n_evt / 16));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = S_TOTAL;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_deepsets_infer, a);
}

}  // namespace rta
