// Inference of the deep-sets surrogate (energy, direction offset and
// gamma/hadron score next to the geometric direction, Sec. 4.1) in ONE
// persistent kernel on the fifth-generation tensor cores: a CTA of 512 threads
// per SM takes an equal share of the bundle's image rows (a range of whole
// events) and carries it from the Hillas rows to the event rows, geometric
// fallback included, in tiles of at most 128 events:
//
//   1. the tile's Hillas rows arrive by one bulk copy; per event (a pair of
//      lanes) the used images and the two-image baseline;
//   2. the features of up to 512 rows at once, then per 128 image rows the
//      per-telescope network 16 -> 128 -> 128 (ReLU; BF16 activations re-staged
//      as the next layer's operand) and the sum over each event's used images
//      (image order, channel by channel);
//   3. the pooled vectors [sum / 40, mean] as the A operand of the event
//      network 256 -> 256 (ReLU), whose BF16-rounded activations are the A
//      operand of the 256 -> 4 output layer (N padded to 16);
//   4. the events whose learned offset exceeds the fallback bound get the
//      stereo intersection of their images, computed with the stereo kernel's
//      own pieces and grouping (rta_stereo_dev.cuh), so their direction equals
//      rta_stereo's bit for bit.
//
// tcgen05 usage: operands in shared memory as canonical K-major core matrices
// (rta_tc.cuh), FP32 accumulators in tensor memory (256 columns: the two
// per-telescope layers, later the event network and the output layer), one
// thread issuing the MMAs and committing them to an mbarrier that the CTA waits
// on with a time limit; four warps share each TMEM lane quarter, each taking a
// slice of the columns. Weights arrive by bulk copies; the event network's
// 128 KB V1^T shares its shared memory with the per-telescope stage (its tail,
// over the staged rows, follows the last feature pass; its head the last
// pooling).
//
// The kernel is launched with programmatic dependent launch: everything before
// griddepcontrol.wait (tensor-memory allocation, barriers, the registered
// telescope tables) overlaps the end of the kernel before it on the stream;
// nothing that earlier stream work may write is read before the wait.
//
// The features and the per-event reductions are the training path's own
// expressions (rta_mlp_dev.cuh), so baselines and used counts equal those of
// k_features bit for bit (the same lanes per event); the layers sum their exact
// BF16 products in FP32 in the tensor core's order, so the outputs agree with
// the training-path forward to accumulation-order effects.
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
constexpr int LDH = SUR_H + 8;      // row stride of the row-major hidden tile used for pooling

// Shared memory. Region U holds W1^T, W2^T, the feature tile, the hidden tile
// and the tile's Hillas rows during the per-telescope stage, V1^T during the
// event stage (its tail, over the rows, follows the last block's features; its
// head the last pooling), and the fallback's staged images after it.
constexpr int SB = 4 * TM;                                        // rows whose features are formed in one pass
constexpr size_t U_W = 0;                                         // bf16 W1^T [128][16], W2^T [128][128]
constexpr size_t W_BYTES = size_t(PK_V1T - PK_W1T) * 2;          // 36,864
constexpr size_t U_H = U_W + W_BYTES;                             // bf16 H1 canonical [128][128]; H2 row-major [128][LDH]
constexpr size_t U_X = U_H + size_t(TM) * LDH * 2;                // bf16 features of SB rows: 4 canonical [128][16] blocks
constexpr size_t U_ROWS = U_X + size_t(SB) * SUR_XPAD * 2;        // the tile's Hillas rows (64 bytes each)
constexpr size_t V1_BYTES = size_t(SUR_G) * SUR_G * 2;            // 131,072
constexpr size_t U_SIZE = V1_BYTES;
constexpr int MAX_STAGED_ROWS = int((U_SIZE - U_ROWS) / sizeof(rta_hillas_t));   // 672
constexpr int PSTRIDE = SUR_H + 4;                                // pooling-sum row stride (floats): conflict-free reads
constexpr size_t S_P = U_SIZE;                                    // f32 pooling sums [128][PSTRIDE], then bf16 P [128][256]
constexpr size_t S_P_BYTES = size_t(TM) * PSTRIDE * 4;
constexpr size_t S_TCAM = S_P + S_P_BYTES;                        // int [1024] camera of each telescope
constexpr size_t S_TXY = S_TCAM + size_t(RTA_MAX_TEL) * 4;        // float2 [1024] telescope positions
constexpr size_t S_CODE = S_TXY + size_t(RTA_MAX_TEL) * 8;        // f32 [16] camera codes
constexpr size_t S_B1 = S_CODE + size_t(RTA_MAX_CAMS) * 4;        // f32 [128]
constexpr size_t S_B2 = S_B1 + SUR_H * 4;                         // f32 [128]
constexpr size_t S_C1 = S_B2 + SUR_H * 4;                         // f32 [256]
constexpr int NHEAD = 16;           // the output layer's MMA N: its 4 outputs and 12 zero columns
constexpr size_t S_V2 = S_C1 + SUR_G * 4;                         // bf16 V2^T canonical [16][256] (rows 4.. zero)
constexpr size_t S_ROWB = S_V2 + size_t(NHEAD) * SUR_G * 2;       // int64 [129] first row of each event
constexpr size_t S_BASE = S_ROWB + size_t(TM + 1) * 8;            // float2 [128]
constexpr size_t S_EOFF = S_BASE + size_t(TM) * 8;                // int [129 + pad] the tile's event offsets
constexpr size_t S_LO = S_EOFF + size_t(TM + 4) * 4;              // int [128] first image
constexpr size_t S_CNT = S_LO + size_t(TM) * 4;                   // int [128] images (0 if malformed)
constexpr size_t S_NU = S_CNT + size_t(TM) * 4;                   // int [128] used images (-1 if malformed)
constexpr size_t S_INV = S_NU + size_t(TM) * 4;                   // f32 [128] 1 / max(1, used images)
constexpr size_t S_FB = S_INV + size_t(TM) * 4;                   // int [128] fallback list; [128] its count
constexpr size_t S_FBB = S_FB + size_t(TM + 4) * 4;               // int [128] fallback events for the CTA; [128] count
constexpr size_t S_RED = S_FBB + size_t(TM + 4) * 4;              // DW [8][5], int [8][2]: CTA-wide stereo sums
constexpr size_t S_TEL = S_RED + size_t(ST_NTC / 32) * (5 * sizeof(DW) + 2 * 4);    // int [672] staged rows' telescopes
constexpr size_t S_USED = S_TEL + size_t(MAX_STAGED_ROWS) * 4;    // u8 [SB]
constexpr size_t S_BAR = S_USED + SB;                             // 6 mbarriers, TMEM address, abort flag
constexpr size_t S_TOTAL = S_BAR + 64;
static_assert(U_X % 16 == 0 && U_H % 16 == 0 && U_ROWS % 16 == 0 && MAX_STAGED_ROWS >= SB, "U layout");
static_assert(S_P % 16 == 0 && S_P_BYTES >= size_t(TM) * SUR_G * 2, "pooling region holds the P operand");
static_assert(S_TXY % 8 == 0 && S_ROWB % 8 == 0 && S_BASE % 8 == 0 && S_RED % 8 == 0 && S_BAR % 8 == 0,
              "aligned tables");
static_assert(size_t(NW) * RTA_STEREO_MAX_M * sizeof(StereoImg) <= U_ROWS, "fallback staging in U");
static_assert(S_TOTAL <= 227 * 1024, "one CTA per SM");

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

// ------------------------------------------------------------------ the kernel
__global__ void __launch_bounds__(NT, 1) k_deepsets_infer(const InferArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __nv_bfloat16* Ws = reinterpret_cast<__nv_bfloat16*>(sm + U_W);
    __nv_bfloat16* Xs = reinterpret_cast<__nv_bfloat16*>(sm + U_X);
    __nv_bfloat16* Hs = reinterpret_cast<__nv_bfloat16*>(sm + U_H);
    rta_hillas_t* rows_s = reinterpret_cast<rta_hillas_t*>(sm + U_ROWS);
    float* Pacc = reinterpret_cast<float*>(sm + S_P);
    __nv_bfloat16* Ps = reinterpret_cast<__nv_bfloat16*>(sm + S_P);
    int* tcam_s = reinterpret_cast<int*>(sm + S_TCAM);
    float2* txy_s = reinterpret_cast<float2*>(sm + S_TXY);
    float* code_s = reinterpret_cast<float*>(sm + S_CODE);
    float* b1s = reinterpret_cast<float*>(sm + S_B1);
    float* b2s = reinterpret_cast<float*>(sm + S_B2);
    float* c1s = reinterpret_cast<float*>(sm + S_C1);
    __nv_bfloat16* V2s = reinterpret_cast<__nv_bfloat16*>(sm + S_V2);
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
    uint64_t* bar_mma = reinterpret_cast<uint64_t*>(sm + S_BAR);    // MMA completion
    uint64_t* bar_w = bar_mma + 1;                                    // W1^T, W2^T copy
    uint64_t* bar_rows = bar_mma + 2;                                 // the tile's Hillas rows
    uint64_t* bar_vt = bar_mma + 3;                                   // V1^T tail copy
    uint64_t* bar_vh = bar_mma + 4;                                   // V1^T head copy
    uint32_t* tmem_s = reinterpret_cast<uint32_t*>(sm + S_BAR + 48);
    volatile int* abort_s = reinterpret_cast<volatile int*>(sm + S_BAR + 52);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const FeatArgs& f = a.f;
    const int64_t n_evt = f.n_evt, n_img = f.n_img;
    const int n_tel = min(f.n_tel, RTA_MAX_TEL);

    // ---- set-up that reads nothing earlier stream work may write
    if (warp == 0) {
        tc_alloc(tmem_s, 256);
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
    {
        // telescope tables (registration copies, complete before any launch)
        int tc[RTA_MAX_TEL / NT];
        float2 txy[RTA_MAX_TEL / NT];
#pragma unroll
        for (int k = 0; k < RTA_MAX_TEL / NT; ++k) {
            const int i = tid + k * NT;
            tc[k] = i < n_tel ? f.tel_cam[i] : 0;
            txy[k] = i < n_tel ? f.tel_xy[i] : make_float2(0.f, 0.f);
        }
        const float code = tid < RTA_MAX_CAMS ? f.cam_code[tid] : 0.f;
#pragma unroll
        for (int k = 0; k < RTA_MAX_TEL / NT; ++k) {
            const int i = tid + k * NT;
            if (i < n_tel) {
                tcam_s[i] = tc[k];
                txy_s[i] = txy[k];
            }
        }
        if (tid < RTA_MAX_CAMS) code_s[tid] = code;
    }
    // ---- everything below may read what the kernels before this one wrote
    grid_dependency_wait();
    if (tid == 0) {
        mbar_arrive_expect_tx(bar_w, uint32_t(W_BYTES));
        bulk_copy(Ws, a.pk + PK_W1T, uint32_t(W_BYTES), bar_w, l2_policy_evict_last());
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_s;
    const uint32_t idesc_h = tc_idesc_bf16(TM, SUR_H), idesc_g = tc_idesc_bf16(TM, SUR_G),
                   idesc_o = tc_idesc_bf16(TM, NHEAD);
    const uint32_t v2_addr = smem_addr(V2s);
    const uint32_t x_addr = smem_addr(Xs), h_addr = smem_addr(Hs), w1_addr = smem_addr(Ws),
                   w2_addr = smem_addr(Ws + SUR_H * SUR_XPAD), p_addr = smem_addr(Ps), v_addr = smem_addr(sm);
    const int q = warp & 3, row = 32 * q + lane, slice = warp >> 2;
    const int c_half = slice * (SUR_H / NSLICE), g_half = slice * (SUR_G / NSLICE);
    const uint32_t t_lane = uint32_t(32 * q) << 16;
    const int sub = lane % SUR_EVT_LANES, grp = lane / SUR_EVT_LANES;
    const float c2[4] = {a.p[OFF_C2 + 0], a.p[OFF_C2 + 1], a.p[OFF_C2 + 2], a.p[OFF_C2 + 3]};
    uint32_t ph_mma = 0, ph_w = 0, ph_rows = 0, ph_vt = 0, ph_vh = 0;
    bool alive = true;
    // what thread 0 has issued and the CTA has not yet waited for (drained before exit)
    bool mma_fly = false, w_fly = (tid == 0), rows_fly = false, vt_fly = false, vh_fly = false;

    int64_t ev_begin, ev_end;
    event_range(f.evt_off, n_evt, fb_s, ev_begin, ev_end);
    for (int64_t e0 = ev_begin; e0 < ev_end; e0 += TM) {
        const int ne = int(min(int64_t(TM), ev_end - e0));
        if (e0 != ev_begin && tid == 0) {          // the event stage overwrote W1^T / W2^T
            mbar_arrive_expect_tx(bar_w, uint32_t(W_BYTES));
            bulk_copy(Ws, a.pk + PK_W1T, uint32_t(W_BYTES), bar_w, l2_policy_evict_last());
            w_fly = true;
        }
        // ---- the tile's event offsets (and, with the first tile, the biases and the output
        // layer's weights, whose loads overlap); pooling sums start at zero
        const int eo = tid <= ne ? f.evt_off[e0 + tid] : 0;
        if (e0 == ev_begin) {
            const float bb1 = tid < SUR_H ? a.p[OFF_B1 + tid] : 0.f, bb2 = tid < SUR_H ? a.p[OFF_B2 + tid] : 0.f;
            const float c1 = tid < SUR_G ? a.p[OFF_C1 + tid] : 0.f;
            // V2^T as the output layer's B operand: row n < 4 is output n, the rest zero
            __nv_bfloat16 v2[NHEAD * SUR_G / NT];
#pragma unroll
            for (int k = 0; k < NHEAD * SUR_G / NT; ++k) {
                const int i = tid + k * NT, n = i / SUR_G, kk = i % SUR_G;
                v2[k] = n < 4 ? a.pb[OFF_V2 + kk * 4 + n] : __float2bfloat16(0.f);
            }
            if (tid < SUR_H) {
                b1s[tid] = bb1;
                b2s[tid] = bb2;
            }
            if (tid < SUR_G) c1s[tid] = c1;
#pragma unroll
            for (int k = 0; k < NHEAD * SUR_G / NT; ++k) {
                const int i = tid + k * NT;
                V2s[canon_off(i / SUR_G, i % SUR_G, SUR_G)] = v2[k];
            }
            fence_proxy_async_smem();
        }
        if (tid <= ne) eoff_s[tid] = eo;
        for (int i = tid; i < TM * PSTRIDE; i += NT) Pacc[i] = 0.f;
        if (tid == 0) *fb_n = *fbb_n = 0;
        __syncthreads();
        // ---- the tile's Hillas rows in shared memory when its offsets are well formed
        // (ascending, inside [0, n_img]) and they fit; else every row is read from global memory
        const bool ordered = tid >= ne || (eoff_s[tid] <= eoff_s[tid + 1] && eoff_s[tid] >= 0 && eoff_s[tid + 1] <= n_img);
        const bool wellformed = __syncthreads_and(ordered);
        const bool staged = wellformed && a.rows_aligned && eoff_s[ne] - eoff_s[0] <= MAX_STAGED_ROWS &&
                            eoff_s[ne] > eoff_s[0];
        if (wellformed && tid <= ne) rowb[tid] = int64_t(eoff_s[tid]) - eoff_s[0];   // the tile's rows in order
        const int row_first = staged ? eoff_s[0] : 0;
        const rta_hillas_t* hrows = staged ? rows_s : f.h;
        if (staged) {
            if (tid == 0) {
                const uint32_t bytes = uint32_t(eoff_s[ne] - eoff_s[0]) * uint32_t(sizeof(rta_hillas_t));
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar_rows, bytes);
                bulk_copy(rows_s, f.h + row_first, bytes, bar_rows, l2_policy_evict_first());
                rows_fly = true;
            }
            for (int k = tid; k < eoff_s[ne] - row_first; k += NT) tel_s[k] = f.img_tel[row_first + k];
            alive = tc_wait(bar_rows, ph_rows, abort_s, a.o.status);
            if (!alive) break;
            ph_rows ^= 1u;
            rows_fly = false;
        } else if (tid == 0) {                       // the rows region is free: V1^T's tail now
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar_vt, uint32_t(U_SIZE - U_ROWS));
            bulk_copy(sm + U_ROWS, a.pk + PK_V1T + U_ROWS / 2, uint32_t(U_SIZE - U_ROWS), bar_vt,
                      l2_policy_evict_last());
            vt_fly = true;
        }
        bool tail_issued = !staged;
        // ---- per-event prologue, SUR_EVT_LANES lanes per event (as k_features), 128 events per pass
        for (int p0 = 0; p0 < ne; p0 += NT / SUR_EVT_LANES) {
            const int el = p0 + (32 / SUR_EVT_LANES) * warp + grp;
            int i0 = 0, n = 0;
            bool ok = false;
            if (el < ne) {
                i0 = eoff_s[el];
                const int i1 = eoff_s[el + 1];
                ok = !(i0 < 0 || i1 < i0 || i1 > n_img);
                n = ok ? i1 - i0 : 0;
            }
            float bx, by;
            int cnt;
            sur_event_baseline(hrows, i0 - row_first, n, sub, nullptr, bx, by, cnt);
            if (sub == 0 && el < ne) {
                base_s[el] = make_float2(bx, by);
                lo_s[el] = i0;
                cnt_s[el] = n;
                nu_s[el] = ok ? cnt : -1;
                inv_s[el] = __frcp_rn(fmaxf(1.f, float(ok ? cnt : 0)));   // = 1.f / n (both round to nearest)
            }
        }
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
        __syncthreads();
        const int64_t R = rowb[ne];
        bool w_pending = true;                          // this tile's W1^T, W2^T not yet waited for

        for (int64_t rb = 0; rb < R; rb += TM) {
            const int xb = int((rb / TM) % (SB / TM));      // this block's feature tile in the pass
            if (xb == 0) {
                // ---- features of rows rb .. rb + SB - 1 (four blocks), all threads; rows past R are zero
#pragma unroll 1
                for (int q = tid; q < SB; q += NT) {
                    const int64_t r = rb + q;
                    __nv_bfloat162 x[SUR_XPAD / 2];
                    bool used = false;
                    if (r < R) {
                        int lo = 0, hi = ne - 1;              // last event whose first row is <= r
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (rowb[mid] <= r) lo = mid;
                            else hi = mid - 1;
                        }
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
                    __nv_bfloat16* xt = Xs + (q / TM) * (TM * SUR_XPAD);
                    *reinterpret_cast<uint4*>(xt + canon_off(q % TM, 0, SUR_XPAD)) =
                        make_uint4(bf2_bits(x[0]), bf2_bits(x[1]), bf2_bits(x[2]), bf2_bits(x[3]));
                    *reinterpret_cast<uint4*>(xt + canon_off(q % TM, 8, SUR_XPAD)) =
                        make_uint4(bf2_bits(x[4]), bf2_bits(x[5]), bf2_bits(x[6]), bf2_bits(x[7]));
                    used_s[q] = used;
                }
                fence_proxy_async_smem();
                __syncthreads();
                if (!tail_issued && rb + SB >= R && tid == 0) {
                    // the staged rows are read for the last time: V1^T's tail may overwrite them
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(bar_vt, uint32_t(U_SIZE - U_ROWS));
                    bulk_copy(sm + U_ROWS, a.pk + PK_V1T + U_ROWS / 2, uint32_t(U_SIZE - U_ROWS), bar_vt,
                              l2_policy_evict_last());
                    vt_fly = true;
                }
                if (rb + SB >= R) tail_issued = true;
            }
            if (w_pending) {                            // W1^T, W2^T of this tile
                alive = tc_wait(bar_w, ph_w, abort_s, a.o.status);
                if (!alive) break;
                ph_w ^= 1u;
                w_pending = w_fly = false;
            }
            // ---- layer 1: D1 = X W1 (one K-step)
            if (tid == 0) {
                tc_fence_after();
                tc_mma(tmem, tc_desc(x_addr + uint32_t(xb * TM * SUR_XPAD * 2), 128u, 16u * SUR_XPAD),
                       tc_desc(w1_addr, 128u, 16u * SUR_XPAD), idesc_h, false);
                tc_commit(bar_mma);
                mma_fly = true;
            }
            alive = tc_wait(bar_mma, ph_mma, abort_s, a.o.status);
            if (!alive) break;
            ph_mma ^= 1u;
            mma_fly = false;
            // ReLU(D1 + b1) in BF16 -> canonical operand of layer 2 (this thread: one row, 64 columns)
#pragma unroll 1
            for (int cb = 0; cb < SUR_H / NSLICE; cb += 32) {
                const int c0 = c_half + cb;
                uint32_t v[32];
                tc_ld32(tmem + t_lane + uint32_t(c0), v);
#pragma unroll
                for (int q8 = 0; q8 < 4; ++q8) {
                    uint32_t w[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int k = 8 * q8 + 2 * i;
                        w[i] = bf2_bits(__floats2bfloat162_rn(fmaxf(__uint_as_float(v[k]) + b1s[c0 + k], 0.f),
                                                              fmaxf(__uint_as_float(v[k + 1]) + b1s[c0 + k + 1], 0.f)));
                    }
                    *reinterpret_cast<uint4*>(Hs + canon_off(row, c0 + 8 * q8, SUR_H)) = make_uint4(w[0], w[1], w[2], w[3]);
                }
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
                           tc_desc(w2_addr + 256u * ks, 128u, 16u * SUR_H), idesc_h, ks > 0);
                tc_commit(bar_mma);
                mma_fly = true;
            }
            alive = tc_wait(bar_mma, ph_mma, abort_s, a.o.status);
            if (!alive) break;
            ph_mma ^= 1u;
            mma_fly = false;
            // ReLU(D2 + b2) in BF16, +0 rows for unused images -> row-major tile for pooling
            const bool urow = used_s[xb * TM + row];
#pragma unroll 1
            for (int cb = 0; cb < SUR_H / NSLICE; cb += 32) {
                const int c0 = c_half + cb;
                uint32_t v[32];
                tc_ld32(tmem + SUR_H + t_lane + uint32_t(c0), v);
                uint4* hr = reinterpret_cast<uint4*>(Hs + row * LDH + c0);
#pragma unroll
                for (int q8 = 0; q8 < 4; ++q8) {
                    uint32_t w[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int k = 8 * q8 + 2 * i;
                        w[i] = bf2_bits(__floats2bfloat162_rn(
                            urow ? fmaxf(__uint_as_float(v[k]) + b2s[c0 + k], 0.f) : 0.f,
                            urow ? fmaxf(__uint_as_float(v[k + 1]) + b2s[c0 + k + 1], 0.f) : 0.f));
                    }
                    hr[q8] = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
            tc_fence_before();
            __syncthreads();
            // ---- pooling: thread = (channel pair, event group); each channel's sum runs
            // over the event's rows in image order
            {
                constexpr int NG = NT / 64;
                const int cp = tid & 63, g4 = tid >> 6;
                const int64_t rend = min(R, rb + TM);
                int ev = 0, hi = ne - 1;                 // first event with a row in [rb, rend)
                while (ev < hi) {
                    const int mid = (ev + hi) >> 1;
                    if (rowb[mid + 1] <= rb) ev = mid + 1;
                    else hi = mid;
                }
                for (int el = ev + g4; el < ne && rowb[el] < rend; el += NG) {
                    const int64_t lo = max(rowb[el], rb), up = min(rowb[el + 1], rend);
                    if (lo >= up) continue;
                    float2 s2 = reinterpret_cast<const float2*>(Pacc + el * PSTRIDE)[cp];
#pragma unroll 4
                    for (int64_t r = lo; r < up; ++r) {
                        const float2 h2 =
                            __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(Hs + (r - rb) * LDH)[cp]);
                        s2.x += h2.x;
                        s2.y += h2.y;
                    }
                    reinterpret_cast<float2*>(Pacc + el * PSTRIDE)[cp] = s2;
                }
            }
            __syncthreads();
        }
        if (!alive) break;
        if (w_pending) {                                // a tile without image rows: the copy must still land
            alive = tc_wait(bar_w, ph_w, abort_s, a.o.status);
            if (!alive) break;
            ph_w ^= 1u;
            w_fly = false;
        }
        if (!tail_issued && tid == 0) {                 // (staged rows but no block: not reached)
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar_vt, uint32_t(U_SIZE - U_ROWS));
            bulk_copy(sm + U_ROWS, a.pk + PK_V1T + U_ROWS / 2, uint32_t(U_SIZE - U_ROWS), bar_vt,
                      l2_policy_evict_last());
            vt_fly = true;
        }
        // ---- the per-telescope stage is done with region U: the head of V1^T follows it in
        if (tid == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar_vh, uint32_t(U_ROWS));
            bulk_copy(sm, a.pk + PK_V1T, uint32_t(U_ROWS), bar_vh, l2_policy_evict_last());
            vh_fly = true;
        }
        // ---- pooled vectors [sum / 40, sum * RN(1 / max(1, n_used))] in BF16, in place of the sums.
        // Item i of this thread: event 8 (k / 128) + k % 8 and channels 8 ((k / 8) % 16) .. + 7,
        // k = tid + 256 i; every sum is read before any operand is written.
        {
            constexpr int NIT = TM * (SUR_H / 8) / NT;       // items per thread
            float sv[NIT][8];
#pragma unroll
            for (int it = 0; it < NIT; ++it) {
                const int k = tid + NT * it;
                const int el = 8 * (k >> 7) + (k & 7), ch = 8 * ((k >> 3) & 15);
                const float4 u0 = *reinterpret_cast<const float4*>(Pacc + el * PSTRIDE + ch);
                const float4 u1 = *reinterpret_cast<const float4*>(Pacc + el * PSTRIDE + ch + 4);
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
        alive = tc_wait(bar_vt, ph_vt, abort_s, a.o.status);
        if (!alive) break;
        ph_vt ^= 1u;
        vt_fly = false;
        alive = tc_wait(bar_vh, ph_vh, abort_s, a.o.status);
        if (!alive) break;
        ph_vh ^= 1u;
        vh_fly = false;
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
        // ---- output layer on the tensor core: G = BF16(ReLU(acc + c1)) (this thread: one row,
        // its slice of the columns) as the A operand in place of P, then y = G V2 (N = 16,
        // outputs in TMEM columns 0-3, over the event network's consumed accumulators)
#pragma unroll 1
        for (int cb = 0; cb < SUR_G / NSLICE; cb += 32) {
            const int c0 = g_half + cb;
            uint32_t rr[32];
            tc_ld32(tmem + t_lane + uint32_t(c0), rr);
#pragma unroll
            for (int q8 = 0; q8 < 4; ++q8) {
                uint32_t w[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int k = 8 * q8 + 2 * i;
                    w[i] = bf2_bits(__floats2bfloat162_rn(fmaxf(__uint_as_float(rr[k]) + c1s[c0 + k], 0.f),
                                                          fmaxf(__uint_as_float(rr[k + 1]) + c1s[c0 + k + 1], 0.f)));
                }
                *reinterpret_cast<uint4*>(Ps + canon_off(row, c0 + 8 * q8, SUR_G)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll 1
            for (int ks = 0; ks < SUR_G / 16; ++ks)
                tc_mma(tmem, tc_desc(p_addr + 256u * ks, 128u, 16u * SUR_G), tc_desc(v2_addr + 256u * ks, 128u, 16u * SUR_G),
                       idesc_o, ks > 0);
            tc_commit(bar_mma);
            mma_fly = true;
        }
        alive = tc_wait(bar_mma, ph_mma, abort_s, a.o.status);
        if (!alive) break;
        ph_mma ^= 1u;
        mma_fly = false;
        if (slice == 0) {
            uint32_t rr[16];
            tc_ld16(tmem + t_lane, rr);
            if (row < ne) {
                float yo[4];
#pragma unroll
                for (int o = 0; o < 4; ++o) yo[o] = __uint_as_float(rr[o]) + c2[o];
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
        }
        tc_fence_before();
        __syncthreads();
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
                        nvalid = stereo_stage(f.h[i0 + tid], f.img_tel[i0 + tid], n_tel, f.tel_xy, a.o.status, imc + tid);
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
                        nvalid += stereo_stage(f.h[i0 + k], f.img_tel[i0 + k], n_tel, f.tel_xy, a.o.status, im + k);
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
    if (warp == 0) tc_dealloc(tmem, 256);
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
