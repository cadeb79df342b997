// Stereo Hillas intersection (direction and core reconstruction, Sec. 4.1).
//
// Eight lanes per event for events of up to eight images (four such events
// share a warp), the whole warp for larger ones; the kernel then fits one wave
// of warps at the usual bundle sizes. The event's images (at most 64) are
// staged in shared memory; its lanes walk the upper triangle of image pairs
// (i < j) 8 or 32 apart and accumulate the weighted intersections; a shuffle
// tree over those lanes sums the five partial sums. The pair arithmetic and its
// precision are described with the shared pieces in rta_stereo_dev.cuh.
#include "rta_stereo_dev.cuh"

namespace rta {

constexpr int ST_WARPS = 8;
constexpr int ST_NT = ST_WARPS * 32;
constexpr int ST_GL = 8;          // lanes per event for small events
constexpr int ST_EPW = 32 / ST_GL; // output rows per warp tile
static_assert(ST_GL == STEREO_SMALL_M, "small events take one lane per image slot of their group");

// the first lane of every ST_GL-lane group
__host__ __device__ constexpr unsigned group_leaders() {
    unsigned v = 0;
    for (int k = 0; k < 32; k += ST_GL) v |= 1u << k;
    return v;
}

// One image of the bundle staged for the pair loop.
__device__ __forceinline__ int stage_image(const StereoArgs& a, int64_t img, StereoImg* dst) {
    return stereo_stage(a.h[img], a.img_tel[img], a.arr.n_tel, a.arr.tel_xy, a.status, dst);
}

// The CTA takes ST_WARPS warp tiles of ST_EPW consecutive output rows per round.
// Events of at most STEREO_SMALL_M images (most of them) are done side by side,
// ST_GL lanes each; up to STEREO_WARP_M images one after another by the warp;
// larger ones go on the CTA's list and are done one after another by the whole
// CTA at the end of the round. Which of the three an event takes depends on its
// own image count only, so its row does not depend on the events around it (a
// sub-list of events gives the same rows).
__global__ void __launch_bounds__(ST_NT) k_stereo(const StereoArgs a) {
    __shared__ StereoImg sh[ST_WARPS][RTA_STEREO_MAX_M];
    __shared__ int big_e[ST_WARPS * ST_EPW], big_i0[ST_WARPS * ST_EPW], big_m[ST_WARPS * ST_EPW];
    __shared__ int n_big;
    __shared__ DW red[ST_WARPS * 5];
    __shared__ int redi[ST_WARPS * 2];
    static_assert(ST_EPW * STEREO_SMALL_M <= RTA_STEREO_MAX_M && ST_EPW * ST_GL == 32, "small events share the warp");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / ST_GL, sub = lane % ST_GL;
    StereoImg* im = sh[warp];
    // Launched as a programmatic dependent of the image kernel. When the caller declared the
    // event offsets and counts settled (written before the image kernel started), they are
    // read before the dependency wait: the counts and the first round's offsets.
    if (!a.settled) grid_dependency_wait();
    // a graph captured at capacity reads the bundle's counts at run time
    const int64_t n_evt = a.n_evt_dev ? min(*a.n_evt_dev, a.n_evt) : a.n_evt;
    const int64_t n_img = a.n_img_dev ? min(*a.n_img_dev, a.n_img) : a.n_img;
    const int64_t n_tiles = (n_evt + ST_EPW - 1) / ST_EPW;
    int pre0 = 0, pre1 = 0;                                // the first round's offsets of this group
    {
        const int64_t e = (int64_t(blockIdx.x) * ST_WARPS + warp) * ST_EPW + g;
        if (e < n_evt) {
            pre0 = a.evt_off[e];
            pre1 = a.evt_off[e + 1];
        }
    }
    if (a.settled) grid_dependency_wait();
    for (int64_t r0 = int64_t(blockIdx.x) * ST_WARPS; r0 < n_tiles; r0 += int64_t(gridDim.x) * ST_WARPS) {
        __syncthreads();                                   // the previous round's list is read
        if (threadIdx.x == 0) n_big = 0;
        __syncthreads();
        const int64_t wt = r0 + warp;
        if (wt < n_tiles) {
            const int64_t e = wt * ST_EPW + g;                 // this group's output row
            int i0 = 0, m = 0;
            bool valid = false;
            if (e < n_evt) {
                const bool first = r0 == int64_t(blockIdx.x) * ST_WARPS;
                const int b0 = first ? pre0 : a.evt_off[e], b1 = first ? pre1 : a.evt_off[e + 1];
                if (b0 < 0 || b1 < b0 || b1 > n_img) {         // malformed CSR: flag, never index
                    if (sub == 0) {
                        atomicOr(a.status, RTA_DEV_BAD_IMAGE);
                        rta_stereo_t r = {};
                        r.flags = RTA_SF_INVALID;
                        a.out[e] = r;
                    }
                } else {
                    valid = true;
                    i0 = b0;
                    m = min(b1 - b0, RTA_STEREO_MAX_M);
                }
            }
            // small events: the group's lanes, slots STEREO_SMALL_M * g ...
            {
                const bool small = valid && m <= STEREO_SMALL_M;
                const int ms = small ? m : 0;
                StereoImg* gi = im + STEREO_SMALL_M * g;
                int nvalid = 0;
                for (int k = sub; k < ms; k += ST_GL) nvalid += stage_image(a, int64_t(i0) + k, gi + k);
                __syncwarp();
                CSum acc[5];
                const int npair = pair_sums<ST_GL>(gi, ms, sub, acc);
                const rta_stereo_t r = group_result<ST_GL>(acc, npair, nvalid);
                if (small && sub == 0) a.out[e] = r;
                __syncwarp();
            }
            // events of up to STEREO_WARP_M images: one at a time, the whole warp
            unsigned mid = __ballot_sync(0xffffffffu, valid && m > STEREO_SMALL_M && m <= STEREO_WARP_M) &
                           group_leaders();
            while (mid) {
                const int src = __ffs(mid) - 1;
                mid &= mid - 1;
                const int bi0 = __shfl_sync(0xffffffffu, i0, src), bm = __shfl_sync(0xffffffffu, m, src);
                int nvalid = 0;
                for (int k = lane; k < bm; k += 32) nvalid += stage_image(a, int64_t(bi0) + k, im + k);
                __syncwarp();
                CSum acc[5];
                const int npair = pair_sums<32>(im, bm, lane, acc);
                const rta_stereo_t r = group_result<32>(acc, npair, nvalid);
                if (lane == 0) a.out[wt * ST_EPW + src / ST_GL] = r;
                __syncwarp();
            }
            // larger events: on the CTA's list
            if (valid && m > STEREO_WARP_M && sub == 0) {
                const int slot = atomicAdd(&n_big, 1);
                big_e[slot] = int(e - r0 * ST_EPW);
                big_i0[slot] = i0;
                big_m[slot] = m;
            }
        }
        __syncthreads();
        // the list, one event at a time, the whole CTA (warp 0's image slots)
        const int nb = n_big;
        for (int b = 0; b < nb; ++b) {
            const int bm = big_m[b];
            int nvalid = 0;
            if (threadIdx.x < bm) nvalid = stage_image(a, int64_t(big_i0[b]) + threadIdx.x, sh[0] + threadIdx.x);
            stereo_bar<ST_NT>();
            CSum acc[5];
            const int npair = pair_sums<ST_NT>(sh[0], bm, threadIdx.x, acc);
            const rta_stereo_t r = cta_result<ST_NT>(acc, npair, nvalid, red, redi);
            if (threadIdx.x == 0) a.out[r0 * ST_EPW + big_e[b]] = r;
        }
    }
}

// Failure-detection self-test: one thread waits on an mbarrier that nothing
// will ever complete, through the same bounded wait the image kernel uses. The
// wait gives up after timeout_ns, the status word gets RTA_DEV_TIMEOUT and the
// kernel returns normally, leaving the context usable.
__global__ void k_wait_selftest(unsigned int* status, uint64_t timeout_ns, unsigned long long* waited_ns) {
    __shared__ uint64_t bar;
    __shared__ int abort;
    if (threadIdx.x != 0) return;
    abort = 0;
    mbar_init(&bar, 1);
    fence_mbar_init();
    const uint64_t t0 = global_ns();
    const bool ok = mbar_wait_ns(&bar, 0, &abort, timeout_ns);
    if (!ok) atomicOr(status, RTA_DEV_TIMEOUT);
    if (waited_ns) *waited_ns = global_ns() - t0;
    // leave no arrival pending: complete the phase ourselves before exiting
    mbar_arrive(&bar);
}

cudaError_t launch_wait_selftest(unsigned int* status, uint64_t timeout_ns, unsigned long long* waited_ns,
                                 cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(status, timeout_ns, waited_ns);
    return cudaGetLastError();
}

cudaError_t launch_stereo(const StereoArgs& a, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(ST_WARPS * 32);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_stereo, a);
}

int stereo_events_per_block() { return ST_WARPS * ST_EPW; }

}  // namespace rta
