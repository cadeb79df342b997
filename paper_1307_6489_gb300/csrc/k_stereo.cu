// Stereo Hillas intersection (direction and core reconstruction, Sec. 4.1).
//
// Eight lanes per event for events of up to eight images (four such events
// share a warp), the whole warp for larger ones; the kernel then fits one wave
// of warps at the usual bundle sizes. The event's images (at most 64) are
// staged in shared memory; its lanes walk the upper triangle of image pairs
// (i < j) 8 or 32 apart and accumulate the weighted intersections; a shuffle
// tree over those lanes sums the five partial sums. The weighted intersection is accumulated without dividing by
// s = sin(psi_j - psi_i):
//   w * p = F * (|s| * c_i + sign(s) * cross(c_j - c_i, u_j) * u_i),
// with F = s_i s_j / (s_i + s_j) (1 - W_i/L_i)(1 - W_j/L_j), the same quantity as
// |s| F * (c_i + u_i cross / s) but well conditioned for nearly parallel axes.
// Precision: when every pair of an event is nearly parallel the result is a
// ratio of small sums, so s must be accurate relative to itself. The angle
// difference is carried exactly as an unevaluated FP32 pair (TwoSum), reduced
// to (-pi/2, pi/2] against a two-word pi (sin(d - pi) = -sin d), and rounded
// once before sinf -- never formed as a difference of products of rounded
// cosines. Each lane's sums are compensated (Neumaier), the lanes are combined
// as FP32 double-word sums and the final ratios are double-word quotients, so
// no step needs FP64 (whose rate on this part is a small fraction of FP32's).
#include "rta_launch.cuh"

namespace rta {

constexpr int ST_WARPS = 8;
constexpr int ST_GL = 8;          // lanes per event for small events
constexpr int ST_EPW = 32 / ST_GL; // output rows per warp tile
constexpr int ST_SMALL_M = 8;     // image count up to which an event takes ST_GL lanes

// the first lane of every ST_GL-lane group
__host__ __device__ constexpr unsigned group_leaders() {
    unsigned v = 0;
    for (int k = 0; k < 32; k += ST_GL) v |= 1u << k;
    return v;
}

// 48 bytes: three 16-byte shared-memory loads per image
struct __align__(16) StereoImg {
    float x, y, c, s;          // centroid, cos psi, sin psi
    float psi, f, tx, ty;      // f = 1 - W/L; telescope position
    float size;
    int used;
    float pad0, pad1;
};

// Compensated running sum (Neumaier's variant of Kahan summation).
struct CSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float t = s + v;
        c += (fabsf(s) >= fabsf(v)) ? (s - t) + v : (v - t) + s;
        s = t;
    }
};

// Unevaluated sum hi + lo of two FP32 words.
struct DW {
    float hi, lo;
};

// a + b for |a| >= |b| (or a == 0): exact.
__device__ __forceinline__ DW fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}

// a + b with the rounding error (Knuth's TwoSum): exact.
__device__ __forceinline__ DW two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ DW dw_add(DW a, DW b) {
    const DW s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ DW dw_warp_sum(DW v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const DW w = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = dw_add(v, w);
    }
    return v;
}

// (a.hi + a.lo) / (b.hi + b.lo) rounded to FP32 (one correction step).
__device__ __forceinline__ float dw_div(DW a, DW b) {
    const float q = a.hi / b.hi;
    const float p = q * b.hi;
    const float pe = fmaf(q, b.hi, -p);                 // q * b.hi = p + pe exactly
    const float r = (((a.hi - p) - pe) + a.lo) - q * b.lo;
    return q + r / b.hi;
}

// One image staged for the pair loop: its direction cosines, 1 - W/L (0 when
// not used for stereo) and telescope position. Returns whether it is used.
__device__ __forceinline__ int stage_image(const StereoArgs& a, int64_t img, StereoImg* dst) {
    const rta_hillas_t hh = a.h[img];
    const int tel = a.img_tel[img];
    const bool tel_ok = tel >= 0 && tel < a.arr.n_tel;
    const bool used = tel_ok && hh.n_pix >= 3 && !(hh.flags & (RTA_HF_EMPTY | RTA_HF_BAD_INPUT));
    if (!tel_ok) atomicOr(a.status, RTA_DEV_BAD_IMAGE);
    StereoImg v;
    float sp, cp;
    sincosf(hh.psi, &sp, &cp);
    v.x = hh.x;
    v.y = hh.y;
    v.c = cp;
    v.s = sp;
    v.psi = hh.psi;
    v.f = used ? 1.f - __fdiv_rn(hh.width, hh.length) : 0.f;
    const float2 t = tel_ok ? a.arr.tel_xy[tel] : make_float2(0.f, 0.f);
    v.tx = t.x;
    v.ty = t.y;
    v.size = hh.size;
    v.used = used;
    v.pad0 = v.pad1 = 0.f;
    *dst = v;
    return used;
}

// Pair sums of one event of m staged images, shared by G lanes (this one is
// lane `sub`): pair p of the row-major upper triangle (i, j), i < j, goes to
// lane p mod G, walked incrementally G pairs at a time.
template <int G>
__device__ __forceinline__ int pair_sums(const StereoImg* im, int m, int sub, CSum (&acc)[5]) {
    const float kPiHi = 3.14159274101257324f;          // RN(pi), above pi
    const float kPiLo = -8.74227765734758577e-8f;      // pi - kPiHi
    const float kHalfPi = 1.57079637050628662f;
    int npair = 0;
    const int T = m * (m - 1) / 2;
    int i = 0, j = 1 + sub;
    while (j >= m && i < m - 1) { ++i; j = j - m + i + 1; }
    for (int p = sub; p < T; p += G) {
        const StereoImg A = im[i], B = im[j];
        j += G;
        while (j >= m && i < m - 1) { ++i; j = j - m + i + 1; }
        if (!A.used || !B.used) continue;
        DW d = two_sum(B.psi, -A.psi);                  // psi_j - psi_i, exactly
        float sgn = 1.f;
        if (d.hi > kHalfPi) {
            d = {d.hi - kPiHi, d.lo - kPiLo};          // d.hi - kPiHi is exact (Sterbenz)
            sgn = -1.f;
        } else if (d.hi <= -kHalfPi) {
            d = {d.hi + kPiHi, d.lo + kPiLo};
            sgn = -1.f;
        }
        const float s = sgn * sinf(d.hi + d.lo);          // sin(psi_j - psi_i), relatively accurate
        if (fabsf(s) < 1e-6f) continue;
        const float F = __fdiv_rn(A.size * B.size, A.size + B.size) * A.f * B.f;
        const float as = fabsf(s);
        const float sg = s > 0.f ? 1.f : -1.f;
        const float cr = (B.x - A.x) * B.s - (B.y - A.y) * B.c;      // cross(c_j - c_i, u_j)
        const float crg = (B.tx - A.tx) * B.s - (B.ty - A.ty) * B.c;
        acc[0].add(F * as);
        acc[1].add(F * (as * A.x + sg * cr * A.c));
        acc[2].add(F * (as * A.y + sg * cr * A.s));
        acc[3].add(F * (as * A.tx + sg * crg * A.c));
        acc[4].add(F * (as * A.ty + sg * crg * A.s));
        ++npair;
    }
    return npair;
}

// Combine the G lanes of each aligned G-lane group (all 32 lanes take part) and
// form the event's row; every lane of a group returns it.
template <int G>
__device__ __forceinline__ rta_stereo_t group_result(CSum (&acc)[5], int npair, int nvalid) {
    DW tot[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        DW v = two_sum(acc[k].s, acc[k].c);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const DW w = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
            v = dw_add(v, w);
        }
        tot[k] = v;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        npair += __shfl_xor_sync(0xffffffffu, npair, o);
        nvalid += __shfl_xor_sync(0xffffffffu, nvalid, o);
    }
    rta_stereo_t r = {};
    r.n_valid = nvalid;
    if (npair > 0 && tot[0].hi + tot[0].lo > 0.f) {
        r.dir_x = dw_div(tot[1], tot[0]);
        r.dir_y = dw_div(tot[2], tot[0]);
        r.core_x = dw_div(tot[3], tot[0]);
        r.core_y = dw_div(tot[4], tot[0]);
    } else {
        r.flags = RTA_SF_INVALID;
    }
    return r;
}

// A warp takes ST_EPW consecutive output rows at a time. Events of at most
// ST_SMALL_M images (most of them) are done side by side, ST_GL lanes each;
// larger ones one after another by the whole warp. Which of the two an event
// takes depends on its own image count only, so its row does not depend on
// the events around it (a sub-list of events gives the same rows).
__global__ void __launch_bounds__(ST_WARPS * 32) k_stereo(const StereoArgs a) {
    __shared__ StereoImg sh[ST_WARPS][RTA_STEREO_MAX_M];
    static_assert(ST_EPW * ST_SMALL_M <= RTA_STEREO_MAX_M && ST_EPW * ST_GL == 32, "small events share the warp");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / ST_GL, sub = lane % ST_GL;
    StereoImg* im = sh[warp];
    // a graph captured at capacity reads the bundle's counts at run time
    int64_t n_evt = a.n_evt_dev ? min(*a.n_evt_dev, a.n_evt) : a.n_evt;
    if (a.evt_idx) n_evt = min(int64_t(*a.n_list_dev), a.n_evt);
    const int64_t n_img = a.n_img_dev ? min(*a.n_img_dev, a.n_img) : a.n_img;
    const int64_t n_tiles = (n_evt + ST_EPW - 1) / ST_EPW;
    for (int64_t wt = int64_t(blockIdx.x) * ST_WARPS + warp; wt < n_tiles; wt += int64_t(gridDim.x) * ST_WARPS) {
        const int64_t e = wt * ST_EPW + g;                 // this group's output row
        int i0 = 0, m = 0;
        bool valid = false;
        if (e < n_evt) {
            const int64_t ev = a.evt_idx ? a.evt_idx[e] : e;
            const int b0 = a.evt_off[ev], b1 = a.evt_off[ev + 1];
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
        // small events: the group's lanes, slots ST_SMALL_M * g ...
        {
            const bool small = valid && m <= ST_SMALL_M;
            const int ms = small ? m : 0;
            StereoImg* gi = im + ST_SMALL_M * g;
            int nvalid = 0;
            for (int k = sub; k < ms; k += ST_GL) nvalid += stage_image(a, int64_t(i0) + k, gi + k);
            __syncwarp();
            CSum acc[5];
            const int npair = pair_sums<ST_GL>(gi, ms, sub, acc);
            const rta_stereo_t r = group_result<ST_GL>(acc, npair, nvalid);
            if (small && sub == 0) a.out[e] = r;
            __syncwarp();
        }
        // larger events: one at a time, the whole warp
        unsigned big = __ballot_sync(0xffffffffu, valid && m > ST_SMALL_M) & group_leaders();
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
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
    k_stereo<<<grid, ST_WARPS * 32, 0, s>>>(a);
    return cudaGetLastError();
}

int stereo_events_per_block() { return ST_WARPS * ST_EPW; }

}  // namespace rta
