// Stereo Hillas intersection (direction and core reconstruction, Sec. 4.1).
//
// One warp per event. The event's images (at most 64) are staged in shared
// memory; the lanes walk the upper triangle of image pairs (i < j) 32 apart and
// accumulate the weighted intersections; a shuffle tree sums the five partial
// sums. The weighted intersection is accumulated without dividing by
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

__global__ void __launch_bounds__(ST_WARPS * 32) k_stereo(const StereoArgs a) {
    __shared__ StereoImg sh[ST_WARPS][RTA_STEREO_MAX_M];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    StereoImg* im = sh[warp];
    const float kPiHi = 3.14159274101257324f;          // RN(pi), above pi
    const float kPiLo = -8.74227765734758577e-8f;      // pi - kPiHi
    const float kHalfPi = 1.57079637050628662f;
    // a graph captured at capacity reads the bundle's counts at run time
    int64_t n_evt = a.n_evt_dev ? min(*a.n_evt_dev, a.n_evt) : a.n_evt;
    if (a.evt_idx) n_evt = min(int64_t(*a.n_list_dev), a.n_evt);
    const int64_t n_img = a.n_img_dev ? min(*a.n_img_dev, a.n_img) : a.n_img;
    for (int64_t e = int64_t(blockIdx.x) * ST_WARPS + warp; e < n_evt; e += int64_t(gridDim.x) * ST_WARPS) {
        const int64_t ev = a.evt_idx ? a.evt_idx[e] : e;       // the event; e is the output row
        const int i0 = a.evt_off[ev], i1 = a.evt_off[ev + 1];
        if (i0 < 0 || i1 < i0 || i1 > n_img) {            // malformed CSR: flag, never index
            if (lane == 0) {
                atomicOr(a.status, RTA_DEV_BAD_IMAGE);
                rta_stereo_t r = {};
                r.flags = RTA_SF_INVALID;
                a.out[e] = r;
            }
            continue;
        }
        const int m = min(i1 - i0, RTA_STEREO_MAX_M);
        int nvalid_lane = 0;
        for (int k = lane; k < m; k += 32) {
            const rta_hillas_t hh = a.h[i0 + k];
            const int tel = a.img_tel[i0 + k];
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
            im[k] = v;
            nvalid_lane += used;
        }
        __syncwarp();
        CSum acc[5];
        int npair = 0;
        // pair p of the row-major upper triangle: (i, j), i < j; lanes start at p = lane
        const int T = m * (m - 1) / 2;
        int i = 0, j = 1 + lane;
        while (j >= m && i < m - 1) { ++i; j = j - m + i + 1; }
        for (int p = lane; p < T; p += 32) {
            const StereoImg A = im[i], B = im[j];
            j += 32;
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
        DW tot[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const DW v = two_sum(acc[k].s, acc[k].c);
            tot[k] = dw_warp_sum(v);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            npair += __shfl_xor_sync(0xffffffffu, npair, o);
            nvalid_lane += __shfl_xor_sync(0xffffffffu, nvalid_lane, o);
        }
        if (lane == 0) {
            rta_stereo_t r = {};
            r.n_valid = nvalid_lane;
            if (npair > 0 && tot[0].hi + tot[0].lo > 0.f) {
                r.dir_x = dw_div(tot[1], tot[0]);
                r.dir_y = dw_div(tot[2], tot[0]);
                r.core_x = dw_div(tot[3], tot[0]);
                r.core_y = dw_div(tot[4], tot[0]);
            } else {
                r.flags = RTA_SF_INVALID;
            }
            a.out[e] = r;
        }
        __syncwarp();
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

int stereo_events_per_block() { return ST_WARPS; }

}  // namespace rta
