// Stereo Hillas intersection (direction and core reconstruction, Sec. 4.1).
//
// One warp per event. The event's images (at most 64) are staged in shared
// memory; the lanes then share out the m*m index pairs (i, j), keep those with
// i < j, and accumulate the weighted intersections; a shuffle tree sums the five
// partial sums. The weighted intersection is accumulated without dividing by
// s = sin(psi_j - psi_i):
//   w * p = F * (|s| * c_i + sign(s) * cross(c_j - c_i, u_j) * u_i),
// with F = s_i s_j / (s_i + s_j) (1 - W_i/L_i)(1 - W_j/L_j), the same quantity as
// |s| F * (c_i + u_i cross / s) but well conditioned for nearly parallel axes.
// Precision: when every pair of an event is nearly parallel the result is a
// ratio of small sums, so s must be accurate relative to itself. It is taken as
// sinf of the angle difference computed exactly in FP64 and reduced to
// (-pi/2, pi/2] (sin(d - pi) = -sin d), never as a difference of products of
// rounded cosines; everything else is FP32, each lane's sums are compensated
// (Kahan-Babuska) and the lanes are combined in FP64.
#include "rta_launch.cuh"

namespace rta {

constexpr int ST_WARPS = 8;

struct StereoImg {
    float x, y, c, s, psi, f, tx, ty, size;  // f = 1 - W/L
    int used;
};

// Compensated running sum (Neumaier's variant of Kahan summation).
struct CSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float t = s + v;
        c += (fabsf(s) >= fabsf(v)) ? (s - t) + v : (v - t) + s;
        s = t;
    }
    __device__ __forceinline__ double value() const { return double(s) + double(c); }
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(ST_WARPS * 32) k_stereo(const StereoArgs a) {
    __shared__ StereoImg sh[ST_WARPS][RTA_STEREO_MAX_M];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    StereoImg* im = sh[warp];
    const double kPi = 3.141592653589793;
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
            im[k] = v;
            nvalid_lane += used;
        }
        __syncwarp();
        CSum acc[5];
        int npair = 0;
        for (int p = lane; p < m * m; p += 32) {
            const int i = p / m, j = p - i * m;
            if (j <= i) continue;
            const StereoImg A = im[i], B = im[j];
            if (!A.used || !B.used) continue;
            double d = double(B.psi) - double(A.psi);     // exact: both are FP32 values
            float sgn = 1.f;
            if (d > 0.5 * kPi) { d -= kPi; sgn = -1.f; }
            else if (d <= -0.5 * kPi) { d += kPi; sgn = -1.f; }
            const float s = sgn * sinf(float(d));         // sin(psi_j - psi_i), relatively accurate
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
        double tot[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) tot[k] = warp_sum_d(acc[k].value());
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            npair += __shfl_xor_sync(0xffffffffu, npair, o);
            nvalid_lane += __shfl_xor_sync(0xffffffffu, nvalid_lane, o);
        }
        if (lane == 0) {
            rta_stereo_t r = {};
            r.n_valid = nvalid_lane;
            if (npair > 0 && tot[0] > 0.0) {
                r.dir_x = float(tot[1] / tot[0]);
                r.dir_y = float(tot[2] / tot[0]);
                r.core_x = float(tot[3] / tot[0]);
                r.core_y = float(tot[4] / tot[0]);
            } else {
                r.flags = RTA_SF_INVALID;
            }
            a.out[e] = r;
        }
        __syncwarp();
    }
}

cudaError_t launch_stereo(const StereoArgs& a, int grid, cudaStream_t s) {
    k_stereo<<<grid, ST_WARPS * 32, 0, s>>>(a);
    return cudaGetLastError();
}

int stereo_events_per_block() { return ST_WARPS; }

}  // namespace rta
