// Stereo Hillas intersection (direction and core reconstruction, Sec. 4.1).
//
// One warp per event. The event's images (at most 64) are staged in shared
// memory; lanes then take the pairs (i, j > i) and accumulate the weighted
// intersections, and a shuffle tree sums the five partial sums. The weighted
// intersection is accumulated without dividing by sin(psi_j - psi_i):
//   w * p = F * (|s| * c_i + sign(s) * cross(c_j - c_i, u_j) * u_i),
// with F = s_i s_j / (s_i + s_j) (1 - W_i/L_i)(1 - W_j/L_j) and s = cross(u_i, u_j),
// which is the same quantity as |s| F * (c_i + u_i cross / s) but stays well
// conditioned for nearly parallel axes. The pair arithmetic is FP64: when every
// pair of an event is nearly parallel, the result is a ratio of two small sums
// and FP32 rounding of the axis directions alone would move it by far more
// than the rounding of the inputs. The work is a few hundred pairs per event,
// far below the image kernel's cost.
#include "rta_launch.cuh"

namespace rta {

constexpr int ST_WARPS = 8;


struct StereoImg {
    double x, y, c, s, f, tx, ty, size;  // f = 1 - W/L, 0 if unused
    int used;
    int pad;
};

__global__ void __launch_bounds__(ST_WARPS * 32) k_stereo(const StereoArgs a) {
    __shared__ StereoImg sh[ST_WARPS][RTA_STEREO_MAX_M];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    StereoImg* im = sh[warp];
    for (int64_t e = int64_t(blockIdx.x) * ST_WARPS + warp; e < a.n_evt; e += int64_t(gridDim.x) * ST_WARPS) {
        const int i0 = a.evt_off[e], i1 = a.evt_off[e + 1];
        if (i0 < 0 || i1 < i0 || i1 > a.n_img) {            // malformed CSR: flag, never index
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
            double sp = 0.0, cp = 1.0;
            if (used) sincos(double(hh.psi), &sp, &cp);
            v.x = hh.x;
            v.y = hh.y;
            v.c = cp;
            v.s = sp;
            v.f = used ? 1.0 - double(hh.width) / double(hh.length) : 0.0;
            const float2 t = tel_ok ? a.arr.tel_xy[tel] : make_float2(0.f, 0.f);
            v.tx = t.x;
            v.ty = t.y;
            v.size = hh.size;
            v.used = used;
            v.pad = 0;
            im[k] = v;
            nvalid_lane += used;
        }
        __syncwarp();
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        int npair = 0;
        for (int i = 0; i < m; ++i) {
            if (!im[i].used) continue;
            const StereoImg A = im[i];
            for (int j = i + 1 + lane; j < m; j += 32) {
                const StereoImg B = im[j];
                if (!B.used) continue;
                const double s = A.c * B.s - A.s * B.c;   // sin(psi_j - psi_i)
                if (fabs(s) < 1e-6) continue;
                const double F = A.size * B.size / (A.size + B.size) * A.f * B.f;
                const double as = fabs(s);
                const double sg = s > 0.0 ? 1.0 : -1.0;
                const double cr = (B.x - A.x) * B.s - (B.y - A.y) * B.c;      // cross(c_j - c_i, u_j)
                const double crg = (B.tx - A.tx) * B.s - (B.ty - A.ty) * B.c;
                acc[0] += F * as;
                acc[1] += F * (as * A.x + sg * cr * A.c);
                acc[2] += F * (as * A.y + sg * cr * A.s);
                acc[3] += F * (as * A.tx + sg * crg * A.c);
                acc[4] += F * (as * A.ty + sg * crg * A.s);
                ++npair;
            }
        }
#pragma unroll
        for (int k = 0; k < 5; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            npair += __shfl_xor_sync(0xffffffffu, npair, o);
            nvalid_lane += __shfl_xor_sync(0xffffffffu, nvalid_lane, o);
        }
        if (lane == 0) {
            rta_stereo_t r = {};
            r.n_valid = nvalid_lane;
            if (npair > 0 && acc[0] > 0.0) {
                r.dir_x = float(acc[1] / acc[0]);
                r.dir_y = float(acc[2] / acc[0]);
                r.core_x = float(acc[3] / acc[0]);
                r.core_y = float(acc[4] / acc[0]);
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
