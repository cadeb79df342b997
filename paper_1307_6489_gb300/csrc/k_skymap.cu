// Sky-count map of reconstructed directions (the input of the science alert
// search on multiple timescales, Sec. 2.1 (ii) and Sec. 4.2): 256 x 256 bins of
// 0.02 deg covering [-2.56, 2.56) deg in both nominal-frame coordinates, filled
// into one-second slabs; the map of a moment is the sum of the last 30 slabs.
//
// Binning, in FP32 with round-to-nearest and no contraction:
//   ix = floor((x + 2.56f) * 50.0f), kept when 0 <= ix < 256 (same for y);
//   bin = iy * 256 + ix. Events flagged RTA_EF_NO_DIRECTION are not counted.
#include "rta_launch.cuh"

namespace rta {

__device__ __forceinline__ int sky_bin(float v) {
    const float u = __fmul_rn(__fadd_rn(v, 2.56f), 50.0f);
    if (!(u >= 0.f) || !(u < float(RTA_SKY_N))) return -1;   // also rejects NaN
    return int(floorf(u));
}

__global__ void k_skymap_fill(const rta_event_t* ev, int64_t n_evt, unsigned int* slab) {
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n_evt; e += int64_t(gridDim.x) * blockDim.x) {
        const rta_event_t r = ev[e];
        if (r.flags & RTA_EF_NO_DIRECTION) continue;
        const int ix = sky_bin(r.dir_x), iy = sky_bin(r.dir_y);
        if (ix < 0 || iy < 0) continue;
        atomicAdd(slab + iy * RTA_SKY_N + ix, 1u);
    }
}

// out[b] = sum over the selected slabs (bit s of `use`) of slabs[s][b]; integer sums are exact.
__global__ void k_skymap_sum(const unsigned int* slabs, unsigned long long use, unsigned int* out) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < RTA_SKY_N * RTA_SKY_N; b += gridDim.x * blockDim.x) {
        unsigned int s = 0;
        for (int k = 0; k < RTA_SKY_SLABS; ++k)
            if ((use >> k) & 1ull) s += slabs[size_t(k) * RTA_SKY_N * RTA_SKY_N + b];
        out[b] = s;
    }
}

// Event rows from geometric stereo rows (used when no learned model is attached).
__global__ void k_stereo_to_events(const rta_stereo_t* st, int64_t n_evt, rta_event_t* ev) {
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n_evt; e += int64_t(gridDim.x) * blockDim.x) {
        const rta_stereo_t s = st[e];
        rta_event_t r = {};
        r.log_energy = __int_as_float(0x7fc00000);   // no energy estimate
        r.gammaness = __int_as_float(0x7fc00000);
        r.dir_x = s.dir_x;
        r.dir_y = s.dir_y;
        r.n_used = s.n_valid;
        r.flags = (s.flags & RTA_SF_INVALID) ? RTA_EF_NO_DIRECTION : 0u;
        ev[e] = r;
    }
}

cudaError_t launch_skymap_fill(const rta_event_t* ev, int64_t n_evt, unsigned int* slab, cudaStream_t s) {
    const int grid = int(n_evt / 256 + 1 < 4096 ? n_evt / 256 + 1 : 4096);
    k_skymap_fill<<<grid, 256, 0, s>>>(ev, n_evt, slab);
    return cudaGetLastError();
}

cudaError_t launch_skymap_sum(const unsigned int* slabs, unsigned long long use, unsigned int* out, cudaStream_t s) {
    k_skymap_sum<<<256, 256, 0, s>>>(slabs, use, out);
    return cudaGetLastError();
}

cudaError_t launch_stereo_to_events(const rta_stereo_t* st, int64_t n_evt, rta_event_t* ev, cudaStream_t s) {
    const int grid = int(n_evt / 256 + 1 < 4096 ? n_evt / 256 + 1 : 4096);
    k_stereo_to_events<<<grid, 256, 0, s>>>(st, n_evt, ev);
    return cudaGetLastError();
}

}  // namespace rta
