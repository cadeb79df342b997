// Sky-count map of reconstructed directions and the transient search on it
// (the science alert search on multiple timescales, Sec. 2.1 (ii) and Sec. 4.2):
// 256 x 256 bins of 0.02 deg covering [-2.56, 2.56) deg in both nominal-frame
// coordinates, filled into one-second slabs (a ring of 30) and one-minute slabs
// (a ring of 60); the map of a moment is the sum of the last 30 one-second slabs.
//
// Transient search, per window (on seconds, off seconds before them): on and off
// counts per bin from the ring, row prefix sums, disk sums around every bin,
// and the Li & Ma (1983, Eq. 17) significance of the on/off pair in FP64 --
// a few hundred thousand FP64 operations per window, small even at GB300's
// FP64 rate -- with the bins at or above the threshold appended to a list.
//
// Binning, in FP32 with round-to-nearest and no contraction:
//   ix = floor((x + 2.56f) * 50.0f), kept when 0 <= ix < 256 (same for y);
//   bin = iy * 256 + ix. Events flagged RTA_EF_NO_DIRECTION are not counted.
#include "rta_launch.cuh"

namespace rta {

__global__ void k_skymap_fill(const rta_event_t* ev, int64_t n_evt, unsigned int* slab, unsigned int* slab_min) {
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n_evt; e += int64_t(gridDim.x) * blockDim.x) {
        const rta_event_t r = ev[e];
        if (r.flags & RTA_EF_NO_DIRECTION) continue;
        const int ix = sky_bin(r.dir_x), iy = sky_bin(r.dir_y);
        if (ix < 0 || iy < 0) continue;
        if (slab) atomicAdd(slab + iy * RTA_SKY_N + ix, 1u);
        if (slab_min) atomicAdd(slab_min + iy * RTA_SKY_N + ix, 1u);
    }
}

// Per-bin counts of a window from a ring of n_slabs slabs: bit k of use_on /
// use_off selects slab k. Integer sums, exact.
__global__ void k_window_counts(const unsigned int* slabs, int n_slabs, unsigned long long use_on,
                                unsigned long long use_off, unsigned int* on, unsigned int* off) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < RTA_SKY_N * RTA_SKY_N; b += gridDim.x * blockDim.x) {
        unsigned int so = 0, sf = 0;
        for (int k = 0; k < n_slabs; ++k) {
            const unsigned int v = slabs[size_t(k) * RTA_SKY_N * RTA_SKY_N + b];
            if ((use_on >> k) & 1ull) so += v;
            if ((use_off >> k) & 1ull) sf += v;
        }
        on[b] = so;
        off[b] = sf;
    }
}

// Row prefix sums pre[y * 257 + x] = sum of m[y][x'] for x' < x, one warp per
// (row, map); each lane owns eight consecutive columns.
__global__ void k_row_prefix(const unsigned int* on, const unsigned int* off, unsigned int* pre_on,
                             unsigned int* pre_off) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= 2 * RTA_SKY_N) return;
    const int y = w % RTA_SKY_N;
    const unsigned int* m = (w < RTA_SKY_N ? on : off) + y * RTA_SKY_N;
    unsigned int* pre = (w < RTA_SKY_N ? pre_on : pre_off) + y * (RTA_SKY_N + 1);
    unsigned int v[8], t = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        v[i] = m[8 * lane + i];
        t += v[i];
    }
    unsigned int incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    unsigned int run = incl - t;          // exclusive prefix of this lane's block
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        pre[8 * lane + i] = run;
        run += v[i];
    }
    if (lane == 31) pre[RTA_SKY_N] = run;
}

// Li & Ma (1983) Eq. 17, signed; the expression order of the oracle.
__device__ __forceinline__ double li_ma(double n_on, double n_off, double alpha) {
    const double tot = n_on + n_off;
    if (!(tot > 0.0)) return 0.0;
    const double t1 = n_on > 0.0 ? n_on * log((1.0 + alpha) / alpha * (n_on / tot)) : 0.0;
    const double t2 = n_off > 0.0 ? n_off * log((1.0 + alpha) * (n_off / tot)) : 0.0;
    const double s = sqrt(fmax(2.0 * (t1 + t2), 0.0));
    return n_on >= alpha * n_off ? s : -s;
}

// Disk sums around every bin (hw[dy + R]: half-width of the disk's row dy),
// significance, and the bins at or above s_min appended to `alerts`.
__global__ void k_transient(const unsigned int* pre_on, const unsigned int* pre_off, const int* hw, int R,
                            double alpha, double s_min, int window, rta_alert_t* alerts, unsigned int* n_alerts,
                            unsigned int cap, double* sig, int64_t* d_on, int64_t* d_off) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < RTA_SKY_N * RTA_SKY_N; b += gridDim.x * blockDim.x) {
        const int y = b / RTA_SKY_N, x = b % RTA_SKY_N;
        int64_t so = 0, sf = 0;
        for (int dy = -R; dy <= R; ++dy) {
            const int yy = y + dy;
            if (yy < 0 || yy >= RTA_SKY_N) continue;
            const int w = hw[dy + R];
            const int x0 = max(0, x - w), x1 = min(RTA_SKY_N - 1, x + w);
            const int r = yy * (RTA_SKY_N + 1);
            so += int64_t(pre_on[r + x1 + 1]) - int64_t(pre_on[r + x0]);
            sf += int64_t(pre_off[r + x1 + 1]) - int64_t(pre_off[r + x0]);
        }
        const double s = li_ma(double(so), double(sf), alpha);
        if (sig) sig[b] = s;
        if (d_on) d_on[b] = so;
        if (d_off) d_off[b] = sf;
        if (alerts && s >= s_min) {
            const unsigned int k = atomicAdd(n_alerts, 1u);
            if (k < cap) {
                rta_alert_t a;
                a.window = window;
                a.ix = x;
                a.iy = y;
                a.pad = 0;
                a.n_on = so;
                a.n_off = sf;
                a.alpha = alpha;
                a.significance = s;
                alerts[k] = a;
            }
        }
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
        ev[e] = stereo_event_row(st[e]);
    }
}

cudaError_t launch_skymap_fill(const rta_event_t* ev, int64_t n_evt, unsigned int* slab, unsigned int* slab_min,
                               cudaStream_t s) {
    const int grid = int(n_evt / 256 + 1 < 4096 ? n_evt / 256 + 1 : 4096);
    k_skymap_fill<<<grid, 256, 0, s>>>(ev, n_evt, slab, slab_min);
    return cudaGetLastError();
}

cudaError_t launch_transient(const TransientArgs& t, cudaStream_t s) {
    k_window_counts<<<256, 256, 0, s>>>(t.slabs, t.n_slabs, t.use_on, t.use_off, t.on, t.off);
    k_row_prefix<<<2 * RTA_SKY_N * 32 / 256, 256, 0, s>>>(t.on, t.off, t.pre_on, t.pre_off);
    k_transient<<<256, 256, 0, s>>>(t.pre_on, t.pre_off, t.hw, t.R, t.alpha, t.s_min, t.window, t.alerts, t.n_alerts,
                                    t.cap, t.sig, t.d_on, t.d_off);
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
