// Lookup-table reconstruction: the calibration matrices of the real-time
// reconstruction (Sec. 4.1), i.e. per camera type a grid over (image size,
// impact distance) of the mean and spread of image width, length and log10 E
// of gamma-ray images; scaled width and length and a weighted energy per event.
//
// k_lut_events: one block per group of events. All threads compute the
// per-image terms of the group's images, enumerated flat (an exclusive scan of
// the events' image counts) and staged in shared memory piece by piece; then
// each event's thread adds its own terms in image order, so the result does
// not depend on the launch shape. Bin decisions are FP32 comparisons; every
// FP64 step is a single IEEE rounding (explicit _rn intrinsics keep the
// compiler from fusing a multiply into an add). The per-cell divisions live in
// the table's lookup form (k_lut_prepare), so an image costs two FP64
// subtractions and two multiplications before the sums.
//
// FP64 runs at 2 lanes per clock per SM on this part, so a warp-wide FP64
// instruction holds its sub-partition's pipe for a long time whatever the
// number of active lanes. The group's events are therefore dealt round-robin
// to the four warps (slot k -> warp k % 4, lane k / 4): the per-event sums and
// divisions of one group run on all four sub-partitions at once.
//
// k_lut_train: one thread per training event, FP64 atomic sums per cell.
// k_lut_finalize, k_lut_prepare: one thread per cell.
#include <algorithm>

#include "rta_launch.cuh"

namespace rta {

namespace {

constexpr int LUT_THREADS = 128;
constexpr int LUT_WARPS = LUT_THREADS / 32;
constexpr int LUT_MAX_EPB = 128;    // events per group at most (one thread each)
constexpr int LUT_PIECE = 1024;     // per-image terms staged per pass

// The lookup form of one cell (RTA_LUT_LOOKUP_BYTES = 64 bytes).
struct LutLookup {
    double inv_w, inv_l;    // 1 / sigma_w, 1 / sigma_l
    double w_e, w_e_mean;   // 1 / sigma_e^2, that times mean_e
    double mean_w, mean_l;
    long long used;
    long long pad;
};
static_assert(sizeof(LutLookup) == RTA_LUT_LOOKUP_BYTES, "lookup cell layout");

struct LutSmem {
    float se[RTA_LUT_MAX_BINS + 1];
    float de[RTA_LUT_MAX_BINS + 1];
    long long cnt[LUT_MAX_EPB];        // image count of each event slot
    long long pre[LUT_MAX_EPB + 1];    // flat offset of each slot's first image in the group
    int first[LUT_MAX_EPB];            // its first image index
    float2 core[LUT_MAX_EPB];
    double tw[LUT_PIECE], tl[LUT_PIECE], tn[LUT_PIECE], td[LUT_PIECE];
    int tu[LUT_PIECE];                 // 1: the image is used
};

// i with e[i] <= v < e[i + 1], -1 outside [e[0], e[n]) or for NaN. For sorted
// edges this is the bin; for any edges the result stays in [-1, n).
__device__ __forceinline__ int bin_of(float v, const float* e, int n) {
    if (!(v >= e[0]) || !(v < e[n])) return -1;
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (v >= e[mid]) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Ground distance from a telescope to the core, one FP32 rounding per operation.
__device__ __forceinline__ float impact_distance(float cx, float cy, float2 t) {
    const float dx = __fsub_rn(cx, t.x), dy = __fsub_rn(cy, t.y);
    return __fsqrt_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)));
}

struct LutImage {
    float size, width, length;
    int cam;
    float2 txy;
    bool ok;
};

// The fields of image i the tables need, and whether it counts (a known
// telescope, >= 3 pixels, neither empty nor bad input).
__device__ __forceinline__ LutImage load_image(const LutArgs& a, int64_t i) {
    const float4* hr = reinterpret_cast<const float4*>(a.h + i);
    const float4 h0 = __ldg(hr), h1 = __ldg(hr + 1), h2 = __ldg(hr + 2);
    const int tel = __ldg(a.img_tel + i);
    LutImage m;
    m.size = h0.x;
    m.length = h0.w;
    m.width = h1.x;
    const bool tel_ok = tel >= 0 && tel < a.arr.n_tel;
    m.ok = tel_ok && __float_as_int(h2.z) >= 3 && !(__float_as_uint(h2.w) & (RTA_HF_EMPTY | RTA_HF_BAD_INPUT));
    m.cam = tel_ok ? __ldg(a.arr.tel_cam + tel) : 0;
    m.txy = tel_ok ? __ldg(a.arr.tel_xy + tel) : make_float2(0.f, 0.f);
    return m;
}

__device__ __forceinline__ int64_t cell_index(const LutArgs& a, int cam, int iu, int ir) {
    return (int64_t(cam) * a.n_size + iu) * a.n_dist + ir;
}

// The terms of the group's images with flat index in [p0, p1), p1 - p0 <=
// LUT_PIECE, into shared memory. A thread takes LUT_ILP images at a time and
// issues each stage's loads for all of them before using any, so the chain
// image row -> telescope -> cell costs three memory latencies per batch
// instead of three per image.
constexpr int LUT_ILP = 4;

__device__ __forceinline__ void stage_terms(const LutArgs& a, LutSmem& sm, int epb, long long p0, long long p1) {
    for (long long base = p0 + threadIdx.x; base < p1; base += LUT_THREADS * LUT_ILP) {
        int64_t img[LUT_ILP];
        int slot[LUT_ILP];
        bool live[LUT_ILP];
#pragma unroll
        for (int u = 0; u < LUT_ILP; ++u) {
            const long long j = base + u * LUT_THREADS;
            live[u] = j < p1;
            int lo = 0, hi = epb;              // sm.pre[lo] <= j < sm.pre[hi]
            if (live[u]) {
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (sm.pre[mid] <= j) lo = mid;
                    else hi = mid;
                }
            }
            slot[u] = lo;
            img[u] = live[u] ? int64_t(sm.first[lo]) + (j - sm.pre[lo]) : 0;
        }
        float4 h0[LUT_ILP];
        float wid[LUT_ILP];
        int2 pf[LUT_ILP];
        int tel[LUT_ILP];
#pragma unroll
        for (int u = 0; u < LUT_ILP; ++u) {
            if (live[u]) {
                const float4* hr = reinterpret_cast<const float4*>(a.h + img[u]);
                h0[u] = __ldg(hr);                                   // size, x, y, length
                wid[u] = __ldg(reinterpret_cast<const float*>(hr + 1));  // width
                pf[u] = __ldg(reinterpret_cast<const int2*>(hr + 2) + 1);  // n_pix, flags
                tel[u] = __ldg(a.img_tel + img[u]);
            } else {
                h0[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                wid[u] = 0.f;
                pf[u] = make_int2(0, 0);
                tel[u] = -1;
            }
        }
        bool ok[LUT_ILP];
        int cam[LUT_ILP];
        float2 txy[LUT_ILP];
#pragma unroll
        for (int u = 0; u < LUT_ILP; ++u) {
            ok[u] = live[u] && tel[u] >= 0 && tel[u] < a.arr.n_tel && pf[u].x >= 3 &&
                    !(uint32_t(pf[u].y) & (RTA_HF_EMPTY | RTA_HF_BAD_INPUT));
            cam[u] = ok[u] ? __ldg(a.arr.tel_cam + tel[u]) : 0;
            txy[u] = ok[u] ? __ldg(a.arr.tel_xy + tel[u]) : make_float2(0.f, 0.f);
        }
        const LutLookup* lk[LUT_ILP];
#pragma unroll
        for (int u = 0; u < LUT_ILP; ++u) {
            lk[u] = nullptr;
            if (ok[u]) {
                const float2 c = sm.core[slot[u]];
                const int iu = bin_of(h0[u].x, sm.se, a.n_size);
                const int ir = bin_of(impact_distance(c.x, c.y, txy[u]), sm.de, a.n_dist);
                if (iu >= 0 && ir >= 0)
                    lk[u] = reinterpret_cast<const LutLookup*>(a.lookup) + cell_index(a, cam[u], iu, ir);
            }
        }
        double2 f0[LUT_ILP], f1[LUT_ILP], f2[LUT_ILP];
        long long f3[LUT_ILP];
#pragma unroll
        for (int u = 0; u < LUT_ILP; ++u) {
            if (lk[u]) {
                const double2* cp = reinterpret_cast<const double2*>(lk[u]);
                f0[u] = __ldg(cp);
                f1[u] = __ldg(cp + 1);
                f2[u] = __ldg(cp + 2);
                f3[u] = __ldg(reinterpret_cast<const long long*>(cp + 3));
            } else {
                f0[u] = f1[u] = f2[u] = make_double2(0.0, 0.0);
                f3[u] = 0;
            }
        }
#pragma unroll
        for (int u = 0; u < LUT_ILP; ++u) {
            if (!live[u]) continue;
            // f0 = (1/sigma_w, 1/sigma_l), f1 = (w_e, w_e mean_e), f2 = (mean_w, mean_l), f3 = used
            const bool used = f3[u] != 0;
            const int k = int(base + u * LUT_THREADS - p0);
            sm.tw[k] = used ? __dmul_rn(__dsub_rn(double(wid[u]), f2[u].x), f0[u].x) : 0.0;
            sm.tl[k] = used ? __dmul_rn(__dsub_rn(double(h0[u].w), f2[u].y), f0[u].y) : 0.0;
            sm.tn[k] = f1[u].y;
            sm.td[k] = f1[u].x;
            sm.tu[k] = used;
        }
    }
}

__global__ void __launch_bounds__(LUT_THREADS) k_lut_events(const LutArgs a) {
    __shared__ LutSmem sm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int slot = lane * LUT_WARPS + warp;          // this thread's event in the group
    for (int k = tid; k <= a.n_size; k += LUT_THREADS) sm.se[k] = a.size_edges[k];
    for (int k = tid; k <= a.n_dist; k += LUT_THREADS) sm.de[k] = a.dist_edges[k];
    const int epb = a.events_per_block;
    const double cw_lo = a.cut[0], cw_hi = a.cut[1], cl_lo = a.cut[2], cl_hi = a.cut[3];
    for (int64_t e0 = int64_t(blockIdx.x) * epb; e0 < a.n_evt; e0 += int64_t(gridDim.x) * epb) {
        const int64_t e = e0 + slot;
        const bool mine = slot < epb && e < a.n_evt;
        int state = 3;                       // 0 fold, 1 malformed, 2 no core, 3 no event
        if (slot < epb) {
            long long cnt = 0;
            int i0 = 0;
            if (mine) {
                i0 = a.evt_off[e];
                const int i1 = a.evt_off[e + 1];
                if (i0 < 0 || i1 < i0 || i1 > a.n_img) {
                    state = 1;
                    atomicOr(a.status, RTA_DEV_BAD_IMAGE);
                } else {
                    const float4* sr = reinterpret_cast<const float4*>(a.stereo + e);
                    const float4 s0 = __ldg(sr), s1 = __ldg(sr + 1);
                    if (__float_as_uint(s1.y) & RTA_SF_INVALID) {
                        state = 2;
                    } else {
                        state = 0;
                        cnt = i1 - i0;
                        sm.core[slot] = make_float2(s0.z, s0.w);
                    }
                }
            }
            sm.cnt[slot] = cnt;
            sm.first[slot] = i0;
        }
        __syncthreads();
        // exclusive scan of the slots' image counts: warp 0, four slots a lane
        if (warp == 0) {
            long long v[4], s = 0;
            for (int q = 0; q < 4; ++q) {
                const int k = lane * 4 + q;
                v[q] = k < epb ? sm.cnt[k] : 0;
                s += v[q];
            }
            long long incl = s;
            for (int d = 1; d < 32; d <<= 1) {
                const long long u = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += u;
            }
            long long run = incl - s;
            for (int q = 0; q < 4; ++q) {
                const int k = lane * 4 + q;
                if (k < epb) sm.pre[k] = run;
                run += v[q];
            }
            if (lane == 31) sm.pre[epb] = incl;    // the group's image total
        }
        __syncthreads();
        const long long total = sm.pre[epb];
        const long long my0 = slot < epb ? sm.pre[slot] : 0, my1 = slot < epb ? sm.pre[slot + 1] : 0;
        double sw = 0.0, sl = 0.0, sn = 0.0, sd = 0.0;
        int n = 0;
        for (long long p0 = 0; p0 < total; p0 += LUT_PIECE) {
            const long long p1 = min(total, p0 + LUT_PIECE);
            stage_terms(a, sm, epb, p0, p1);
            __syncthreads();
            const long long j0 = max(my0, p0), j1 = min(my1, p1);
            for (long long j = j0; j < j1; ++j) {
                const int k = int(j - p0);
                if (sm.tu[k]) {
                    ++n;
                    sw = __dadd_rn(sw, sm.tw[k]);
                    sl = __dadd_rn(sl, sm.tl[k]);
                    sn = __dadd_rn(sn, sm.tn[k]);
                    sd = __dadd_rn(sd, sm.td[k]);
                }
            }
            __syncthreads();
        }
        if (mine) {
            float4 o0 = make_float4(0.f, 0.f, 0.f, 0.f), o1 = o0;
            uint32_t flags = 0;
            int n_used = 0;
            if (state == 1) {
                flags = RTA_LF_MALFORMED;
                n_used = -1;
            } else if (state == 2) {
                flags = RTA_LF_NO_CORE;
            } else if (n == 0) {
                flags = RTA_LF_NO_IMAGE;
            } else {
                const double dn = double(n);
                const double mscw = __ddiv_rn(sw, dn), mscl = __ddiv_rn(sl, dn);
                const double le = __ddiv_rn(sn, sd);
                const double sg = __dsqrt_rn(__ddiv_rn(1.0, sd));
                if (cw_lo <= mscw && mscw <= cw_hi && cl_lo <= mscl && mscl <= cl_hi) flags = RTA_LF_GAMMA;
                n_used = n;
                o0 = make_float4(__double2float_rn(le), __double2float_rn(sg), __double2float_rn(mscw),
                                 __double2float_rn(mscl));
            }
            o1.x = __int_as_float(n_used);
            o1.y = __uint_as_float(flags);
            float4* op = reinterpret_cast<float4*>(a.out + e);
            op[0] = o0;
            op[1] = o1;
        }
        __syncthreads();   // the next group reuses the shared arrays
    }
}

__global__ void __launch_bounds__(256) k_lut_train(const LutArgs a) {
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < a.n_evt;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int i0 = a.evt_off[e], i1 = a.evt_off[e + 1];
        if (i0 < 0 || i1 < i0 || i1 > a.n_img) continue;
        if (a.use && !a.use[e]) continue;
        const float cx = a.core_xy[2 * e], cy = a.core_xy[2 * e + 1];
        const double le = double(a.log_e[e]);
        for (int i = i0; i < i1; ++i) {
            const LutImage m = load_image(a, i);
            if (!m.ok) continue;
            const int iu = bin_of(m.size, a.size_edges, a.n_size);
            const int ir = bin_of(impact_distance(cx, cy, m.txy), a.dist_edges, a.n_dist);
            if (iu < 0 || ir < 0) continue;
            double* s = a.acc + 8 * cell_index(a, m.cam, iu, ir);
            const double w = double(m.width), l = double(m.length);
            atomicAdd(s + 0, 1.0);
            atomicAdd(s + 1, w);
            atomicAdd(s + 2, __dmul_rn(w, w));
            atomicAdd(s + 3, l);
            atomicAdd(s + 4, __dmul_rn(l, l));
            atomicAdd(s + 5, le);
            atomicAdd(s + 6, __dmul_rn(le, le));
        }
    }
}

__global__ void __launch_bounds__(256) k_lut_finalize(const double* acc, int64_t n_cells, int min_count,
                                                      rta_lut_cell_t* cells) {
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < n_cells;
         c += int64_t(gridDim.x) * blockDim.x) {
        const double* s = acc + 8 * c;
        const double n = s[0];
        float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (n >= double(min_count)) {
            for (int k = 0; k < 3; ++k) {
                const double mean = __ddiv_rn(s[1 + 2 * k], n);
                double var = __dsub_rn(__ddiv_rn(s[2 + 2 * k], n), __dmul_rn(mean, mean));
                if (var < 0.0) var = 0.0;
                v[2 * k] = __double2float_rn(mean);
                v[2 * k + 1] = __double2float_rn(__dsqrt_rn(var));
            }
        }
        const int ni = n < 2147483647.0 ? int(n) : 2147483647;
        float4* o = reinterpret_cast<float4*>(cells + c);
        o[0] = make_float4(__int_as_float(ni), v[0], v[1], v[2]);
        o[1] = make_float4(v[3], v[4], v[5], 0.f);
    }
}

__global__ void __launch_bounds__(256) k_lut_prepare(const rta_lut_cell_t* cells, int64_t n_cells,
                                                     LutLookup* lookup) {
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < n_cells;
         c += int64_t(gridDim.x) * blockDim.x) {
        const float4* cp = reinterpret_cast<const float4*>(cells + c);
        const float4 c0 = __ldg(cp), c1 = __ldg(cp + 1);
        // c0 = (n, mean_w, sigma_w, mean_l), c1 = (sigma_l, mean_e, sigma_e, -)
        LutLookup o = {};
        if (__float_as_int(c0.x) >= 1 && c0.z > 0.f && c1.x > 0.f && c1.z > 0.f) {
            o.inv_w = __ddiv_rn(1.0, double(c0.z));
            o.inv_l = __ddiv_rn(1.0, double(c1.x));
            o.w_e = __ddiv_rn(1.0, __dmul_rn(double(c1.z), double(c1.z)));
            o.w_e_mean = __dmul_rn(double(c1.y), o.w_e);
            o.mean_w = double(c0.y);
            o.mean_l = double(c0.w);
            o.used = 1;
        }
        lookup[c] = o;
    }
}

}  // namespace

int lut_events_per_block(int64_t n_evt, int n_sm) {
    // about one group per SM, 16..128 events each, a multiple of 4 (one per warp)
    int64_t epb = (n_evt + int64_t(n_sm) - 1) / int64_t(n_sm);
    epb = (epb + 3) / 4 * 4;
    return int(std::min<int64_t>(LUT_MAX_EPB, std::max<int64_t>(16, epb)));
}

cudaError_t launch_lut_reconstruct(const LutArgs& a, int grid, cudaStream_t s) {
    k_lut_events<<<grid, LUT_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_lut_accumulate(const LutArgs& a, int grid, cudaStream_t s) {
    k_lut_train<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_lut_prepare(const rta_lut_cell_t* cells, int64_t n_cells, void* lookup, int grid, cudaStream_t s) {
    k_lut_prepare<<<grid, 256, 0, s>>>(cells, n_cells, static_cast<LutLookup*>(lookup));
    return cudaGetLastError();
}

cudaError_t launch_lut_finalize(const double* acc, int64_t n_cells, int min_count, rta_lut_cell_t* cells, int grid,
                                cudaStream_t s) {
    k_lut_finalize<<<grid, 256, 0, s>>>(acc, n_cells, min_count, cells);
    return cudaGetLastError();
}

}  // namespace rta
