// Kernels of the learned deep-sets surrogate (energy, direction offset and
// gamma/hadron score; the paper's Sec. 4.1 asks RT-RECO for energy and
// gamma/hadron separation next to the direction).
//
//   k_features   per event: used images, baseline (two brightest axes), 12 features per image
//   k_pool / k_pool_bwd, k_head_bwd, k_loss, k_adam, k_colsum, k_reduce_splits
// (the dense layers, forward and backward, are tensor-core GEMMs: k_gemm_tc.cu)
//
// Row-major matrices throughout. Activations are stored in BF16 (the operand
// type of the next GEMM); biases, the output layer's backward pass and every
// gradient reduction are FP32.
#include "rta_mlp_dev.cuh"

namespace rta {

// ------------------------------------------------------------------ features
// SUR_EVT_LANES lanes per event; the inference kernel forms baselines and features the same way.
__global__ void __launch_bounds__(256) k_features(const FeatArgs a) {
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int sub = lane % SUR_EVT_LANES;
    constexpr int GROUPS = 32 / SUR_EVT_LANES;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int64_t n_evt = a.n_evt_dev ? min(*a.n_evt_dev, a.n_evt) : a.n_evt;
    const int64_t n_img = a.n_img_dev ? min(*a.n_img_dev, a.n_img) : a.n_img;
    // the whole warp iterates together (the group reductions shuffle across it)
    for (int64_t e0 = int64_t(gwarp) * GROUPS; e0 < n_evt; e0 += nwarps * GROUPS) {
        const int64_t e = e0 + lane / SUR_EVT_LANES;
        int i0 = 0, n = 0;
        bool ok = false;
        if (e < n_evt) {
            i0 = a.evt_off[e];
            const int i1 = a.evt_off[e + 1];
            ok = !(i0 < 0 || i1 < i0 || i1 > n_img);
            n = ok ? i1 - i0 : 0;
        }
        float bx, by;
        int cnt;
        sur_event_baseline(a.h, i0, n, sub, a.used, bx, by, cnt);
        if (e < n_evt && sub == 0) {
            a.base[e] = make_float2(bx, by);
            a.n_used[e] = ok ? cnt : -1;      // -1: malformed event
        }
        for (int k = sub; k < n; k += SUR_EVT_LANES) {
            const rta_hillas_t h = a.h[i0 + k];
            __nv_bfloat162 x[SUR_XPAD / 2];
            sur_image_features(h, a.img_tel[i0 + k], a.tel_cam, a.tel_xy, a.cam_code, a.n_tel, bx, by, x);
            uint4* xr = reinterpret_cast<uint4*>(a.X + int64_t(i0 + k) * SUR_XPAD);
            xr[0] = make_uint4(bf2_bits(x[0]), bf2_bits(x[1]), bf2_bits(x[2]), bf2_bits(x[3]));
            xr[1] = make_uint4(bf2_bits(x[4]), bf2_bits(x[5]), bf2_bits(x[6]), bf2_bits(x[7]));
        }
    }
}

// Sum of the split-K partials in a fixed order.
__global__ void k_reduce_splits(const float* ws, int splits, int64_t n, float* out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += ws[z * n + i];
        out[i] = s;
    }
}

// Column sums of a BF16 or FP32 matrix [rows x cols] (bias gradients), fixed order.
__global__ void k_colsum(const __nv_bfloat16* Xb, const float* Xf, const int64_t* rows_dev, int64_t rows, int cols,
                         float* out) {
    __shared__ float part[8][33];
    const int64_t R = rows_dev ? min(*rows_dev, rows) : rows;
    const int c = blockIdx.x * 32 + (threadIdx.x & 31);
    const int ty = threadIdx.x >> 5;
    float s = 0.f;
    if (c < cols)
        for (int64_t r = ty; r < R; r += 8) s += Xb ? __bfloat162float(Xb[r * cols + c]) : Xf[r * cols + c];
    part[ty][threadIdx.x & 31] = s;
    __syncthreads();
    if (ty == 0 && c < cols) {
        float t = 0.f;
        for (int k = 0; k < 8; ++k) t += part[k][threadIdx.x & 31];
        out[c] = t;
    }
}

// ------------------------------------------------------------------ pooling
// P[e] = [sum_used h2 / 40, sum_used h2 / max(1, n_used)] (BF16). One block per event, 128 threads (one per channel).
// The mean multiplies by the event's reciprocal count (RN(1 / n)), as the inference kernel does.
__global__ void __launch_bounds__(SUR_H) k_pool(const PoolArgs a) {
    const int64_t n_evt = a.n_evt_dev ? min(*a.n_evt_dev, a.n_evt) : a.n_evt;
    const int ch = threadIdx.x;
    for (int64_t e = blockIdx.x; e < n_evt; e += gridDim.x) {
        const int i0 = a.evt_off[e], i1 = a.evt_off[e + 1];
        float s = 0.f;
        int cnt = 0;
        if (a.n_used[e] >= 0)
            for (int i = i0; i < i1; ++i)
                if (a.used[i]) {
                    s += __bfloat162float(a.H2[int64_t(i) * SUR_H + ch]);
                    ++cnt;
                }
        a.P[e * 2 * SUR_H + ch] = __float2bfloat16(s * (1.f / SUR_POOL_DIV));
        a.P[e * 2 * SUR_H + SUR_H + ch] = __float2bfloat16(s * (1.f / fmaxf(1.f, float(cnt))));
    }
}

// dZ2[i] = used_i * (dP[e][:H] / 40 + dP[e][H:] / max(1, n)) * (H2[i] > 0), BF16.
__global__ void __launch_bounds__(SUR_H) k_pool_bwd(const PoolArgs a) {
    const int64_t n_evt = a.n_evt_dev ? min(*a.n_evt_dev, a.n_evt) : a.n_evt;
    const int ch = threadIdx.x;
    for (int64_t e = blockIdx.x; e < n_evt; e += gridDim.x) {
        const int i0 = a.evt_off[e], i1 = a.evt_off[e + 1];
        int cnt = 0;
        if (a.n_used[e] >= 0)
            for (int i = i0; i < i1; ++i) cnt += a.used[i] ? 1 : 0;
        const float g = __bfloat162float(a.dP[e * 2 * SUR_H + ch]) * (1.f / SUR_POOL_DIV) +
                        __bfloat162float(a.dP[e * 2 * SUR_H + SUR_H + ch]) * (1.f / fmaxf(1.f, float(cnt)));
        if (a.n_used[e] < 0) continue;
        for (int i = i0; i < i1; ++i) {
            const float h = __bfloat162float(a.H2[int64_t(i) * SUR_H + ch]);
            a.dZ2[int64_t(i) * SUR_H + ch] = __float2bfloat16(a.used[i] && h > 0.f ? g : 0.f);
        }
    }
}

// ------------------------------------------------------------------ output layer, loss, outputs
// Per-event loss terms and dL/dy (mean over n_evt events).
__global__ void k_loss(const LossArgs a) {
    const int64_t n_evt = a.n_evt_dev ? min(*a.n_evt_dev, a.n_evt) : a.n_evt;
    const float inv_n = 1.f / float(n_evt > 1 ? n_evt : 1);
    const float ids2 = 1.f / (SUR_DIR_SIGMA * SUR_DIR_SIGMA);
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < a.n_evt; e += int64_t(gridDim.x) * blockDim.x) {
        if (e >= n_evt) { a.lterm[e] = 0.f; continue; }
        const float* y = a.Y + e * 4;
        const float gam = a.is_gamma[e] ? 1.f : 0.f;
        const float2 b = a.base[e];
        const float2 src = a.src[e];
        const float r0 = y[0] - a.logE[e];
        const float r1 = y[1] - (src.x - b.x), r2 = y[2] - (src.y - b.y);
        const float sig = 1.f / (1.f + expf(-y[3]));
        const float bce = fmaxf(y[3], 0.f) + log1pf(expf(-fabsf(y[3]))) - gam * y[3];
        a.lterm[e] = gam * (r0 * r0 + (r1 * r1 + r2 * r2) * ids2) + bce;
        a.dY[e * 4 + 0] = 2.f * gam * r0 * inv_n;
        a.dY[e * 4 + 1] = 2.f * gam * r1 * ids2 * inv_n;
        a.dY[e * 4 + 2] = 2.f * gam * r2 * ids2 * inv_n;
        a.dY[e * 4 + 3] = (sig - gam) * inv_n;
    }
}

// Sum of the loss terms / n in a fixed order (one block).
__global__ void k_loss_sum(const float* lterm, int64_t n, const int64_t* n_dev, float* out) {
    __shared__ float part[256];
    const int64_t N = n_dev ? min(*n_dev, n) : n;
    float s = 0.f;
    for (int64_t i = threadIdx.x; i < N; i += 256) s += lterm[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0] / float(N > 1 ? N : 1);
}

// Backward of the output layer: dV2 = G^T dY (256 x 4, one block per 32 rows of V2),
// dG = (dY V2^T) * (G > 0) (BF16), dc2 = sum dY.
__global__ void k_head_bwd_dg(const HeadArgs a) {
    const int64_t n_evt = a.n_evt_dev ? min(*a.n_evt_dev, a.n_evt) : a.n_evt;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n_evt * SUR_G;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t e = i / SUR_G;
        const int k = int(i - e * SUR_G);
        const float g = __bfloat162float(a.G[i]);
        float d = 0.f;
#pragma unroll
        for (int o = 0; o < 4; ++o) d += a.dY[e * 4 + o] * __bfloat162float(a.V2b[k * 4 + o]);
        a.dG[i] = __float2bfloat16(g > 0.f ? d : 0.f);
    }
}

__global__ void k_head_bwd_dv2(const HeadArgs a) {
    // one block of 256 threads per (row k of V2): sum over events of G[e][k] * dY[e][o]
    __shared__ float part[4][256];
    const int64_t n_evt = a.n_evt_dev ? min(*a.n_evt_dev, a.n_evt) : a.n_evt;
    const int k = blockIdx.x;
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t e = threadIdx.x; e < n_evt; e += blockDim.x) {
        const float g = k < SUR_G ? __bfloat162float(a.G[e * SUR_G + k]) : 1.f;   // row SUR_G: bias (dc2)
#pragma unroll
        for (int o = 0; o < 4; ++o) s[o] += g * a.dY[e * 4 + o];
    }
#pragma unroll
    for (int o = 0; o < 4; ++o) part[o][threadIdx.x] = s[o];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int o = 0; o < 4; ++o) part[o][threadIdx.x] += part[o][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) {
        if (k < SUR_G) a.dV2[k * 4 + threadIdx.x] = part[threadIdx.x][0];
        else a.dc2[threadIdx.x] = part[threadIdx.x][0];
    }
}

// ------------------------------------------------------------------ Adam
// FP32 master weights; BF16 copies of the GEMM operands refreshed in the same pass.
__global__ void k_adam(const AdamArgs a) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < a.n; i += int64_t(gridDim.x) * blockDim.x) {
        const float g = a.g[i];
        const float m = a.b1 * a.m[i] + (1.f - a.b1) * g;
        const float v = a.b2 * a.v[i] + (1.f - a.b2) * g * g;
        a.m[i] = m;
        a.v[i] = v;
        const float mh = m / a.bc1, vh = v / a.bc2;
        const float p = a.p[i] - a.lr * mh / (sqrtf(vh) + a.eps);
        a.p[i] = p;
        a.pb[i] = __float2bfloat16(p);
    }
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_features(const FeatArgs& a, int grid, cudaStream_t s) {
    k_features<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_pool(const PoolArgs& a, int grid, bool bwd, cudaStream_t s) {
    if (bwd) k_pool_bwd<<<grid, SUR_H, 0, s>>>(a);
    else k_pool<<<grid, SUR_H, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_head_bwd(const HeadArgs& a, int grid, cudaStream_t s) {
    k_head_bwd_dg<<<grid, 256, 0, s>>>(a);
    k_head_bwd_dv2<<<SUR_G + 1, 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_loss(const LossArgs& a, int grid, float* d_loss, cudaStream_t s) {
    k_loss<<<grid, 256, 0, s>>>(a);
    if (d_loss) k_loss_sum<<<1, 256, 0, s>>>(a.lterm, a.n_evt, a.n_evt_dev, d_loss);
    return cudaGetLastError();
}
cudaError_t launch_colsum(const __nv_bfloat16* Xb, const float* Xf, const int64_t* rows_dev, int64_t rows, int cols,
                          float* out, cudaStream_t s) {
    k_colsum<<<(cols + 31) / 32, 256, 0, s>>>(Xb, Xf, rows_dev, rows, cols, out);
    return cudaGetLastError();
}
cudaError_t launch_reduce_splits(const float* ws, int splits, int64_t n, float* out, cudaStream_t s) {
    k_reduce_splits<<<int((n + 255) / 256), 256, 0, s>>>(ws, splits, n, out);
    return cudaGetLastError();
}
cudaError_t launch_adam(const AdamArgs& a, cudaStream_t s) {
    k_adam<<<int((a.n + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace rta
