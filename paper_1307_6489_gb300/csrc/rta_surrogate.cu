// Host side of the learned deep-sets surrogate: model state (FP32 master
// weights, their BF16 twin, Adam moments, gradients), the forward pass, one
// training step (forward, loss, backward, Adam) and inference with the
// geometric fallback. Every step runs in the kernels of k_mlp.cu / k_stereo.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "rta.h"
#include "rta_mlp.cuh"

namespace {

int sfail(int code, const char* fmt, ...) {
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    rta::set_last_error(msg);
    return code;
}

#define S_TRY(call)                                                                              \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return sfail(RTA_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

constexpr int64_t SPLIT_WS = int64_t(1) << 20;   // floats of split-K partial sums

}  // namespace

struct rta_model {
    rta_ctx* ctx = nullptr;
    int device = 0;
    float* p = nullptr;              // FP32 master weights (internal layout)
    __nv_bfloat16* pb = nullptr;     // BF16 twin
    __nv_bfloat16* pk = nullptr;     // tensor-core layout of the inference weights
    float* m = nullptr;
    float* v = nullptr;
    float* g = nullptr;
    float* cam_code = nullptr;       // per camera id
    float* split_ws = nullptr;
    int64_t step = 0;
    int n_sm = 1;
    // workspace
    int64_t cap_img = 0, cap_evt = 0;
    __nv_bfloat16 *X = nullptr, *H1 = nullptr, *H2 = nullptr, *dZ1 = nullptr, *dZ2 = nullptr;
    uint8_t* used = nullptr;
    float2* base = nullptr;
    int32_t* n_used = nullptr;
    __nv_bfloat16 *P = nullptr, *G = nullptr, *dG = nullptr, *dP = nullptr;
    float *Y = nullptr, *dY = nullptr, *lterm = nullptr;
};

namespace {

void free_ws(rta_model* md) {
    void* ptrs[] = {md->X, md->H1, md->H2, md->dZ1, md->dZ2, md->used, md->base, md->n_used, md->P, md->G, md->dG,
                    md->dP, md->Y, md->dY, md->lterm};
    for (void* q : ptrs) cudaFree(q);
    md->X = md->H1 = md->H2 = md->dZ1 = md->dZ2 = nullptr;
    md->used = nullptr;
    md->base = nullptr;
    md->n_used = nullptr;
    md->P = md->G = md->dG = md->dP = nullptr;
    md->Y = md->dY = md->lterm = nullptr;
    md->cap_img = md->cap_evt = 0;
}

// Grow the activation workspace to hold n_img images and n_evt events.
int reserve(rta_model* md, int64_t n_img, int64_t n_evt) {
    if (n_img <= md->cap_img && n_evt <= md->cap_evt) return RTA_OK;
    const int64_t ci = std::max<int64_t>(n_img, md->cap_img) + 1024, ce = std::max<int64_t>(n_evt, md->cap_evt) + 256;
    free_ws(md);
    auto al = [](void** p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
    bool ok = al((void**)&md->X, sizeof(__nv_bfloat16) * ci * SUR_XPAD) &&
              al((void**)&md->H1, sizeof(__nv_bfloat16) * ci * SUR_H) &&
              al((void**)&md->H2, sizeof(__nv_bfloat16) * ci * SUR_H) &&
              al((void**)&md->dZ1, sizeof(__nv_bfloat16) * ci * SUR_H) &&
              al((void**)&md->dZ2, sizeof(__nv_bfloat16) * ci * SUR_H) && al((void**)&md->used, ci) &&
              al((void**)&md->base, sizeof(float2) * ce) && al((void**)&md->n_used, sizeof(int32_t) * ce) &&
              al((void**)&md->P, sizeof(__nv_bfloat16) * ce * SUR_G) &&
              al((void**)&md->G, sizeof(__nv_bfloat16) * ce * SUR_G) &&
              al((void**)&md->dG, sizeof(__nv_bfloat16) * ce * SUR_G) &&
              al((void**)&md->dP, sizeof(__nv_bfloat16) * ce * SUR_G) && al((void**)&md->Y, sizeof(float) * ce * 4) &&
              al((void**)&md->dY, sizeof(float) * ce * 4) && al((void**)&md->lterm, sizeof(float) * ce);
    if (!ok) {
        free_ws(md);
        return sfail(RTA_E_NOMEM, "surrogate workspace allocation failed");
    }
    md->cap_img = ci;
    md->cap_evt = ce;
    return RTA_OK;
}

int blocks_for(int64_t n, int per) { return int(std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per, 65535))); }

// D = op(A) op(B) on the tensor cores. ta: A stored [K x M]; tb: B stored [N x K].
int gemm(rta_model* md, const __nv_bfloat16* A, int64_t lda, bool ta, const __nv_bfloat16* B, int64_t ldb, bool tb,
         int64_t M, int64_t N, int64_t K, int epi, const float* bias, const __nv_bfloat16* mask, int64_t ldmask,
         __nv_bfloat16* Cb, float* Cf, int64_t ldc, int splits, cudaStream_t s, int n_store = 0) {
    rta::GemmArgs g;
    g.A = A;
    g.B = B;
    g.lda = lda;
    g.ldb = ldb;
    g.ldc = ldc;
    g.ldmask = ldmask;
    g.M = M;
    g.N = N;
    g.K = K;
    g.epi = epi;
    g.n_store = n_store;
    g.bias = bias;
    g.mask = mask;
    g.Cb = Cb;
    g.Cf = Cf;
    g.status = rta::surrogate_ctx_status(md->ctx);
    S_TRY(rta::launch_gemm(g, ta, !tb, splits, md->n_sm, s));
    return RTA_OK;
}

// Weight gradient [M x N] = A^T B with the reduction split into K-ranges whose
// partial sums are added in a fixed order.
int weight_grad(rta_model* md, const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, int64_t M,
                int64_t N, int64_t K, float* out, cudaStream_t s) {
    const int64_t tiles = (M + 127) / 128;
    // about one work item per SM, each at least 8 chunks (512 rows) of the reduction
    int64_t splits = std::max<int64_t>(1, std::min<int64_t>(md->n_sm / tiles, (K + 511) / 512));
    splits = std::min<int64_t>(splits, SPLIT_WS / (M * N));
    const int used = rta::gemm_tc_splits(K, int(splits));
    int rc = gemm(md, A, lda, true, B, ldb, false, M, N, K, rta::EPI_F32_SPLIT, nullptr, nullptr, 0, nullptr,
                  md->split_ws, N, int(splits), s);
    if (rc) return rc;
    S_TRY(rta::launch_reduce_splits(md->split_ws, used, M * N, out, s));
    return RTA_OK;
}

// Argument checks of a batch; with_workspace: also grow the layer-by-layer
// workspace to the batch (the training path and the raw forward pass need it,
// the fused inference kernel does not).
int check_batch(rta_model* md, const rta_hillas_t* d_h, const int32_t* d_img_tel, int64_t n_img,
                const int32_t* d_evt_off, int64_t n_evt, bool with_workspace = true) {
    if (!md) return sfail(RTA_E_INVALID, "model is NULL");
    if (cudaSetDevice(md->device) != cudaSuccess) return sfail(RTA_E_CUDA, "cudaSetDevice failed");
    if (n_img < 0 || n_evt < 0 || n_img > (int64_t(1) << 30) || n_evt > (int64_t(1) << 30))
        return sfail(RTA_E_INVALID, "batch size out of range");
    if (n_evt > 0 && (!d_evt_off || (n_img > 0 && (!d_h || !d_img_tel)))) return sfail(RTA_E_INVALID, "NULL pointer");
    return with_workspace ? reserve(md, std::max<int64_t>(n_img, 1), std::max<int64_t>(n_evt, 1)) : RTA_OK;
}

int forward(rta_model* md, const rta_hillas_t* d_h, const int32_t* d_img_tel, int64_t n_img, const int32_t* d_evt_off,
            int64_t n_evt, cudaStream_t s) {
    rta::FeatArgs f;
    f.h = d_h;
    f.img_tel = d_img_tel;
    f.evt_off = d_evt_off;
    f.n_img = n_img;
    f.n_evt = n_evt;
    f.n_img_dev = nullptr;
    f.n_evt_dev = nullptr;
    int rc = rta::surrogate_ctx_tables(md->ctx, &f.tel_cam, &f.tel_xy, &f.n_tel, nullptr);
    if (rc) return rc;
    f.cam_code = md->cam_code;
    f.X = md->X;
    f.used = md->used;
    f.base = md->base;
    f.n_used = md->n_used;
    if (n_img > 0) S_TRY(cudaMemsetAsync(md->X, 0, sizeof(__nv_bfloat16) * n_img * SUR_XPAD, s));
    S_TRY(rta::launch_features(f, blocks_for(n_evt, 256 / rta::SUR_EVT_LANES), s));
    const __nv_bfloat16* pb = md->pb;
    if (n_img > 0) {
        if ((rc = gemm(md, md->X, SUR_XPAD, false, pb + rta::OFF_W1, SUR_H, false, n_img, SUR_H, SUR_XPAD,
                       rta::EPI_BIAS_RELU_BF16, md->p + rta::OFF_B1, nullptr, 0, md->H1, nullptr, SUR_H, 1, s)))
            return rc;
        if ((rc = gemm(md, md->H1, SUR_H, false, pb + rta::OFF_W2, SUR_H, false, n_img, SUR_H, SUR_H,
                       rta::EPI_BIAS_RELU_BF16, md->p + rta::OFF_B2, nullptr, 0, md->H2, nullptr, SUR_H, 1, s)))
            return rc;
    }
    rta::PoolArgs pa = {};
    pa.evt_off = d_evt_off;
    pa.n_evt = n_evt;
    pa.used = md->used;
    pa.n_used = md->n_used;
    pa.H2 = md->H2;
    pa.P = md->P;
    S_TRY(rta::launch_pool(pa, blocks_for(n_evt, 1), false, s));
    if ((rc = gemm(md, md->P, SUR_G, false, pb + rta::OFF_V1, SUR_G, false, n_evt, SUR_G, SUR_G, rta::EPI_BIAS_RELU_BF16,
                   md->p + rta::OFF_C1, nullptr, 0, md->G, nullptr, SUR_G, 1, s)))
        return rc;
    // output layer: Y = G V2 + c2 (V2 widened to 16 zero columns; 4 stored)
    if ((rc = gemm(md, md->G, SUR_G, false, md->pk + rta::PK_V2P, 16, false, n_evt, 16, SUR_G, rta::EPI_F32_BIAS,
                   md->p + rta::OFF_C2, nullptr, 0, nullptr, md->Y, 4, 1, s, 4)))
        return rc;
    return RTA_OK;
}

// Internal <-> packed parameter layout (the packed one drops W1's padding rows).
struct Seg {
    int64_t off_int, off_pack, rows, cols, pad_rows;
};

std::vector<Seg> segments() {
    std::vector<Seg> v;
    int64_t pk = 0;
    auto add = [&](int64_t off, int64_t rows, int64_t cols, int64_t pad_rows) {
        v.push_back({off, pk, rows, cols, pad_rows});
        pk += rows * cols;
    };
    add(rta::OFF_W1, SUR_NF, SUR_H, SUR_XPAD);
    add(rta::OFF_B1, 1, SUR_H, 1);
    add(rta::OFF_W2, SUR_H, SUR_H, SUR_H);
    add(rta::OFF_B2, 1, SUR_H, 1);
    add(rta::OFF_V1, SUR_G, SUR_G, SUR_G);
    add(rta::OFF_C1, 1, SUR_G, 1);
    add(rta::OFF_V2, SUR_G, 4, SUR_G);
    add(rta::OFF_C2, 1, 4, 1);
    return v;
}

uint16_t to_bf16_bits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    return uint16_t((u + 0x7FFFu + lsb) >> 16);
}

int upload_params(rta_model* md, const std::vector<float>& internal) {
    // work of the model still running on any stream (a training step, an inference)
    // finishes before its weights are replaced
    S_TRY(cudaDeviceSynchronize());
    std::vector<uint16_t> b(internal.size());
    for (size_t i = 0; i < internal.size(); ++i) b[i] = to_bf16_bits(internal[i]);
    S_TRY(cudaMemcpy(md->p, internal.data(), sizeof(float) * internal.size(), cudaMemcpyHostToDevice));
    S_TRY(cudaMemcpy(md->pb, b.data(), sizeof(uint16_t) * b.size(), cudaMemcpyHostToDevice));
    S_TRY(rta::launch_pack_tc(md->pb, md->pk, 0));
    S_TRY(cudaDeviceSynchronize());
    return RTA_OK;
}

}  // namespace

// The inference launch; settled: the kernel before it on the stream is the image kernel, so
// the event offsets, telescope ids and weights may be read before its dependency wait.
static int infer(rta_model* md, const rta_hillas_t* d_h, const int32_t* d_img_tel, int64_t n_img, const int32_t* d_evt_off,
          int64_t n_evt, float fallback_deg, rta_event_t* d_out, cudaStream_t s, bool settled) {
    int rc = check_batch(md, d_h, d_img_tel, n_img, d_evt_off, n_evt, false);
    if (rc) return rc;
    if (n_evt == 0) return RTA_OK;
    if (!d_out) return sfail(RTA_E_INVALID, "NULL output");
    if (!(fallback_deg > 0.f)) return sfail(RTA_E_INVALID, "fallback bound must be > 0");
    rta::InferArgs ia = {};
    ia.f.h = d_h;
    ia.f.img_tel = d_img_tel;
    ia.f.evt_off = d_evt_off;
    ia.f.n_img = n_img;
    ia.f.n_evt = n_evt;
    if ((rc = rta::surrogate_ctx_tables(md->ctx, &ia.f.tel_cam, &ia.f.tel_xy, &ia.f.n_tel, nullptr))) return rc;
    ia.f.cam_code = md->cam_code;
    ia.pb = md->pb;
    ia.p = md->p;
    ia.pk = md->pk;
    ia.rows_aligned = (reinterpret_cast<uintptr_t>(d_h) & 15u) == 0;
    ia.settled = settled ? 1 : 0;
    ia.o.fallback_deg = fallback_deg;
    ia.o.out = d_out;
    ia.o.status = rta::surrogate_ctx_status(md->ctx);
    S_TRY(rta::launch_infer(ia, md->n_sm, s));
    return RTA_OK;
}

// The serving loop's inference on a batch gathered on the device: capacities max_img and
// max_evt, actual counts in *d_n_img and *d_n_evt; the counts and tables were written before
// the image kernel that precedes this launch started (read before the dependency wait).
int rta::serve_infer(rta_model* md, const rta_hillas_t* d_h, const int32_t* d_img_tel, int64_t max_img,
                     const int32_t* d_evt_off, int64_t max_evt, const int64_t* d_n_img, const int64_t* d_n_evt,
                     float fallback_deg, rta_event_t* d_out, cudaStream_t s) {
    if (!md || !d_n_img || !d_n_evt || !d_out || max_img < 1 || max_evt < 1) return sfail(RTA_E_INVALID, "bad batch");
    rta::InferArgs ia = {};
    ia.f.h = d_h;
    ia.f.img_tel = d_img_tel;
    ia.f.evt_off = d_evt_off;
    ia.f.n_img = max_img;
    ia.f.n_evt = max_evt;
    ia.f.n_img_dev = d_n_img;
    ia.f.n_evt_dev = d_n_evt;
    int rc = rta::surrogate_ctx_tables(md->ctx, &ia.f.tel_cam, &ia.f.tel_xy, &ia.f.n_tel, nullptr);
    if (rc) return rc;
    ia.f.cam_code = md->cam_code;
    ia.pb = md->pb;
    ia.p = md->p;
    ia.pk = md->pk;
    ia.rows_aligned = (reinterpret_cast<uintptr_t>(d_h) & 15u) == 0;
    ia.settled = 1;
    ia.o.fallback_deg = fallback_deg;
    ia.o.out = d_out;
    ia.o.status = rta::surrogate_ctx_status(md->ctx);
    S_TRY(rta::launch_infer(ia, md->n_sm, s));
    return RTA_OK;
}

extern "C" {

int rta_surrogate_num_params(void) { return int(rta::N_PARAM_PACKED); }

int rta_surrogate_create(rta_ctx* ctx, uint64_t seed, const float* h_cam_code, rta_model** out) {
    if (!ctx || !out) return sfail(RTA_E_INVALID, "NULL argument");
    int dev = 0;
    int rc = rta::surrogate_ctx_tables(ctx, nullptr, nullptr, nullptr, &dev);
    if (rc) return rc;
    S_TRY(cudaSetDevice(dev));
    rta_model* md = new rta_model();
    md->ctx = ctx;
    md->device = dev;
    if (cudaDeviceGetAttribute(&md->n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || md->n_sm < 1)
        md->n_sm = 1;
    const size_t n = rta::N_PARAM_INTERNAL;
    bool ok = cudaMalloc(&md->p, n * 4) == cudaSuccess && cudaMalloc(&md->pb, n * 2) == cudaSuccess &&
              cudaMalloc(&md->pk, sizeof(__nv_bfloat16) * rta::N_PK) == cudaSuccess &&
              cudaMalloc(&md->m, n * 4) == cudaSuccess && cudaMalloc(&md->v, n * 4) == cudaSuccess &&
              cudaMalloc(&md->g, n * 4) == cudaSuccess && cudaMalloc(&md->cam_code, 4 * RTA_MAX_CAMS) == cudaSuccess &&
              cudaMalloc(&md->split_ws, sizeof(float) * SPLIT_WS) == cudaSuccess;
    if (!ok) {
        rta_surrogate_destroy(md);
        return sfail(RTA_E_NOMEM, "model allocation failed");
    }
    cudaMemset(md->m, 0, n * 4);
    cudaMemset(md->v, 0, n * 4);
    cudaMemset(md->g, 0, n * 4);
    float codes[RTA_MAX_CAMS] = {};
    if (h_cam_code) memcpy(codes, h_cam_code, sizeof codes);
    cudaMemcpy(md->cam_code, codes, sizeof codes, cudaMemcpyHostToDevice);
    // He-normal weights, zero biases (splitmix64 + Box-Muller; a model's own start)
    std::vector<float> w(n, 0.f);
    uint64_t st = seed ^ 0x9E3779B97F4A7C15ull;
    auto next = [&]() {
        st += 0x9E3779B97F4A7C15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto normal = [&]() {
        const double u1 = (double(next() >> 11) + 0.5) / 9007199254740992.0;
        const double u2 = (double(next() >> 11) + 0.5) / 9007199254740992.0;
        return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    };
    for (const Seg& sg : segments()) {
        if (sg.rows == 1) continue;   // biases start at zero
        const double sd = sqrt(2.0 / double(sg.rows));
        for (int64_t r = 0; r < sg.rows; ++r)
            for (int64_t c = 0; c < sg.cols; ++c) w[sg.off_int + r * sg.cols + c] = float(sd * normal());
    }
    if ((rc = upload_params(md, w))) {
        rta_surrogate_destroy(md);
        return rc;
    }
    *out = md;
    return RTA_OK;
}

int rta_surrogate_destroy(rta_model* md) {
    if (!md) return RTA_OK;
    cudaSetDevice(md->device);
    cudaDeviceSynchronize();
    free_ws(md);
    cudaFree(md->p);
    cudaFree(md->pb);
    cudaFree(md->pk);
    cudaFree(md->m);
    cudaFree(md->v);
    cudaFree(md->g);
    cudaFree(md->cam_code);
    cudaFree(md->split_ws);
    delete md;
    return RTA_OK;
}

int rta_surrogate_set_params(rta_model* md, const float* h_params) {
    if (!md || !h_params) return sfail(RTA_E_INVALID, "NULL argument");
    S_TRY(cudaSetDevice(md->device));
    std::vector<float> w(rta::N_PARAM_INTERNAL, 0.f);
    for (const Seg& sg : segments())
        for (int64_t r = 0; r < sg.rows; ++r)
            for (int64_t c = 0; c < sg.cols; ++c) w[sg.off_int + r * sg.cols + c] = h_params[sg.off_pack + r * sg.cols + c];
    return upload_params(md, w);
}

int rta_surrogate_get_params(rta_model* md, int which, float* h_out) {
    if (!md || !h_out || which < 0 || which > 3) return sfail(RTA_E_INVALID, "bad argument");
    S_TRY(cudaSetDevice(md->device));
    S_TRY(cudaDeviceSynchronize());
    const float* src = which == 0 ? md->p : which == 1 ? md->g : which == 2 ? md->m : md->v;
    std::vector<float> w(rta::N_PARAM_INTERNAL);
    S_TRY(cudaMemcpy(w.data(), src, sizeof(float) * w.size(), cudaMemcpyDeviceToHost));
    for (const Seg& sg : segments())
        for (int64_t r = 0; r < sg.rows; ++r)
            for (int64_t c = 0; c < sg.cols; ++c) h_out[sg.off_pack + r * sg.cols + c] = w[sg.off_int + r * sg.cols + c];
    return RTA_OK;
}

int rta_surrogate_get_state(rta_model* md, float* h_params, float* h_m, float* h_v, int64_t* step) {
    if (!md || !step) return sfail(RTA_E_INVALID, "NULL argument");
    int rc;
    if (h_params && (rc = rta_surrogate_get_params(md, 0, h_params))) return rc;
    if (h_m && (rc = rta_surrogate_get_params(md, 2, h_m))) return rc;
    if (h_v && (rc = rta_surrogate_get_params(md, 3, h_v))) return rc;
    *step = md->step;
    return RTA_OK;
}

int rta_surrogate_set_state(rta_model* md, const float* h_params, const float* h_m, const float* h_v, int64_t step) {
    if (!md || !h_params || !h_m || !h_v || step < 0) return sfail(RTA_E_INVALID, "bad argument");
    int rc = rta_surrogate_set_params(md, h_params);
    if (rc) return rc;
    std::vector<float> m(rta::N_PARAM_INTERNAL, 0.f), v(rta::N_PARAM_INTERNAL, 0.f);
    for (const Seg& sg : segments())
        for (int64_t r = 0; r < sg.rows; ++r)
            for (int64_t c = 0; c < sg.cols; ++c) {
                m[sg.off_int + r * sg.cols + c] = h_m[sg.off_pack + r * sg.cols + c];
                v[sg.off_int + r * sg.cols + c] = h_v[sg.off_pack + r * sg.cols + c];
            }
    S_TRY(cudaMemcpy(md->m, m.data(), sizeof(float) * m.size(), cudaMemcpyHostToDevice));
    S_TRY(cudaMemcpy(md->v, v.data(), sizeof(float) * v.size(), cudaMemcpyHostToDevice));
    md->step = step;
    return RTA_OK;
}

int rta_surrogate_forward(rta_model* md, const rta_hillas_t* d_h, const int32_t* d_img_tel, int64_t n_img,
                          const int32_t* d_evt_off, int64_t n_evt, float* d_y, float* d_base, void* stream) {
    int rc = check_batch(md, d_h, d_img_tel, n_img, d_evt_off, n_evt);
    if (rc) return rc;
    if (n_evt == 0) return RTA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = forward(md, d_h, d_img_tel, n_img, d_evt_off, n_evt, s))) return rc;
    if (d_y) S_TRY(cudaMemcpyAsync(d_y, md->Y, sizeof(float) * 4 * n_evt, cudaMemcpyDeviceToDevice, s));
    if (d_base) S_TRY(cudaMemcpyAsync(d_base, md->base, sizeof(float2) * n_evt, cudaMemcpyDeviceToDevice, s));
    return RTA_OK;
}

int rta_surrogate_train_step(rta_model* md, const rta_hillas_t* d_h, const int32_t* d_img_tel, int64_t n_img,
                             const int32_t* d_evt_off, int64_t n_evt, const float* d_log_energy, const float* d_src_xy,
                             const uint8_t* d_is_gamma, float lr, int apply_update, float* d_loss, void* stream) {
    int rc = check_batch(md, d_h, d_img_tel, n_img, d_evt_off, n_evt);
    if (rc) return rc;
    if (n_evt == 0) return RTA_OK;
    if (!d_log_energy || !d_src_xy || !d_is_gamma) return sfail(RTA_E_INVALID, "NULL label pointer");
    if (!(lr >= 0.f)) return sfail(RTA_E_INVALID, "learning rate must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = forward(md, d_h, d_img_tel, n_img, d_evt_off, n_evt, s))) return rc;
    rta::LossArgs la = {};
    la.n_evt = n_evt;
    la.Y = md->Y;
    la.base = md->base;
    la.logE = d_log_energy;
    la.src = reinterpret_cast<const float2*>(d_src_xy);
    la.is_gamma = d_is_gamma;
    la.lterm = md->lterm;
    la.dY = md->dY;
    S_TRY(rta::launch_loss(la, blocks_for(n_evt, 256), d_loss, s));
    // output layer
    rta::HeadArgs ha = {};
    ha.n_evt = n_evt;
    ha.G = md->G;
    ha.V2b = md->pb + rta::OFF_V2;
    ha.dY = md->dY;
    ha.dG = md->dG;
    ha.dV2 = md->g + rta::OFF_V2;
    ha.dc2 = md->g + rta::OFF_C2;
    S_TRY(rta::launch_head_bwd(ha, blocks_for(n_evt * SUR_G, 256), s));
    // event network
    if ((rc = weight_grad(md, md->P, SUR_G, md->dG, SUR_G, SUR_G, SUR_G, n_evt, md->g + rta::OFF_V1, s))) return rc;
    S_TRY(rta::launch_colsum(md->dG, nullptr, nullptr, n_evt, SUR_G, md->g + rta::OFF_C1, s));
    if ((rc = gemm(md, md->dG, SUR_G, false, md->pb + rta::OFF_V1, SUR_G, true, n_evt, SUR_G, SUR_G, rta::EPI_BF16, nullptr,
                   nullptr, 0, md->dP, nullptr, SUR_G, 1, s)))
        return rc;
    // pooling
    rta::PoolArgs pa = {};
    pa.evt_off = d_evt_off;
    pa.n_evt = n_evt;
    pa.used = md->used;
    pa.n_used = md->n_used;
    pa.H2 = md->H2;
    pa.dP = md->dP;
    pa.dZ2 = md->dZ2;
    if (n_img > 0) S_TRY(cudaMemsetAsync(md->dZ2, 0, sizeof(__nv_bfloat16) * n_img * SUR_H, s));
    S_TRY(rta::launch_pool(pa, blocks_for(n_evt, 1), true, s));
    // per-telescope network
    if (n_img > 0) {
        if ((rc = weight_grad(md, md->H1, SUR_H, md->dZ2, SUR_H, SUR_H, SUR_H, n_img, md->g + rta::OFF_W2, s)))
            return rc;
        S_TRY(rta::launch_colsum(md->dZ2, nullptr, nullptr, n_img, SUR_H, md->g + rta::OFF_B2, s));
        if ((rc = gemm(md, md->dZ2, SUR_H, false, md->pb + rta::OFF_W2, SUR_H, true, n_img, SUR_H, SUR_H,
                       rta::EPI_MASK_BF16, nullptr, md->H1, SUR_H, md->dZ1, nullptr, SUR_H, 1, s)))
            return rc;
        if ((rc = weight_grad(md, md->X, SUR_XPAD, md->dZ1, SUR_H, SUR_XPAD, SUR_H, n_img, md->g + rta::OFF_W1, s)))
            return rc;
        S_TRY(rta::launch_colsum(md->dZ1, nullptr, nullptr, n_img, SUR_H, md->g + rta::OFF_B1, s));
    } else {
        S_TRY(cudaMemsetAsync(md->g, 0, sizeof(float) * rta::OFF_V1, s));
    }
    if (apply_update) {
        ++md->step;
        rta::AdamArgs ad;
        ad.n = rta::N_PARAM_INTERNAL;
        ad.p = md->p;
        ad.m = md->m;
        ad.v = md->v;
        ad.g = md->g;
        ad.pb = md->pb;
        ad.lr = lr;
        ad.b1 = 0.9f;
        ad.b2 = 0.999f;
        ad.eps = 1e-8f;
        ad.bc1 = float(1.0 - pow(0.9, double(md->step)));
        ad.bc2 = float(1.0 - pow(0.999, double(md->step)));
        S_TRY(rta::launch_adam(ad, s));
        S_TRY(rta::launch_pack_tc(md->pb, md->pk, s));
    }
    return RTA_OK;
}

int rta_surrogate_infer(rta_model* md, const rta_hillas_t* d_h, const int32_t* d_img_tel, int64_t n_img,
                        const int32_t* d_evt_off, int64_t n_evt, float fallback_deg, rta_event_t* d_out, void* stream) {
    return infer(md, d_h, d_img_tel, n_img, d_evt_off, n_evt, fallback_deg, d_out, (cudaStream_t)stream, false);
}

int rta_reconstruct_learned(rta_model* md, const uint16_t* d_wave, int64_t n_wave, const int64_t* d_wave_off,
                            const int32_t* d_img_tel, int64_t n_img, const int32_t* d_evt_off, int64_t n_evt,
                            int window_mode, int start, int W, float t_hi, float t_lo, int core_needs_neighbour,
                            float fallback_deg, rta_hillas_t* d_hillas, rta_event_t* d_events, void* stream) {
    int rc = check_batch(md, d_hillas, d_img_tel, n_img, d_evt_off, n_evt, false);
    if (rc) return rc;
    if (n_evt > 0 && !d_events) return sfail(RTA_E_INVALID, "NULL output");
    if (!(fallback_deg > 0.f)) return sfail(RTA_E_INVALID, "fallback bound must be > 0");
    rc = rta_image_chain(md->ctx, d_wave, n_wave, d_wave_off, d_img_tel, n_img, window_mode, start, W, t_hi, t_lo,
                         core_needs_neighbour, d_hillas, stream);
    if (rc) return rc;
    // with no image the image kernel is not launched, and the kernel before the inference is
    // unknown: the inputs are then read after the dependency wait
    return infer(md, d_hillas, d_img_tel, n_img, d_evt_off, n_evt, fallback_deg, d_events, (cudaStream_t)stream,
                 n_img > 0);
}

}  // extern "C"
