// Launch-argument blocks and constants of the deep-sets surrogate kernels.
#pragma once

#include <cuda_bf16.h>

#include "rta_launch.cuh"

#define SUR_NF 12            // features per image
#define SUR_XPAD 16          // feature rows padded to 16 (one k-step of the tensor-core MMA)
#define SUR_H 128            // width of the per-telescope network
#define SUR_G 256            // width of the event network (and of the pooled vector)
#define SUR_POOL_DIV 40.f    // sum pooling divisor
#define SUR_DIR_SIGMA 0.1f   // direction scale of the loss (deg)
#define SUR_BASE_MIN_SIN 0.1f

namespace rta {

// Lanes per event of the per-event prologue (used images, baseline): four, so
// that 512 threads take a tile of 128 events at once and an event of 40 images
// takes ten steps per lane.
constexpr int SUR_EVT_LANES = 4;

// internal parameter layout (FP32 master copy and its BF16 twin), element offsets
constexpr int64_t OFF_W1 = 0;                                // [16 x 128], rows 12..15 zero
constexpr int64_t OFF_B1 = OFF_W1 + SUR_XPAD * SUR_H;
constexpr int64_t OFF_W2 = OFF_B1 + SUR_H;                   // [128 x 128]
constexpr int64_t OFF_B2 = OFF_W2 + SUR_H * SUR_H;
constexpr int64_t OFF_V1 = OFF_B2 + SUR_H;                   // [256 x 256]
constexpr int64_t OFF_C1 = OFF_V1 + SUR_G * SUR_G;
constexpr int64_t OFF_V2 = OFF_C1 + SUR_G;                   // [256 x 4]
constexpr int64_t OFF_C2 = OFF_V2 + SUR_G * 4;
constexpr int64_t N_PARAM_INTERNAL = OFF_C2 + 4;
// Weights of the inference kernels' tensor-core layers, transposed to N x K and
// laid out as canonical K-major core matrices (see rta_tc.cuh): W1 (128 x 16),
// W2 (128 x 128), V1 (256 x 256); then the padded output layer. Refreshed from
// the BF16 twin after every parameter change.
constexpr int64_t PK_W1T = 0;
constexpr int64_t PK_W2T = PK_W1T + SUR_H * SUR_XPAD;
constexpr int64_t PK_V1T = PK_W2T + SUR_H * SUR_H;
// V2 widened to 16 zero-padded columns, row-major [256 x 16]: the B operand of
// the training path's output layer.
constexpr int64_t PK_V2P = PK_V1T + SUR_G * SUR_G;
constexpr int64_t N_PK = PK_V2P + SUR_G * 16;
constexpr int64_t N_PARAM_PACKED = SUR_NF * SUR_H + SUR_H + SUR_H * SUR_H + SUR_H + SUR_G * SUR_G + SUR_G + SUR_G * 4 + 4;

struct FeatArgs {
    const rta_hillas_t* h;
    const int32_t* img_tel;
    const int32_t* evt_off;
    int64_t n_img, n_evt;
    const int64_t* n_img_dev;
    const int64_t* n_evt_dev;
    const int32_t* tel_cam;
    const float2* tel_xy;
    const float* cam_code;   // per camera id
    int n_tel;
    __nv_bfloat16* X;        // [n_img x 16]
    uint8_t* used;           // [n_img]
    float2* base;            // [n_evt]
    int32_t* n_used;         // [n_evt], -1 = malformed event
};

// Epilogues: ReLU(D + bias) as BF16; D where mask > 0 (the ReLU derivative) as
// BF16; D as BF16; D as the FP32 partial sum of a split reduction; the first
// n_store columns of D + bias as FP32.
enum { EPI_BIAS_RELU_BF16 = 0, EPI_MASK_BF16 = 1, EPI_F32_SPLIT = 2, EPI_BF16 = 3, EPI_F32_BIAS = 4 };

// D[M x N] = op(A) op(B): A stored [M x K] (K-major) or [K x M] (MN-major), B
// stored [N x K] (K-major) or [K x N] (MN-major); 16 <= N <= 256, N % 16 == 0;
// MN-major row counts and K-major K are multiples of 8; leading dimensions
// and bases 16-byte aligned.
struct GemmArgs {
    const __nv_bfloat16* A;
    const __nv_bfloat16* B;
    int64_t lda, ldb, ldc, ldmask;
    int64_t M, N, K;
    int epi;
    int n_store;             // EPI_F32_BIAS: columns written
    const float* bias;
    const __nv_bfloat16* mask;
    __nv_bfloat16* Cb;
    float* Cf;
    unsigned int* status;    // device status word (RTA_DEV_TIMEOUT)
};

struct PoolArgs {
    const int32_t* evt_off;
    int64_t n_evt;
    const int64_t* n_evt_dev;
    const uint8_t* used;
    const int32_t* n_used;
    const __nv_bfloat16* H2;   // [n_img x 128]
    __nv_bfloat16* P;          // [n_evt x 256]
    const __nv_bfloat16* dP;
    __nv_bfloat16* dZ2;
};

struct HeadArgs {
    int64_t n_evt;
    const int64_t* n_evt_dev;
    const __nv_bfloat16* G;    // [n_evt x 256]
    const __nv_bfloat16* V2b;  // [256 x 4]
    const float* c2;
    float* Y;                  // [n_evt x 4]
    const float* dY;
    __nv_bfloat16* dG;
    float* dV2;
    float* dc2;
};

struct LossArgs {
    int64_t n_evt;
    const int64_t* n_evt_dev;
    const float* Y;
    const float2* base;
    const float* logE;
    const float2* src;
    const uint8_t* is_gamma;
    float* lterm;
    float* dY;
};

struct OutArgs {
    float fallback_deg;        // learned offsets beyond this take the geometric direction
    rta_event_t* out;          // [n_evt]
    unsigned int* status;      // device status word (RTA_DEV_*)
};

// Inference: f carries the inputs and tables (its X/used/base/n_used are not
// touched).
struct InferArgs {
    FeatArgs f;
    const __nv_bfloat16* pb;   // BF16 parameter twin (internal layout)
    const float* p;            // FP32 master (biases)
    const __nv_bfloat16* pk;   // tensor-core weight layout (PK_*)
    int rows_aligned;          // f.h is 16-byte aligned: a tile's rows may arrive by bulk copy
    int settled;               // the event offsets, telescope ids and weights were written before the
                               // kernel this one follows on the stream started: they are read before
                               // the dependency wait (only the Hillas rows are the preceding kernel's)
    OutArgs o;
};

struct AdamArgs {
    int64_t n;
    float* p;
    float* m;
    float* v;
    const float* g;
    __nv_bfloat16* pb;
    float lr, b1, b2, eps, bc1, bc2;
};

cudaError_t launch_features(const FeatArgs& a, int grid, cudaStream_t s);
// Tensor-core GEMM (tcgen05): a_mn / b_mn give the operands' storage order;
// splits > 1 divides K (EPI_F32_SPLIT; gemm_tc_splits gives the number of
// partial sums actually written).
cudaError_t launch_gemm(const GemmArgs& g, bool a_mn, bool b_mn, int splits, int n_sm, cudaStream_t s);
int gemm_tc_splits(int64_t K, int splits);
cudaError_t launch_pool(const PoolArgs& a, int grid, bool bwd, cudaStream_t s);
cudaError_t launch_head_bwd(const HeadArgs& a, int grid, cudaStream_t s);
cudaError_t launch_loss(const LossArgs& a, int grid, float* d_loss, cudaStream_t s);
cudaError_t launch_colsum(const __nv_bfloat16* Xb, const float* Xf, const int64_t* rows_dev, int64_t rows, int cols,
                          float* out, cudaStream_t s);
cudaError_t launch_reduce_splits(const float* ws, int splits, int64_t n, float* out, cudaStream_t s);
cudaError_t launch_adam(const AdamArgs& a, cudaStream_t s);
// The whole inference in one persistent launch (one CTA per SM, n_sm of them at
// most, each with an equal share of the image rows; programmatic dependent
// launch), geometric fallback included.
cudaError_t launch_infer(const InferArgs& a, int n_sm, cudaStream_t s);
// BF16 twin -> tensor-core weight layout
cudaError_t launch_pack_tc(const __nv_bfloat16* pb, __nv_bfloat16* pk, cudaStream_t s);

}  // namespace rta
