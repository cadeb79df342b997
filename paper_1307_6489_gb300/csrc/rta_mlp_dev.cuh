// Device-side pieces of the deep-sets surrogate shared by the layer-by-layer
// kernels (training) and the fused inference kernel, so that both evaluate the
// same expressions in the same order and produce the same bits.
#pragma once

#include "rta_mlp.cuh"

namespace rta {

// D = A B + D on the tensor cores: one m16n8k16 tile, BF16 operands, FP32 accumulators.
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t*>(&v); }

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return uint32_t(__bfloat16_as_ushort(lo)) | (uint32_t(__bfloat16_as_ushort(hi)) << 16);
}

// B fragment of the output layer (256 x 4, BF16, row-major) for k-step ks,
// widened to n = 8 with zero columns.
__device__ __forceinline__ void head_b_fragment(const __nv_bfloat16* __restrict__ V2b, int ks, int gq, int tq,
                                                uint32_t (&b)[2]) {
    const int k = 16 * ks + 2 * tq;
    b[0] = gq < 4 ? pack_bf16(V2b[k * 4 + gq], V2b[(k + 1) * 4 + gq]) : 0u;
    b[1] = gq < 4 ? pack_bf16(V2b[(k + 8) * 4 + gq], V2b[(k + 9) * 4 + gq]) : 0u;
}

// An image takes part in the network when cleaning kept at least three pixels.
__device__ __forceinline__ bool sur_used(const rta_hillas_t& h) {
    return h.n_pix >= 3 && !(h.flags & (RTA_HF_EMPTY | RTA_HF_BAD_INPUT));
}

// Per-event prologue by a group of SUR_EVT_LANES lanes (sub = lane within the
// group) over images [i0, i1) (n = i1 - i0, 0 for a malformed event): number of
// used images, and the baseline direction -- the intersection of the axes of
// the two brightest used images (size descending, index ascending), or the
// size-weighted centroid when they are nearly parallel or only one image is
// used. Every lane of the warp must call it (the group reductions shuffle
// across the full warp); all lanes of a group return the same values.
// used_out (nullable) receives the per-image flags. Its quotients and angle
// functions are the fast forms (absolute errors below 1e-6 on these arguments,
// |angle| < pi), which the training and inference paths share.
__device__ __forceinline__ void sur_event_baseline(const rta_hillas_t* __restrict__ hrows, int i0, int n, int sub,
                                                   uint8_t* used_out, float& bx, float& by, int& n_used) {
    // Sizes are positive, so their bit patterns order like the values; the low
    // word prefers the lower index on ties.
    unsigned long long k1 = 0ull, k2 = 0ull;
    int cnt = 0;
    float sw = 0.f, swx = 0.f, swy = 0.f;
    for (int k = sub; k < n; k += SUR_EVT_LANES) {
        const rta_hillas_t h = hrows[i0 + k];
        const bool used = sur_used(h);
        if (used_out) used_out[i0 + k] = used;
        if (!used) continue;
        ++cnt;
        sw += h.size;
        swx += h.size * h.x;
        swy += h.size * h.y;
        const unsigned long long key =
            (static_cast<unsigned long long>(__float_as_uint(fmaxf(h.size, 0.f))) << 32) | (0xFFFFFFFFu - unsigned(k));
        if (key > k1) { k2 = k1; k1 = key; }
        else if (key > k2) { k2 = key; }
    }
#pragma unroll
    for (int o = SUR_EVT_LANES / 2; o > 0; o >>= 1) {
        const unsigned long long o1 = __shfl_xor_sync(0xffffffffu, k1, o);
        const unsigned long long o2 = __shfl_xor_sync(0xffffffffu, k2, o);
        // top two of {k1, k2, o1, o2} (all keys distinct or zero)
        const unsigned long long hi = k1 > o1 ? k1 : o1;
        const unsigned long long lo = k1 > o1 ? o1 : k1;
        const unsigned long long sec = k1 > o1 ? k2 : o2;
        k1 = hi;
        k2 = lo > sec ? lo : sec;
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
        swx += __shfl_xor_sync(0xffffffffu, swx, o);
        swy += __shfl_xor_sync(0xffffffffu, swy, o);
    }
    const int idx1 = k1 ? int(0xFFFFFFFFu - unsigned(k1 & 0xFFFFFFFFull)) : -1;
    const int idx2 = k2 ? int(0xFFFFFFFFu - unsigned(k2 & 0xFFFFFFFFull)) : -1;
    bx = 0.f;
    by = 0.f;
    bool done = false;
    if (cnt >= 2 && idx1 >= 0 && idx2 >= 0) {
        const rta_hillas_t A = hrows[i0 + idx1], B = hrows[i0 + idx2];
        const float s = __sinf(B.psi - A.psi);
        if (fabsf(s) >= SUR_BASE_MIN_SIN) {
            float sa, ca, sb, cb2;
            __sincosf(A.psi, &sa, &ca);
            __sincosf(B.psi, &sb, &cb2);
            const float k = __fdividef((B.x - A.x) * sb - (B.y - A.y) * cb2, s);
            bx = A.x + k * ca;
            by = A.y + k * sa;
            done = true;
        }
    }
    if (!done && cnt >= 1) {
        bx = __fdividef(swx, sw);
        by = __fdividef(swy, sw);
    }
    n_used = cnt;
}

// The 12 per-image features (padded to 16 with zeros), rounded to BF16 pairs:
// log10 size, offset of the centroid from the baseline (2), length, width,
// cos 2psi, sin 2psi, time gradient / 10, distance to the baseline, camera code,
// telescope position (km, 2).
__device__ __forceinline__ void sur_image_features(const rta_hillas_t& h, int tel, const int32_t* __restrict__ tel_cam,
                                                   const float2* __restrict__ tel_xy, const float* __restrict__ cam_code,
                                                   int n_tel, float bx, float by, __nv_bfloat162 (&out)[SUR_XPAD / 2]) {
    const bool tel_ok = tel >= 0 && tel < n_tel;
    const float2 txy = tel_ok ? tel_xy[tel] : make_float2(0.f, 0.f);
    const float code = tel_ok ? cam_code[tel_cam[tel]] : 0.f;
    const float dx = h.x - bx, dy = h.y - by;
    float s2, c2;
    __sincosf(2.f * h.psi, &s2, &c2);      // fast forms: their errors (~1e-6) are far below the BF16 rounding
    const float f[SUR_XPAD] = {__log10f(fmaxf(h.size, 1e-3f)), dx, dy, h.length, h.width, c2, s2,
                               h.time_grad * 0.1f, sqrtf(dx * dx + dy * dy), code, txy.x * 1e-3f,
                               txy.y * 1e-3f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < SUR_XPAD / 2; ++j) out[j] = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
}

}  // namespace rta
