// Device pieces of the stereo Hillas intersection (direction and core
// reconstruction, Sec. 4.1) shared by the stereo kernel and the learned
// reconstruction's geometric fallback, so that both give the same bits for an
// event: image staging, the pair sums of G lanes, and the combination of the
// lanes into the event's row.
//
// The weighted intersection is accumulated without dividing by
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
#pragma once

#include "rta_launch.cuh"

namespace rta {

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

// (a.hi + a.lo) / (b.hi + b.lo) in FP32: a first quotient from the correctly
// rounded reciprocal of b.hi, then one correction step with the exact residual
// of that quotient (within about one unit in the last place of the result).
__device__ __forceinline__ float dw_div(DW a, DW b) {
    const float rb = __frcp_rn(b.hi);
    const float q = __fmul_rn(a.hi, rb);
    const float p = __fmul_rn(q, b.hi);
    const float pe = __fmaf_rn(q, b.hi, -p);            // q * b.hi = p + pe exactly
    const float r = __fsub_rn(__fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo), __fmul_rn(q, b.lo));
    return __fmaf_rn(r, rb, q);
}

// One image staged for the pair loop from its Hillas row and telescope id: its
// direction cosines, 1 - W/L (0 when not used for stereo) and telescope
// position. Returns whether it is used; an unknown telescope sets the status bit.
__device__ __forceinline__ int stereo_stage(const rta_hillas_t& hh, int tel, int n_tel, const float2* tel_xy,
                                            unsigned int* status, StereoImg* dst) {
    const bool tel_ok = tel >= 0 && tel < n_tel;
    const bool used = tel_ok && hh.n_pix >= 3 && !(hh.flags & (RTA_HF_EMPTY | RTA_HF_BAD_INPUT));
    if (!tel_ok) atomicOr(status, RTA_DEV_BAD_IMAGE);
    StereoImg v;
    float sp, cp;
    sincosf(hh.psi, &sp, &cp);
    v.x = hh.x;
    v.y = hh.y;
    v.c = cp;
    v.s = sp;
    v.psi = hh.psi;
    v.f = used ? 1.f - __fdividef(hh.width, hh.length) : 0.f;
    const float2 t = tel_ok ? tel_xy[tel] : make_float2(0.f, 0.f);
    v.tx = t.x;
    v.ty = t.y;
    v.size = hh.size;
    v.used = used;
    v.pad0 = v.pad1 = 0.f;
    *dst = v;
    return used;
}

// The weighted terms of one image pair (F |s|, then the direction and core
// numerators); false when either image is unused or the axes are parallel
// (|s| < 1e-6). Every multiply-add is written out (fmaf) or explicitly rounded,
// so no kernel that shares this code contracts it differently; the weight's
// quotient is the fast division (2 ulp: a relative 1e-7 on a weight).
__device__ __forceinline__ bool pair_term(const StereoImg& A, const StereoImg& B, float (&t)[5]) {
    const float kPiHi = 3.14159274101257324f;          // RN(pi), above pi
    const float kPiLo = -8.74227765734758577e-8f;      // pi - kPiHi
    const float kHalfPi = 1.57079637050628662f;
    if (!A.used || !B.used) return false;
    DW d = two_sum(B.psi, -A.psi);                      // psi_j - psi_i, exactly
    float sgn = 1.f;
    if (d.hi > kHalfPi) {
        d = {__fsub_rn(d.hi, kPiHi), __fsub_rn(d.lo, kPiLo)};   // d.hi - kPiHi is exact (Sterbenz)
        sgn = -1.f;
    } else if (d.hi <= -kHalfPi) {
        d = {__fadd_rn(d.hi, kPiHi), __fadd_rn(d.lo, kPiLo)};
        sgn = -1.f;
    }
    const float s = sgn * sinf(__fadd_rn(d.hi, d.lo));  // sin(psi_j - psi_i), relatively accurate
    if (fabsf(s) < 1e-6f) return false;
    const float F = __fmul_rn(__fmul_rn(__fdividef(__fmul_rn(A.size, B.size), __fadd_rn(A.size, B.size)), A.f), B.f);
    const float as = fabsf(s);
    const float sg = s > 0.f ? 1.f : -1.f;
    // cross(c_j - c_i, u_j) in the sky and on the ground, signed by s
    const float cr = sg * __fmaf_rn(__fsub_rn(B.x, A.x), B.s, -__fmul_rn(__fsub_rn(B.y, A.y), B.c));
    const float crg = sg * __fmaf_rn(__fsub_rn(B.tx, A.tx), B.s, -__fmul_rn(__fsub_rn(B.ty, A.ty), B.c));
    t[0] = __fmul_rn(F, as);
    t[1] = __fmul_rn(F, __fmaf_rn(as, A.x, __fmul_rn(cr, A.c)));
    t[2] = __fmul_rn(F, __fmaf_rn(as, A.y, __fmul_rn(cr, A.s)));
    t[3] = __fmul_rn(F, __fmaf_rn(as, A.tx, __fmul_rn(crg, A.c)));
    t[4] = __fmul_rn(F, __fmaf_rn(as, A.ty, __fmul_rn(crg, A.s)));
    return true;
}

// Pair sums of one event of m staged images, shared by G lanes (this one is
// lane `sub`): pair p of the row-major upper triangle (i, j), i < j, goes to
// lane p mod G, walked incrementally G pairs at a time. Two pairs are formed
// per iteration (their terms are independent, so their latencies overlap) and
// added in pair order, the order of a one-at-a-time walk.
template <int G>
__device__ __forceinline__ int pair_sums(const StereoImg* im, int m, int sub, CSum (&acc)[5]) {
    int npair = 0;
    const int T = m * (m - 1) / 2;
    int i = 0, j = 1 + sub;
    while (j >= m && i < m - 1) { ++i; j = j - m + i + 1; }
    for (int p = sub; p < T; p += 2 * G) {
        const int i1 = i, j1 = j;
        j += G;
        while (j >= m && i < m - 1) { ++i; j = j - m + i + 1; }
        const bool second = p + G < T;
        const int i2 = second ? i : i1, j2 = second ? j : j1;
        if (second) {
            j += G;
            while (j >= m && i < m - 1) { ++i; j = j - m + i + 1; }
        }
        float t1[5], t2[5];
        const bool ok1 = pair_term(im[i1], im[j1], t1);
        const bool ok2 = second && pair_term(im[i2], im[j2], t2);
        if (ok1) {
#pragma unroll
            for (int k = 0; k < 5; ++k) acc[k].add(t1[k]);
            ++npair;
        }
        if (ok2) {
#pragma unroll
            for (int k = 0; k < 5; ++k) acc[k].add(t2[k]);
            ++npair;
        }
    }
    return npair;
}

// The event's row from its summed terms.
__device__ __forceinline__ rta_stereo_t stereo_row(const DW (&tot)[5], int npair, int nvalid) {
    rta_stereo_t r = {};
    r.n_valid = nvalid;
    if (npair > 0 && tot[0].hi + tot[0].lo > 0.f) {
        r.dir_x = dw_div(tot[1], tot[0]);
        r.dir_y = dw_div(tot[2], tot[0]);
        r.core_x = dw_div(tot[3], tot[0]);
        r.core_y = dw_div(tot[4], tot[0]);
    } else {
        r.flags = RTA_SF_INVALID;
    }
    return r;
}

// Combine the G lanes of each aligned G-lane group (all 32 lanes take part) and
// form the event's row; every lane of a group returns it.
template <int G>
__device__ __forceinline__ rta_stereo_t group_result(CSum (&acc)[5], int npair, int nvalid) {
    DW tot[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        DW v = two_sum(acc[k].s, acc[k].c);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const DW w = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
            v = dw_add(v, w);
        }
        tot[k] = v;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        npair += __shfl_xor_sync(0xffffffffu, npair, o);
        nvalid += __shfl_xor_sync(0xffffffffu, nvalid, o);
    }
    return stereo_row(tot, npair, nvalid);
}

// Events of more than STEREO_WARP_M images take a whole CTA: their pairs are
// spread over every thread, which cuts the longest chains (an event of 40
// images has 780 pairs) by the CTA's width. Up to STEREO_SMALL_M images take
// eight lanes, up to STEREO_WARP_M a warp. Which one an event takes depends on
// its own image count only.
constexpr int STEREO_SMALL_M = 8;
constexpr int STEREO_WARP_M = 24;

// Barrier of the NT threads of a group of warps (named barrier BAR), so that a
// larger CTA can run the CTA-wide stereo on a subset of its warps (or on two
// subsets at once, with different barriers).
template <int NT, int BAR = 1>
__device__ __forceinline__ void stereo_bar() {
    asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(NT) : "memory");
}

// Combine the sums of the NT threads of a group (warps gw .. gw + NT/32 - 1 of
// the CTA; by default the first NT threads) in a fixed order (a shuffle tree per
// warp, then the warps in index order) and form the event's row; every one of
// them returns it. red: NT / 32 * 5 double words and redi: NT / 32 * 2 ints of
// shared memory of the group. The group's threads must all call it, and no other
// thread; BAR is the group's named barrier.
template <int NT, int BAR = 1>
__device__ __forceinline__ rta_stereo_t cta_result(CSum (&acc)[5], int npair, int nvalid, DW* red, int* redi,
                                                   int gw = 0) {
    constexpr int NWC = NT / 32;
    const int lane = threadIdx.x & 31, warp = (threadIdx.x >> 5) - gw;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const DW v = dw_warp_sum(two_sum(acc[k].s, acc[k].c));
        if (lane == 0) red[warp * 5 + k] = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        npair += __shfl_xor_sync(0xffffffffu, npair, o);
        nvalid += __shfl_xor_sync(0xffffffffu, nvalid, o);
    }
    if (lane == 0) {
        redi[warp * 2] = npair;
        redi[warp * 2 + 1] = nvalid;
    }
    stereo_bar<NT, BAR>();
    DW tot[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        tot[k] = red[k];
        for (int w = 1; w < NWC; ++w) tot[k] = dw_add(tot[k], red[w * 5 + k]);
    }
    int np = 0, nv = 0;
    for (int w = 0; w < NWC; ++w) {
        np += redi[w * 2];
        nv += redi[w * 2 + 1];
    }
    stereo_bar<NT, BAR>();                             // red and redi may be reused
    return stereo_row(tot, np, nv);
}

}  // namespace rta
