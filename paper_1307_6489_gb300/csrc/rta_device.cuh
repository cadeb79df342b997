// Device-side building blocks shared by the librta kernels: the device view of
// the registered cameras and array, launch parameter blocks, and thin inline-PTX
// wrappers for mbarriers, bulk (TMA engine) copies, named barriers and the
// global timer used to bound every wait.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rta.h"

#define RTA_MAX_PIX 4096
#define RTA_MAX_SAMPLES 128
#define RTA_MAX_W 16
#define RTA_MAX_TEL 1024
#define RTA_NB_PAD 8          // neighbour rows padded to 8 x int16 = 16 bytes
#define RTA_CALIB_ALIGN 8     // calibration rows of each telescope start on a multiple of 8
#define RTA_STEREO_MAX_M 64
#define RTA_WAIT_TIMEOUT_NS 2000000000ull

namespace rta {

struct DevCam {
    int P, S, K, pad;
    const float2* xy;        // P pixel centres (deg)
    const int4* nb;          // P rows of 8 int16 neighbour ids (-1 = none)
};

struct DevArray {
    const DevCam* cams;      // RTA_MAX_CAMS entries in device memory
    const int32_t* tel_cam;  // n_tel
    const float2* tel_xy;    // n_tel (m)
    const int64_t* tel_row;  // n_tel: first (8-aligned) calibration row
    const int32_t* p16;      // padded calibration table
    const float* scale;
    int n_tel;
    int max_P;
};

struct ProcParams {
    int sliding, start, W, core_nb;
    float t_hi, t_lo;
    // Runtime copies of the constants 1 and 128. Integer multiply-adds by a value
    // the compiler cannot see run on the FMA pipe, so part of the window search
    // leaves the integer ALU pipe, which it would otherwise saturate.
    int one, k128;
    // digital-filter-style extractor: charge from integer weights over the window
    int filter, csum;
    int wts[RTA_MAX_W];
    // neighbour-peak window: two sweeps over every image (keys, then charges)
    int nbpeak;
};

// ------------------------------------------------------------------ PTX helpers
// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute may start while the kernel before it on the
// stream is finishing; this wait (a no-op otherwise) returns once that kernel
// has completed and its memory is visible. Nothing an earlier kernel writes may
// be read before it.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// The kernel after this one on the stream, when launched as a programmatic
// dependent, may be scheduled once every CTA of this kernel has signalled (or
// exited): a CTA signals when it has taken its last work item, so that the next
// kernel's set-up runs on SMs freed by the tail of this one. Its wait still
// sees all of this kernel's writes.
__device__ __forceinline__ void grid_dependents_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// As mbar_try_wait, but a thread whose phase is not complete may sleep in the
// instruction until the phase completes, at most suspend_ns: waiting warps stop
// taking issue slots from working ones.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t suspend_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(suspend_ns)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `parity` to complete. Gives up after timeout_ns or as
// soon as *abort becomes non-zero (both checked between sleeps of at most
// 100 us); returns false then.
__device__ __forceinline__ bool mbar_wait_ns(uint64_t* bar, uint32_t parity, volatile int* abort, uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait_sleep(bar, parity, 100000u)) {
        if (*abort) return false;
        if (global_ns() - t0 > timeout_ns) return false;
    }
    return true;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
    return mbar_wait_ns(bar, parity, abort, RTA_WAIT_TIMEOUT_NS);
}

// 16 bytes global -> shared by the calling thread without holding registers
// (cp.async); complete for this thread after cp_async_wait_all.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// One bulk copy global -> shared through the TMA engine, completing `bytes` of
// transaction count on `bar`. dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                         uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// a*b - c*d with one rounding error (Kahan's FMA-based difference of products)
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
    float w = c * d;
    float e = __fmaf_rn(-c, d, w);
    float f = __fmaf_rn(a, b, -w);
    return f + e;
}

}  // namespace rta
