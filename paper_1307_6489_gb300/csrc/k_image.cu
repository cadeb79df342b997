// The unfused image-stage kernels (k_clean, k_hillas) and the host-side
// launchers of the fused image kernel; the kernels themselves live in
// k_image_chain.cuh, whose neighbour-peak and byte-stream instantiations are
// compiled in k_image_nb.cu and k_image_stream.cu.
#include "k_image_chain.cuh"

namespace rta {

// ------------------------------------------------------------------ unfused stage kernels

// Bitmaps of one image from per-pixel values in global memory: the warp that
// covers 32 consecutive pixels writes their word.
__device__ __forceinline__ void ballot_words(int P, int tid, int nthr, uint32_t* w0, uint32_t* w1, const float* q,
                                             float t0, float t1) {
    for (int base = 0; base < P; base += nthr) {
        const int p = base + tid;
        const float v = p < P ? q[p] : 0.f;
        const uint32_t b0 = __ballot_sync(0xffffffffu, p < P && v >= t0);
        const uint32_t b1 = __ballot_sync(0xffffffffu, p < P && v >= t1);
        if ((tid & 31) == 0 && (p >> 5) < words_of(P)) {
            w0[p >> 5] = b0;
            if (w1) w1[p >> 5] = b1;
        }
    }
}

__global__ void __launch_bounds__(256) k_clean(const CleanArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* sq = reinterpret_cast<float*>(smem_raw);
    const int maxw = words_of(a.arr.max_P);
    uint32_t* bits0 = reinterpret_cast<uint32_t*>(sq + a.arr.max_P);
    const ImgBits ib = {bits0, bits0 + maxw, bits0 + 2 * maxw, bits0 + 3 * maxw};
    for (int64_t img = blockIdx.x; img < a.n_img; img += gridDim.x) {
        const int tel = a.img_tel[img];
        if (tel < 0 || tel >= a.arr.n_tel) {
            if (threadIdx.x == 0) atomicOr(a.status, RTA_DEV_BAD_IMAGE);
            continue;
        }
        const DevCam C = a.arr.cams[a.arr.tel_cam[tel]];
        const int64_t off = a.pix_off[img];
        if (off < 0 || off + C.P > a.n_q) {
            if (threadIdx.x == 0) atomicOr(a.status, RTA_DEV_BAD_IMAGE);
            continue;
        }
        for (int p = threadIdx.x; p < C.P; p += blockDim.x) sq[p] = a.q[off + p];
        __syncthreads();
        ballot_words(C.P, threadIdx.x, blockDim.x, ib.hi, ib.lo, sq, a.pp.t_hi, a.pp.t_lo);
        __syncthreads();
        clean_bits(C, a.pp, ib, threadIdx.x, blockDim.x, BlockBar());
        for (int p = threadIdx.x; p < C.P; p += blockDim.x) a.mask[off + p] = bit_of(ib.mask, p) ? 1 : 0;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_hillas(const HillasArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ float red[3 * NCW * 8];
    float* sq = reinterpret_cast<float*>(smem_raw);
    float* st = sq + a.arr.max_P;
    float* sm = st + a.arr.max_P;
    uint32_t* mask = reinterpret_cast<uint32_t*>(sm + a.arr.max_P);
    for (int64_t img = blockIdx.x; img < a.n_img; img += gridDim.x) {
        const int tel = a.img_tel[img];
        if (tel < 0 || tel >= a.arr.n_tel) {
            if (threadIdx.x == 0) {
                atomicOr(a.status, RTA_DEV_BAD_IMAGE);
                write_bad_row(a.out + img);
            }
            continue;
        }
        const DevCam C = a.arr.cams[a.arr.tel_cam[tel]];
        const int64_t off = a.pix_off[img];
        if (off < 0 || off + C.P > a.n_q) {
            if (threadIdx.x == 0) {
                atomicOr(a.status, RTA_DEV_BAD_IMAGE);
                write_bad_row(a.out + img);
            }
            continue;
        }
        for (int p = threadIdx.x; p < C.P; p += blockDim.x) {
            sq[p] = a.q[off + p];
            if (a.t) st[p] = a.t[off + p];
            sm[p] = a.mask[off + p] ? 1.f : 0.f;
        }
        __syncthreads();
        ballot_words(C.P, threadIdx.x, blockDim.x, mask, nullptr, sm, 0.5f, 0.5f);
        __syncthreads();
        hillas_bits(sq, a.t ? st : nullptr, C, mask, red, threadIdx.x, blockDim.x, BlockBar(), a.out + img);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host-side launchers
// Tile-shape variants of the fused kernel: (integrator warps, pixels per thread).
struct ChainVariant {
    int iw, ppt, min_blocks;   // integrator warps, pixels per thread, CTAs per SM the registers are sized for
};
static const ChainVariant kVariants[RTA_CHAIN_VARIANTS] = {{8, 1, 2}, {4, 2, 2}, {8, 2, 2}, {4, 1, 2}, {8, 1, 3}};

int chain_variant_warps(int v) { return kVariants[v].iw; }
int chain_variant_ppt(int v) { return kVariants[v].ppt; }
int chain_variant_min_blocks(int v) { return kVariants[v].min_blocks; }
int chain_threads(int v) { return kVariants[v].iw * 32 + 64; }

int chain_stage_wave_bytes(int v, int max_S) {
    const int chunk = kVariants[v].iw * 32 * kVariants[v].ppt;
    int swb = ((chunk * 2 * max_S + 16) + 127) & ~127;
    const int cap = 48 * 1024;
    return swb < cap ? swb : cap;
}

size_t chain_smem_bytes(int v, int nstage, int stage_wave_bytes, int max_P, int nb_keys, int stream_recs) {
    const size_t head = (sizeof(ChainSmem) + 127) & ~size_t(127);
    const size_t words = (max_P + 31) / 32;
    const size_t chunk = size_t(kVariants[v].iw) * 32 * kVariants[v].ppt;
    const size_t keys = nb_keys ? 10 * size_t(max_P) + 16 : 0;   // 64-bit keys, 16-bit candidate ids
    const size_t recs = stream_recs ? 2 * sizeof(StreamImg) + 16 : 0;   // the producer's two stream records
    return head + size_t(nstage) * (stage_wave_bytes + 2 * chunk * 4) + NSLOT * slot_bytes(max_P) + 8 * words + 16 +
           keys + recs;
}

int chain_chunk_pixels(int v, int stage_wave_bytes, int S) {
    return chunk_pixels(kVariants[v].iw * 32 * kVariants[v].ppt, stage_wave_bytes, S);
}

template <int IW, int PPT, int MB>
static cudaError_t launch_t(const ChainArgs& a, int grid, size_t smem, cudaStream_t s, bool occupancy_only,
                            int* occ) {
    auto kern = k_image_chain<IW, PPT, MB, false>;
    // the dynamic shared-memory opt-in is per device; remember the largest size set
    static size_t attr_bytes[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || attr_bytes[dev] < smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_bytes[dev] = smem;
    }
    if (occupancy_only) {
        *occ = 0;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, IW * 32 + 64, smem);
    }
    kern<<<grid, IW * 32 + 64, smem, s>>>(a);
    return cudaGetLastError();
}

static cudaError_t dispatch(int v, const ChainArgs& a, int grid, size_t smem, cudaStream_t s, bool occ_only,
                            int* occ) {
    switch (v) {
    case 0: return launch_t<8, 1, 2>(a, grid, smem, s, occ_only, occ);
    case 1: return launch_t<4, 2, 2>(a, grid, smem, s, occ_only, occ);
    case 2: return launch_t<8, 2, 2>(a, grid, smem, s, occ_only, occ);
    case 3: return launch_t<4, 1, 2>(a, grid, smem, s, occ_only, occ);
    case 4: return launch_t<8, 1, 3>(a, grid, smem, s, occ_only, occ);   // registers for three CTAs per SM
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_image_chain(int v, const ChainArgs& a, int grid, size_t smem, cudaStream_t s) {
    // the image chain on a contiguous bundle (flat window, neighbour-peak window or
    // digital filter) runs a lean instantiation; the per-pixel outputs (integrate-only
    // charges and times, cleaning masks) are compiled into the general ones only
    if (!a.smeta && !a.integrate_only && !a.mask_out)
        return dispatch_image_chain_lean(v, a, grid, smem, s, false, nullptr);
    if (a.pp.nbpeak) return dispatch_image_chain_nb(v, a, grid, smem, s, false, nullptr);
    if (a.smeta) return dispatch_image_chain_stream(v, a, grid, smem, s, false, nullptr);
    return dispatch(v, a, grid, smem, s, false, nullptr);
}

int chain_occupancy(int v, size_t smem, int kind) {
    int n = 0;
    ChainArgs dummy = {};
    const cudaError_t e = kind == CHAIN_NB       ? dispatch_image_chain_nb(v, dummy, 0, smem, nullptr, true, &n)
                          : kind == CHAIN_STREAM ? dispatch_image_chain_stream(v, dummy, 0, smem, nullptr, true, &n)
                                                 : dispatch(v, dummy, 0, smem, nullptr, true, &n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_clean(const CleanArgs& a, int grid, cudaStream_t s) {
    const size_t smem = size_t(a.arr.max_P) * 4 + size_t(16) * ((a.arr.max_P + 31) / 32) + 16;
    k_clean<<<grid, 256, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_hillas(const HillasArgs& a, int grid, cudaStream_t s) {
    const size_t smem = size_t(a.arr.max_P) * 12 + size_t(4) * ((a.arr.max_P + 31) / 32) + 16;
    k_hillas<<<grid, 256, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace rta
