// The lean instantiations of the fused image kernel (k_image_chain.cuh): the
// image chain on contiguous bundles without the integrate-only outputs -- the
// flat window and the neighbour-peak window (LEAN = true, also without the
// digital filter) and the digital filter (FILT = true) -- so that those
// branches are not compiled into the kernels the reconstruction runs. Compiled
// apart from the other instantiations so that the builds run in parallel.
#include "k_image_chain.cuh"

namespace rta {

// FILT: the form with the digital filter (LEAN = false, FILT = true).
template <int IW, int PPT, int MB, bool NB, bool FILT = false>
static cudaError_t launch_lean(const ChainArgs& a, int grid, size_t smem, cudaStream_t s, bool occupancy_only,
                               int* occ) {
    auto kern = k_image_chain<IW, PPT, MB, NB, false, !FILT, FILT>;
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

// The same tile variants as the other window modes (kVariants in k_image.cu).
cudaError_t dispatch_image_chain_lean(int v, const ChainArgs& a, int grid, size_t smem, cudaStream_t s,
                                      bool occ_only, int* occ) {
    if (a.pp.nbpeak) {
        switch (v) {
        case 0: return launch_lean<8, 1, 2, true>(a, grid, smem, s, occ_only, occ);
        case 1: return launch_lean<4, 2, 2, true>(a, grid, smem, s, occ_only, occ);
        case 2: return launch_lean<8, 2, 2, true>(a, grid, smem, s, occ_only, occ);
        case 3: return launch_lean<4, 1, 2, true>(a, grid, smem, s, occ_only, occ);
        case 4: return launch_lean<8, 1, 3, true>(a, grid, smem, s, occ_only, occ);
        default: return cudaErrorInvalidValue;
        }
    }
    if (a.pp.filter) {
        switch (v) {
        case 0: return launch_lean<8, 1, 2, false, true>(a, grid, smem, s, occ_only, occ);
        case 1: return launch_lean<4, 2, 2, false, true>(a, grid, smem, s, occ_only, occ);
        case 2: return launch_lean<8, 2, 2, false, true>(a, grid, smem, s, occ_only, occ);
        case 3: return launch_lean<4, 1, 2, false, true>(a, grid, smem, s, occ_only, occ);
        case 4: return launch_lean<8, 1, 3, false, true>(a, grid, smem, s, occ_only, occ);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (v) {
    case 0: return launch_lean<8, 1, 2, false>(a, grid, smem, s, occ_only, occ);
    case 1: return launch_lean<4, 2, 2, false>(a, grid, smem, s, occ_only, occ);
    case 2: return launch_lean<8, 2, 2, false>(a, grid, smem, s, occ_only, occ);
    case 3: return launch_lean<4, 1, 2, false>(a, grid, smem, s, occ_only, occ);
    case 4: return launch_lean<8, 1, 3, false>(a, grid, smem, s, occ_only, occ);   // registers for three CTAs per SM
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace rta
