// The byte-stream instantiations of the fused image kernel (k_image_chain with
// STREAM = true, k_image_chain.cuh): the producer copies each chunk from the
// segments of an ingested stream. The stream path never runs integrate-only; a
// lean form (LEAN = true) also leaves out the digital filter and serves every
// other window mode. Compiled apart so the builds run in parallel.
#include "k_image_chain.cuh"

namespace rta {

template <int IW, int PPT, int MB, bool LEAN>
static cudaError_t launch_stream(const ChainArgs& a, int grid, size_t smem, cudaStream_t s, bool occupancy_only,
                                 int* occ) {
    auto kern = k_image_chain<IW, PPT, MB, false, true, LEAN>;
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
cudaError_t dispatch_image_chain_stream(int v, const ChainArgs& a, int grid, size_t smem, cudaStream_t s,
                                        bool occ_only, int* occ) {
    if (!a.pp.filter && !occ_only) {
        switch (v) {
        case 0: return launch_stream<8, 1, 2, true>(a, grid, smem, s, occ_only, occ);
        case 1: return launch_stream<4, 2, 2, true>(a, grid, smem, s, occ_only, occ);
        case 2: return launch_stream<8, 2, 2, true>(a, grid, smem, s, occ_only, occ);
        case 3: return launch_stream<4, 1, 2, true>(a, grid, smem, s, occ_only, occ);
        case 4: return launch_stream<8, 1, 3, true>(a, grid, smem, s, occ_only, occ);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (v) {
    case 0: return launch_stream<8, 1, 2, false>(a, grid, smem, s, occ_only, occ);
    case 1: return launch_stream<4, 2, 2, false>(a, grid, smem, s, occ_only, occ);
    case 2: return launch_stream<8, 2, 2, false>(a, grid, smem, s, occ_only, occ);
    case 3: return launch_stream<4, 1, 2, false>(a, grid, smem, s, occ_only, occ);
    case 4: return launch_stream<8, 1, 3, false>(a, grid, smem, s, occ_only, occ);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace rta
