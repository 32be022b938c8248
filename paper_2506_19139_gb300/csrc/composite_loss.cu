// The loss-channel instances (distortion and extent, Sec. 3.3, App. C.1-C.2) of the composite
// kernels, in a unit of their own so that the two halves of the instantiations compile in parallel.
#include "composite_kernels.cuh"

namespace sof {

cudaError_t launch_composite_loss(const CompositeParams &p, int total_tiles, int tile, int chunk, int reorder_k,
                                  bool bwd, cudaStream_t s) {
    return bwd ? dispatch<true, true>(p, total_tiles, tile, chunk, reorder_k, s)
               : dispatch<false, true>(p, total_tiles, tile, chunk, reorder_k, s);
}

cudaError_t launch_composite_fallback_loss(const CompositeParams &p, int tile, bool bwd, cudaStream_t s) {
    if (tile == 8) return bwd ? launch_fb<8, true, true>(p, s) : launch_fb<8, false, true>(p, s);
    if (tile == 16) return bwd ? launch_fb<16, true, true>(p, s) : launch_fb<16, false, true>(p, s);
    if (tile == 32) return bwd ? launch_fb<32, true, true>(p, s) : launch_fb<32, false, true>(p, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_composite_replay_loss(const CompositeParams &p, int total_tiles, int tile, cudaStream_t s) {
    const unsigned grid = (unsigned)(((long long)total_tiles * tile * tile + 255) / 256);
    if (tile == 8)
        return launch_replay_instance<8, true>(p, grid, s);
    else if (tile == 16)
        return launch_replay_instance<16, true>(p, grid, s);
    else if (tile == 32)
        return launch_replay_instance<32, true>(p, grid, s);
    return cudaErrorInvalidValue;
}

}  // namespace sof
