// Launchers of the exact-order composite (forward and backward), its fallback, the backward replay
// and the opacity at the exact depth; the kernels are in composite_kernels.cuh, and their
// loss-channel instances are compiled in composite_loss.cu.
#include "composite_kernels.cuh"

namespace sof {

cudaError_t launch_composite_fwd(const CompositeParams &p, int total_tiles, int tile, int chunk, int reorder_k,
                                 cudaStream_t s) {
    if (p.loss_sums) return launch_composite_loss(p, total_tiles, tile, chunk, reorder_k, false, s);
    return dispatch<false, false>(p, total_tiles, tile, chunk, reorder_k, s);
}

cudaError_t launch_composite_fallback(const CompositeParams &p, int tile, bool bwd, cudaStream_t s) {
    if (p.loss_sums) return launch_composite_fallback_loss(p, tile, bwd, s);
    if (tile == 8) return bwd ? launch_fb<8, true>(p, s) : launch_fb<8, false>(p, s);
    if (tile == 32) return bwd ? launch_fb<32, true>(p, s) : launch_fb<32, false>(p, s);
    if (tile == 16) return bwd ? launch_fb<16, true>(p, s) : launch_fb<16, false>(p, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_composite_replay(const CompositeParams &p, int total_tiles, int tile, cudaStream_t s) {
    if (total_tiles <= 0 || !p.hit_list) return cudaSuccess;
    note_launches(1);
    const unsigned grid = (unsigned)(((long long)total_tiles * tile * tile + 255) / 256);
    if (p.loss_sums) return launch_composite_replay_loss(p, total_tiles, tile, s);
    if (tile == 8)
        return launch_replay_instance<8, false>(p, grid, s);
    else if (tile == 16)
        return launch_replay_instance<16, false>(p, grid, s);
    else if (tile == 32)
        return launch_replay_instance<32, false>(p, grid, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_opacity_at_depth(const CompositeParams &p, int total_tiles, int tile, bool bwd, cudaStream_t s) {
    if (total_tiles <= 0 || !p.hit_list) return cudaSuccess;
    note_launches(1);
    const unsigned grid = (unsigned)(((long long)total_tiles * tile * tile + 255) / 256);
#define SOF_OPA(TT)                                                              \
    if (tile == TT) {                                                            \
        if (bwd)                                                                 \
            k_opacity_at_depth<TT, true><<<grid, 256, 0, s>>>(p);                \
        else                                                                     \
            k_opacity_at_depth<TT, false><<<grid, 256, 0, s>>>(p);               \
        return cudaGetLastError();                                               \
    }
    SOF_OPA(8)
    SOF_OPA(16)
    SOF_OPA(32)
#undef SOF_OPA
    return cudaErrorInvalidValue;
}

cudaError_t launch_composite_bwd(const CompositeParams &p, int total_tiles, int tile, int chunk, int reorder_k,
                                 cudaStream_t s) {
    if (p.loss_sums) return launch_composite_loss(p, total_tiles, tile, chunk, reorder_k, true, s);
    return dispatch<true, false>(p, total_tiles, tile, chunk, reorder_k, s);
}

}  // namespace sof
