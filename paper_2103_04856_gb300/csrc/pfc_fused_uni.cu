// pfc_fused_uni.cu -- batched fused sweeps whose problems share one
// coefficient set and step size (k_fused<..., UNI = true>): the per-voxel
// arithmetic reads them from the launch's fixed fields, not from the
// descriptor of the run's problem.  Its own translation unit, so that these
// instantiations build in parallel with the others.
#include "pfc_fused_kernel.cuh"

namespace pfc {

template <bool SYM>
static cudaError_t launch_uni(const Launch<float, BATCH_MAX>& L, int tile_y, int mode, cudaStream_t s)
{
    if (mode == MODE_GRAD)
        return tile_y == 8    ? launch_kernel<float, 8, MODE_GRAD, BATCH_MAX, 0, SYM, false, true>(L, L.grid, s)
               : tile_y == 13 ? launch_kernel<float, 13, MODE_GRAD, BATCH_MAX, 0, SYM, false, true>(L, L.grid, s)
                              : launch_kernel<float, 16, MODE_GRAD, BATCH_MAX, 0, SYM, false, true>(L, L.grid, s);
    if (mode == MODE_STEP)
        return tile_y == 8    ? launch_kernel<float, 8, MODE_STEP, BATCH_MAX, 0, SYM, false, true>(L, L.grid, s)
               : tile_y == 13 ? launch_kernel<float, 13, MODE_STEP, BATCH_MAX, 0, SYM, false, true>(L, L.grid, s)
                              : launch_kernel<float, 16, MODE_STEP, BATCH_MAX, 0, SYM, false, true>(L, L.grid, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_fused_uni(const Launch<float, BATCH_MAX>& L, int tile_y, int mode, bool sym, cudaStream_t s)
{
    return sym ? launch_uni<true>(L, tile_y, mode, s) : launch_uni<false>(L, tile_y, mode, s);
}

}  // namespace pfc
