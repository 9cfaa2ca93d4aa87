// pfc_fused_sym.cu -- the fused sweep for launches whose problems all have
// c3 = c5 = 0 (polynomials symmetric in kappa1, kappa2): FP32, no extensions.
// The sqrt(D+) terms of eq. Feps have weight c3 T + c5 q = 0 there; this
// instantiation does not compile them in (nor the refinement of D that serves
// them), with the same result bits as the general sweep.
#include "pfc_fused_kernel.cuh"

namespace pfc {

template <int MAXI>
cudaError_t launch_fused_sym(const Launch<float, MAXI>& L, int tile_y, int mode, cudaStream_t s)
{
    if constexpr (MAXI == 1) {
        if (mode == MODE_ENERGY)
            return tile_y == 8    ? launch_kernel<float, 8, MODE_ENERGY, 1, 0, true>(L, L.grid, s)
                   : tile_y == 13 ? launch_kernel<float, 13, MODE_ENERGY, 1, 0, true>(L, L.grid, s)
                                  : launch_kernel<float, 16, MODE_ENERGY, 1, 0, true>(L, L.grid, s);
    }
    if (mode == MODE_GRAD)
        return tile_y == 8    ? launch_kernel<float, 8, MODE_GRAD, MAXI, 0, true>(L, L.grid, s)
               : tile_y == 13 ? launch_kernel<float, 13, MODE_GRAD, MAXI, 0, true>(L, L.grid, s)
                              : launch_kernel<float, 16, MODE_GRAD, MAXI, 0, true>(L, L.grid, s);
    if (mode == MODE_STEP)
        return tile_y == 8    ? launch_kernel<float, 8, MODE_STEP, MAXI, 0, true>(L, L.grid, s)
               : tile_y == 13 ? launch_kernel<float, 13, MODE_STEP, MAXI, 0, true>(L, L.grid, s)
                              : launch_kernel<float, 16, MODE_STEP, MAXI, 0, true>(L, L.grid, s);
    return cudaErrorInvalidValue;
}
template cudaError_t launch_fused_sym<1>(const Launch<float, 1>&, int, int, cudaStream_t);
template cudaError_t launch_fused_sym<BATCH_MAX>(const Launch<float, BATCH_MAX>&, int, int, cudaStream_t);

}  // namespace pfc
