// pfc_fused_slab.cu -- the fused sweep of a z-slab: the planes beyond the
// slab's ends come from its halo buffer instead of the periodic wrap.  Its
// own translation unit, so that the instantiations build in parallel with
// pfc_fused.cu and no other launch carries the halo check.
#include "pfc_fused_kernel.cuh"

namespace pfc {

template <typename T, int TY, int EXT>
static cudaError_t launch_halo_mode(const Inst<T>& in, int mode, int max_run, cudaStream_t s)
{
    Launch<T, 1> L;
    L.n = 1;
    L.inst[0] = in;
    plan(L, TY, max_run);
    switch (mode) {
    case MODE_ENERGY: return launch_kernel<T, TY, MODE_ENERGY, 1, EXT, false, true>(L, L.grid, s);
    case MODE_GRAD: return launch_kernel<T, TY, MODE_GRAD, 1, EXT, false, true>(L, L.grid, s);
    case MODE_STEP: return launch_kernel<T, TY, MODE_STEP, 1, EXT, false, true>(L, L.grid, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_fused_halo(const Inst<T>& in, int mode, int tile_y, int max_run, cudaStream_t s)
{
    if (in.cf) return cudaErrorInvalidValue;   // slabs carry no coefficient field
    if (in.C.proj) return launch_halo_mode<T, EXT_TILE_Y, 2>(in, mode, max_run, s);
    if (needs_ext(in)) return launch_halo_mode<T, EXT_TILE_Y, 1>(in, mode, max_run, s);
    if (tile_y == 8) return launch_halo_mode<T, 8, 0>(in, mode, max_run, s);
    if (tile_y == 13) return launch_halo_mode<T, 13, 0>(in, mode, max_run, s);
    return launch_halo_mode<T, 16, 0>(in, mode, max_run, s);
}
template cudaError_t launch_fused_halo<float>(const Inst<float>&, int, int, int, cudaStream_t);
template cudaError_t launch_fused_halo<double>(const Inst<double>&, int, int, int, cudaStream_t);

}  // namespace pfc
