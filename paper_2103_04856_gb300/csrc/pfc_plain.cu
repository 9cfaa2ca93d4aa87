// pfc_plain.cu -- the plain, unfused GPU path: what a framework's autograd
// would launch for eq. Feps.  Every intermediate goes through HBM:
//   deriv   : u            -> 9 stencil fields (grad u, Hess u)
//   local   : u, stencils  -> energy density + 10 cotangent fields
//   adjoint : cotangents   -> g (transposed stencils)
//   reduce  : e, g, u      -> E, lambda, max|g|, mean|g|, mass (FP64)
//   update  : u, g, lambda -> u - tau (g - lambda)
// It shares the per-voxel arithmetic (voxel_eval) with the fused sweep and
// is the baseline the fused sweep is measured against.
#include "pfc_device.cuh"

namespace pfc {

__device__ __forceinline__ int wrapp(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

#define PFC_GRID_STRIDE(i, n) \
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < (n); i += (long)gridDim.x * blockDim.x)

template <typename T>
__global__ void k_plain_deriv(const T* __restrict__ u, PlainBufs<T> b, int nx, int ny, int nz)
{
    const long n = (long)nx * ny * nz;
    PFC_GRID_STRIDE(i, n)
    {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long)nx * ny));
        auto at = [&](int dx, int dy, int dz) {
            return u[((long)wrapp(z + dz, nz) * ny + wrapp(y + dy, ny)) * nx + wrapp(x + dx, nx)];
        };
        const T u0 = at(0, 0, 0);
        const T xp = at(1, 0, 0), xm = at(-1, 0, 0), yp = at(0, 1, 0), ym = at(0, -1, 0);
        const T zp = at(0, 0, 1), zm = at(0, 0, -1);
        b.d[0][i] = xp - xm;
        b.d[1][i] = yp - ym;
        b.d[2][i] = zp - zm;
        b.d[3][i] = (xp + xm) - T(2) * u0;
        b.d[4][i] = (yp + ym) - T(2) * u0;
        b.d[5][i] = (zp + zm) - T(2) * u0;
        b.d[6][i] = (at(1, 1, 0) - at(1, -1, 0)) - (at(-1, 1, 0) - at(-1, -1, 0));
        b.d[7][i] = (at(1, 0, 1) - at(1, 0, -1)) - (at(-1, 0, 1) - at(-1, 0, -1));
        b.d[8][i] = (at(0, 1, 1) - at(0, 1, -1)) - (at(0, -1, 1) - at(0, -1, -1));
    }
}

// SYM: c3 = c5 = 0, the sqrt(D+) terms (weight zero) are not evaluated
template <typename T, bool SYM>
__global__ void k_plain_local(const T* __restrict__ u, PlainBufs<T> b, long n, Coef<T> C)
{
    PFC_GRID_STRIDE(i, n)
    {
        Cot<T> ct;
        b.e[i] = voxel_eval<T, true, false, false, SYM>(C, u[i], b.d[0][i], b.d[1][i], b.d[2][i], b.d[3][i], b.d[4][i],
                                     b.d[5][i], b.d[6][i], b.d[7][i], b.d[8][i], ct);
        b.ct[0][i] = ct.u;
        b.ct[1][i] = ct.dx;
        b.ct[2][i] = ct.dy;
        b.ct[3][i] = ct.dz;
        b.ct[4][i] = ct.hxx;
        b.ct[5][i] = ct.hyy;
        b.ct[6][i] = ct.hzz;
        b.ct[7][i] = ct.hxy;
        b.ct[8][i] = ct.hxz;
        b.ct[9][i] = ct.hyz;
    }
}

template <typename T>
__global__ void k_plain_adjoint(PlainBufs<T> b, int nx, int ny, int nz)
{
    const long n = (long)nx * ny * nz;
    PFC_GRID_STRIDE(i, n)
    {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long)nx * ny));
        auto at = [&](int f, int dx, int dy, int dz) {
            return b.ct[f][((long)wrapp(z + dz, nz) * ny + wrapp(y + dy, ny)) * nx + wrapp(x + dx, nx)];
        };
        T g = b.ct[0][i];
        // first differences: + cot(j - e_c) - cot(j + e_c)
        g += at(1, -1, 0, 0) - at(1, 1, 0, 0);
        g += at(2, 0, -1, 0) - at(2, 0, 1, 0);
        g += at(3, 0, 0, -1) - at(3, 0, 0, 1);
        // second differences: cot(j - e_c) - 2 cot(j) + cot(j + e_c)
        g += at(4, -1, 0, 0) - T(2) * b.ct[4][i] + at(4, 1, 0, 0);
        g += at(5, 0, -1, 0) - T(2) * b.ct[5][i] + at(5, 0, 1, 0);
        g += at(6, 0, 0, -1) - T(2) * b.ct[6][i] + at(6, 0, 0, 1);
        // mixed: cot(j-c-d) - cot(j-c+d) - cot(j+c-d) + cot(j+c+d)
        g += at(7, -1, -1, 0) - at(7, -1, 1, 0) - at(7, 1, -1, 0) + at(7, 1, 1, 0);
        g += at(8, -1, 0, -1) - at(8, -1, 0, 1) - at(8, 1, 0, -1) + at(8, 1, 0, 1);
        g += at(9, 0, -1, -1) - at(9, 0, -1, 1) - at(9, 0, 1, -1) + at(9, 0, 1, 1);
        b.g[i] = g;
    }
}

template <typename T>
__global__ void k_plain_reduce(const T* __restrict__ u, const T* __restrict__ e, const T* __restrict__ g,
                               long n, Inst<T> in, int mode)
{
    __shared__ double red[32 * NPART];
    double v[NPART] = { 0, 0, 0, 0, 0, 0 };
    PFC_GRID_STRIDE(i, n)
    {
        v[P_E] += (double)e[i];
        v[P_U] += (double)u[i];
        const double gi = (double)g[i];
        v[P_G] += gi;
        v[P_AG] += fabs(gi);
        v[P_GMAX] = fmax(v[P_GMAX], fabs(gi));
    }
    // the explicit update writes the true field: report it as the new stored
    // field with a zero offset
    v[P_OUT] = v[P_U];
    grid_finish(in, blockIdx.x, mode, v, red);
}

template <typename T>
__global__ void k_plain_update(const T* __restrict__ u, const T* __restrict__ g, T* __restrict__ out, long n,
                               T tau, const double* __restrict__ scal)
{
    const T lam = (T)scal[S_LAMBDA];
    PFC_GRID_STRIDE(i, n) out[i] = u[i] - tau * (g[i] - lam);
}

int plain_blocks(long n)
{
    const long b = (n + 255) / 256, cap = 8L * device_sms();
    return (int)(b < cap ? b : cap);
}

template <typename T>
cudaError_t launch_plain(const T* u, T* out, const PlainBufs<T>& b_in, int nx, int ny, int nz, const Coef<T>& C,
                         int mode, T tau, double inv_N, double* partials, int nblocks, unsigned* ints,
                         double* scal, double* trace, int trace_cap, cudaStream_t s)
{
    const long n = (long)nx * ny * nz;
    const int nb = plain_blocks(n);
    PlainBufs<T> b = b_in;
    if (mode == MODE_GRAD) b.g = out;   // the gradient goes straight to the caller
    Inst<T> in{};
    in.nblocks = nblocks;
    in.partials = partials;
    in.ints = ints;
    in.scal = scal;
    in.trace = trace;
    in.trace_cap = trace_cap;
    in.inv_N = inv_N;
    if (nb != nblocks) return cudaErrorInvalidValue;
    k_plain_deriv<T><<<nb, 256, 0, s>>>(u, b, nx, ny, nz);
    if (C.sym) k_plain_local<T, true><<<nb, 256, 0, s>>>(u, b, n, C);
    else k_plain_local<T, false><<<nb, 256, 0, s>>>(u, b, n, C);
    if (mode != MODE_ENERGY) k_plain_adjoint<T><<<nb, 256, 0, s>>>(b, nx, ny, nz);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    // MODE_STEP here: explicit projection (no lazy offset); the finisher's
    // step bookkeeping sees "new stored field = evaluated field", i.e. S_C = 0
    k_plain_reduce<T><<<nb, 256, 0, s>>>(u, b.e, mode == MODE_ENERGY ? b.e : b.g, n, in, mode);
    if (mode == MODE_STEP) k_plain_update<T><<<nb, 256, 0, s>>>(u, b.g, out, n, tau, scal);
    return cudaGetLastError();
}
template cudaError_t launch_plain<float>(const float*, float*, const PlainBufs<float>&, int, int, int,
                                         const Coef<float>&, int, float, double, double*, int, unsigned*,
                                         double*, double*, int, cudaStream_t);
template cudaError_t launch_plain<double>(const double*, double*, const PlainBufs<double>&, int, int, int,
                                          const Coef<double>&, int, double, double, double*, int, unsigned*,
                                          double*, double*, int, cudaStream_t);

}  // namespace pfc
