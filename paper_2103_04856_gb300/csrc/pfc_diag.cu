// pfc_diag.cu -- viability diagnostics of a phase field (Sec. 4.5): the
// discrepancy  h^3 sum |eps/2 |grad u|^2 - W(u)/eps|, the Cahn-Hilliard
// energy  h^3 sum (eps/2 |grad u|^2 + W(u)/eps)  (the diffuse area) and the
// extremes of u.  grad u is the periodic central difference, without xi.
//
// One pass that marches in z (HBM-bound: u is read once); per-thread sums
// in the arithmetic type, FP64 across warps and blocks, combined in a fixed
// order by the last block to finish (ticket).
#include "pfc_device.cuh"

namespace pfc {

namespace {

constexpr int kDX = 32, kDY = 8;
constexpr int kDiagThreads = kDX * kDY;

__device__ __forceinline__ double fmax_(double a, double b) { return a > b ? a : b; }
__device__ __forceinline__ double fmin_(double a, double b) { return a < b ? a : b; }

// Block (32 x 8 threads) = one (x, y) tile; blockIdx.z = a chunk of zc
// planes that every thread marches through, keeping u(z-1), u(z), u(z+1) of
// its column in registers: one new load per voxel from HBM, the four x/y
// neighbours from L1/L2, and no index arithmetic beyond a pointer step.
template <typename T>
__global__ void __launch_bounds__(kDiagThreads) k_diag(const T* __restrict__ u, int nx, int ny, int nz, int zc, T sg,
                                                      T half_eps, T inv_eps, int well, double h3, double* part,
                                                      unsigned* ticket, double* out)
{
    const long pls = (long)nx * ny;
    const int x = blockIdx.x * kDX + threadIdx.x, y = blockIdx.y * kDY + threadIdx.y;
    const int z0 = blockIdx.z * zc, z1 = min(nz, z0 + zc);
    T sd = 0, sc = 0;
    T umax = -INFINITY, umin = INFINITY;
    if (x < nx && y < ny && z0 < z1) {
        const int xm = nbr(x, -1, nx) - x, xp = nbr(x, 1, nx) - x;
        const long ym = (long)(nbr(y, -1, ny) - y) * nx, yp = (long)(nbr(y, 1, ny) - y) * nx;
        const T* col = u + (long)y * nx + x;
        T um = col[(long)nbr(z0, -1, nz) * pls];
        T u0 = col[(long)z0 * pls];
        const T* c = col + (long)z0 * pls;
#pragma unroll 4
        for (int z = z0; z < z1; ++z, c += pls) {
            const T up = col[(long)(z + 1 == nz ? 0 : z + 1) * pls];
            const T gx = sg * (c[xp] - c[xm]);
            const T gy = sg * (c[yp] - c[ym]);
            const T gz = sg * (up - um);
            const T kin = half_eps * fma_(gx, gx, fma_(gy, gy, gz * gz));
            T W;
            if (well == 0) {
                const T t = u0 - u0 * u0;   // u (1 - u)
                W = t * t;
            } else {
                const T t = T(1) - u0 * u0;
                W = T(0.25) * t * t;
            }
            const T pot = W * inv_eps;
            const T d = kin - pot;
            sd += d < T(0) ? -d : d;
            sc += kin + pot;
            umax = u0 > umax ? u0 : umax;
            umin = u0 < umin ? u0 : umin;
            um = u0;
            u0 = up;
        }
    }
    // FP64 beyond the thread: warp shuffles, then one value per warp
    double v[4] = { (double)sd, (double)sc, (double)umax, (double)umin };
    __shared__ double red[kDiagThreads / 32][4];
    __shared__ int last;
    const int tid = threadIdx.y * kDX + threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        v[1] += __shfl_xor_sync(0xffffffffu, v[1], o);
        v[2] = fmax_(v[2], __shfl_xor_sync(0xffffffffu, v[2], o));
        v[3] = fmin_(v[3], __shfl_xor_sync(0xffffffffu, v[3], o));
    }
    if (lane == 0)
        for (int k = 0; k < 4; ++k) red[wid][k] = v[k];
    __syncthreads();
    const int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (tid == 0) {
        double s0 = 0, s1 = 0, mx = -INFINITY, mn = INFINITY;
        for (int w = 0; w < kDiagThreads / 32; ++w) {
            s0 += red[w][0];
            s1 += red[w][1];
            mx = fmax_(mx, red[w][2]);
            mn = fmin_(mn, red[w][3]);
        }
        double* p = part + (size_t)bid * 4;
        p[0] = s0; p[1] = s1; p[2] = mx; p[3] = mn;
        __threadfence();
        last = atomicAdd(ticket, 1u) == (unsigned)nblocks - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s0 = 0, s1 = 0, mx = -INFINITY, mn = INFINITY;
    for (int b = tid; b < nblocks; b += kDiagThreads) {
        const double* p = part + (size_t)b * 4;
        s0 += __ldcg(p);
        s1 += __ldcg(p + 1);
        mx = fmax_(mx, __ldcg(p + 2));
        mn = fmin_(mn, __ldcg(p + 3));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        mx = fmax_(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = fmin_(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    __syncthreads();
    if (lane == 0) { red[wid][0] = s0; red[wid][1] = s1; red[wid][2] = mx; red[wid][3] = mn; }
    __syncthreads();
    if (tid != 0) return;
    s0 = 0; s1 = 0; mx = -INFINITY; mn = INFINITY;
    for (int w = 0; w < kDiagThreads / 32; ++w) {
        s0 += red[w][0];
        s1 += red[w][1];
        mx = fmax_(mx, red[w][2]);
        mn = fmin_(mn, red[w][3]);
    }
    out[0] = h3 * s0;
    out[1] = h3 * s1;
    out[2] = s1 > 0.0 ? s0 / s1 : 0.0;
    out[3] = mx;
    out[4] = mn;
    __threadfence();
    *ticket = 0;
}

}  // namespace

static dim3 diag_grid(int nx, int ny, int nz, int* zc)
{
    const long tiles = (long)((nx + kDX - 1) / kDX) * ((ny + kDY - 1) / kDY);
    const long target = 32L * device_sms();   // blocks to aim for: about 4 waves of 8 per SM
    long chunks = (target + tiles - 1) / tiles;
    if (chunks > nz) chunks = nz;
    if (chunks < 1) chunks = 1;
    *zc = (int)((nz + chunks - 1) / chunks);
    chunks = (nz + *zc - 1) / *zc;
    return dim3((nx + kDX - 1) / kDX, (ny + kDY - 1) / kDY, (unsigned)chunks);
}

long diag_blocks(int nx, int ny, int nz)
{
    int zc;
    const dim3 g = diag_grid(nx, ny, nz, &zc);
    return (long)g.x * g.y * g.z;
}

template <typename T>
cudaError_t launch_diagnostics(const T* u, int nx, int ny, int nz, double h, double eps, int well, double* part,
                               unsigned* ticket, double* out, cudaStream_t s)
{
    int zc;
    const dim3 g = diag_grid(nx, ny, nz, &zc);
    k_diag<T><<<g, dim3(kDX, kDY), 0, s>>>(u, nx, ny, nz, zc, (T)(1.0 / (2.0 * h)), (T)(0.5 * eps), (T)(1.0 / eps),
                                          well, h * h * h, part, ticket, out);
    return cudaGetLastError();
}
template cudaError_t launch_diagnostics<float>(const float*, int, int, int, double, double, int, double*, unsigned*,
                                               double*, cudaStream_t);
template cudaError_t launch_diagnostics<double>(const double*, int, int, int, double, double, int, double*, unsigned*,
                                                double*, cudaStream_t);

}  // namespace pfc
