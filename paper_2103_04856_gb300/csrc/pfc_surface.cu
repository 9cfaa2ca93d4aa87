// pfc_surface.cu -- cells of the curvature diagram (Sec. 4.1, eq.
// curva_diagram): the surface {u = level} triangulated by marching
// tetrahedra, each triangle giving (area, kappa1, kappa2) with the diffuse
// curvatures (eqs. kepsa/kepsb, k_curvatures) interpolated trilinearly at
// its barycenter.
//
// Every voxel (x, y, z) owns the cube spanning to (x+1, y+1, z+1) (periodic)
// and splits it into the six tetrahedra of the Freudenthal triangulation
// (from corner 000 to corner 111 along the axes in each of the six orders,
// so neighbouring cubes agree on their shared faces).  In a tetrahedron
// with one corner on its own side of the level the surface is a triangle
// around that corner; with two on each side it is a quadrilateral, split
// into two triangles along a fixed diagonal.  Edge points interpolate
// u - level linearly.
//
// Records come out in cube order (z, y, x), then tetrahedron order, then
// triangle order, which makes the output deterministic: pass 1 counts the
// triangles of every cube and sums them per block, a one-block scan turns
// the block sums into offsets, pass 2 recomputes the cubes and writes.
#include "pfc_device.cuh"

namespace pfc {

namespace {

constexpr int kSurfThreads = 256;
constexpr int kScanThreads = 1024;

// axis orders of the six tetrahedra
__constant__ unsigned char c_axes[6][3] = { { 0, 1, 2 }, { 0, 2, 1 }, { 1, 0, 2 },
                                            { 1, 2, 0 }, { 2, 0, 1 }, { 2, 1, 0 } };

// corner c = i + 2j + 4k of the cube at voxel (x, y, z)
template <typename T>
__device__ __forceinline__ void load_corners(const T* __restrict__ u, int x, int y, int z, int nx, int ny, int nz,
                                             T v[8], long idx[8])
{
    const int x1 = x + 1 == nx ? 0 : x + 1, y1 = y + 1 == ny ? 0 : y + 1, z1 = z + 1 == nz ? 0 : z + 1;
    const long pls = (long)nx * ny;
    const long r00 = (long)z * pls + (long)y * nx, r10 = (long)z * pls + (long)y1 * nx;
    const long r01 = (long)z1 * pls + (long)y * nx, r11 = (long)z1 * pls + (long)y1 * nx;
    idx[0] = r00 + x; idx[1] = r00 + x1; idx[2] = r10 + x; idx[3] = r10 + x1;
    idx[4] = r01 + x; idx[5] = r01 + x1; idx[6] = r11 + x; idx[7] = r11 + x1;
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = u[idx[c]];
}

__device__ __forceinline__ void tet_corners(int t, int w[4])
{
    w[0] = 0;
    w[1] = 1 << c_axes[t][0];
    w[2] = w[1] | (1 << c_axes[t][1]);
    w[3] = 7;
}

// triangles of a cube whose corners above the level form the bit mask `above`
__device__ __forceinline__ int cube_triangles(unsigned above)
{
    int n = 0;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
        int w[4];
        tet_corners(t, w);
        const int np = ((above >> w[0]) & 1) + ((above >> w[1]) & 1) + ((above >> w[2]) & 1) + ((above >> w[3]) & 1);
        n += np == 2 ? 2 : (np == 1 || np == 3 ? 1 : 0);
    }
    return n;
}

template <typename T>
__device__ __forceinline__ unsigned above_mask(const T v[8], T level)
{
    unsigned m = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) m |= (v[c] > level ? 1u : 0u) << c;
    return m;
}

__device__ __forceinline__ long cube_coords(long i, int nx, int ny, int* x, int* y, int* z)
{
    const long pls = (long)nx * ny;
    *z = (int)(i / pls);
    const long r = i - (long)(*z) * pls;
    *y = (int)(r / nx);
    *x = (int)(r - (long)(*y) * nx);
    return i;
}

// block sum of per-thread counts; thread 0 gets the total
__device__ __forceinline__ unsigned block_sum_u(unsigned v, unsigned* sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    unsigned t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kSurfThreads / 32; ++w) t += sh[w];
    return t;
}

template <typename T>
__global__ void __launch_bounds__(kSurfThreads) k_surf_count(const T* __restrict__ u, int nx, int ny, int nz,
                                                             T level, unsigned* __restrict__ block_counts)
{
    __shared__ unsigned sh[kSurfThreads / 32];
    const long n = (long)nx * ny * nz;
    const long i = (long)blockIdx.x * kSurfThreads + threadIdx.x;
    unsigned cnt = 0;
    if (i < n) {
        int x, y, z;
        cube_coords(i, nx, ny, &x, &y, &z);
        T v[8];
        long idx[8];
        load_corners(u, x, y, z, nx, ny, nz, v, idx);
        cnt = (unsigned)cube_triangles(above_mask(v, level));
    }
    const unsigned t = block_sum_u(cnt, sh);
    if (threadIdx.x == 0) block_counts[blockIdx.x] = t;
}

// Exclusive scan of nb block counts into offsets (one block); total at offsets[nb].
__global__ void __launch_bounds__(kScanThreads) k_surf_scan(const unsigned* __restrict__ counts, long nb,
                                                            long long* __restrict__ offsets)
{
    __shared__ long long part[kScanThreads];
    const long per = (nb + kScanThreads - 1) / kScanThreads;
    const long b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
    long long s = 0;
    for (long b = b0; b < b1; ++b) s += counts[b];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {          // 1024 partial sums, in order
        long long acc = 0;
        for (int k = 0; k < kScanThreads; ++k) {
            const long long v = part[k];
            part[k] = acc;
            acc += v;
        }
        offsets[nb] = acc;
    }
    __syncthreads();
    long long acc = part[threadIdx.x];
    for (long b = b0; b < b1; ++b) {
        offsets[b] = acc;
        acc += counts[b];
    }
}

template <typename T>
__device__ __forceinline__ void edge_point(const T f[8], int a, int b, T q[3])
{
    const T t = f[a] / (f[a] - f[b]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T qa = (T)((a >> k) & 1), qb = (T)((b >> k) & 1);
        q[k] = qa + t * (qb - qa);
    }
}

template <typename T>
__device__ __forceinline__ void write_cell(const T P0[3], const T P1[3], const T P2[3], const T k1c[8],
                                           const T k2c[8], T h2, long long slot, long long cap, T* __restrict__ cells)
{
    if (slot >= cap) return;
    T a[3], b[3], bc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a[k] = P1[k] - P0[k];
        b[k] = P2[k] - P0[k];
        bc[k] = (P0[k] + P1[k] + P2[k]) / T(3);
    }
    const T cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
    const T area = T(0.5) * sqrt_(cx * cx + cy * cy + cz * cz) * h2;
    T s1 = 0, s2 = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const T wx = (c & 1) ? bc[0] : T(1) - bc[0];
        const T wy = ((c >> 1) & 1) ? bc[1] : T(1) - bc[1];
        const T wz = ((c >> 2) & 1) ? bc[2] : T(1) - bc[2];
        const T w = wx * wy * wz;
        s1 += w * k1c[c];
        s2 += w * k2c[c];
    }
    cells[3 * slot + 0] = area;
    cells[3 * slot + 1] = s1;
    cells[3 * slot + 2] = s2;
}

template <typename T>
__global__ void __launch_bounds__(kSurfThreads) k_surf_emit(const T* __restrict__ u, const T* __restrict__ k1,
                                                            const T* __restrict__ k2, int nx, int ny, int nz, T level,
                                                            T h2, const long long* __restrict__ offsets,
                                                            long long cap, T* __restrict__ cells)
{
    __shared__ unsigned sh[kSurfThreads];
    const long n = (long)nx * ny * nz;
    const long i = (long)blockIdx.x * kSurfThreads + threadIdx.x;
    T v[8];
    long idx[8];
    unsigned above = 0;
    int cnt = 0;
    if (i < n) {
        int x, y, z;
        cube_coords(i, nx, ny, &x, &y, &z);
        load_corners(u, x, y, z, nx, ny, nz, v, idx);
        above = above_mask(v, level);
        cnt = cube_triangles(above);
    }
    // exclusive scan of the block's counts (Hillis-Steele in shared memory)
    sh[threadIdx.x] = (unsigned)cnt;
    __syncthreads();
    for (int o = 1; o < kSurfThreads; o <<= 1) {
        const unsigned add = threadIdx.x >= o ? sh[threadIdx.x - o] : 0u;
        __syncthreads();
        sh[threadIdx.x] += add;
        __syncthreads();
    }
    if (cnt == 0) return;
    long long slot = offsets[blockIdx.x] + (long long)(sh[threadIdx.x] - (unsigned)cnt);
    T f[8], k1c[8], k2c[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        f[c] = v[c] - level;
        k1c[c] = k1[idx[c]];
        k2c[c] = k2[idx[c]];
    }
    for (int t = 0; t < 6; ++t) {
        int w[4];
        tet_corners(t, w);
        int pos[4], neg[4], np = 0, nn = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if ((above >> w[k]) & 1) pos[np++] = w[k];
            else neg[nn++] = w[k];
        }
        T A[3], B[3], C[3], D[3];
        if (np == 1) {
            edge_point(f, pos[0], neg[0], A);
            edge_point(f, pos[0], neg[1], B);
            edge_point(f, pos[0], neg[2], C);
            write_cell(A, B, C, k1c, k2c, h2, slot++, cap, cells);
        } else if (np == 3) {
            edge_point(f, pos[0], neg[0], A);
            edge_point(f, pos[1], neg[0], B);
            edge_point(f, pos[2], neg[0], C);
            write_cell(A, B, C, k1c, k2c, h2, slot++, cap, cells);
        } else if (np == 2) {
            edge_point(f, pos[0], neg[0], A);
            edge_point(f, pos[0], neg[1], B);
            edge_point(f, pos[1], neg[1], C);
            edge_point(f, pos[1], neg[0], D);
            write_cell(A, B, C, k1c, k2c, h2, slot++, cap, cells);
            write_cell(A, C, D, k1c, k2c, h2, slot++, cap, cells);
        }
    }
}

// Area-weighted 2-D histogram of (kappa1, kappa2) over [lo, hi)^2, values
// outside clamped into the edge bins; hist[b1 * nbins + b2] (FP64 atomics).
template <typename T>
__global__ void k_curv_hist(const T* __restrict__ cells, long long n, int nbins, double lo, double inv_w,
                            double* __restrict__ hist)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double a = (double)cells[3 * i], c1 = (double)cells[3 * i + 1], c2 = (double)cells[3 * i + 2];
        int b1 = (int)floor((c1 - lo) * inv_w), b2 = (int)floor((c2 - lo) * inv_w);
        b1 = b1 < 0 ? 0 : (b1 >= nbins ? nbins - 1 : b1);
        b2 = b2 < 0 ? 0 : (b2 >= nbins ? nbins - 1 : b2);
        atomicAdd(hist + (size_t)b1 * nbins + b2, a);
    }
}

}  // namespace

long surface_blocks(long n) { return (n + kSurfThreads - 1) / kSurfThreads; }

template <typename T>
cudaError_t launch_surface_cells(const T* u, const T* k1, const T* k2, int nx, int ny, int nz, double h, double level,
                                 unsigned* block_counts, long long* offsets, T* cells, long long cap, cudaStream_t s)
{
    const long n = (long)nx * ny * nz;
    const long nb = surface_blocks(n);
    k_surf_count<T><<<(unsigned)nb, kSurfThreads, 0, s>>>(u, nx, ny, nz, (T)level, block_counts);
    k_surf_scan<<<1, kScanThreads, 0, s>>>(block_counts, nb, offsets);
    k_surf_emit<T><<<(unsigned)nb, kSurfThreads, 0, s>>>(u, k1, k2, nx, ny, nz, (T)level, (T)(h * h), offsets, cap,
                                                         cells);
    return cudaGetLastError();
}
template cudaError_t launch_surface_cells<float>(const float*, const float*, const float*, int, int, int, double,
                                                 double, unsigned*, long long*, float*, long long, cudaStream_t);
template cudaError_t launch_surface_cells<double>(const double*, const double*, const double*, int, int, int, double,
                                                  double, unsigned*, long long*, double*, long long, cudaStream_t);

template <typename T>
cudaError_t launch_curvature_histogram(const T* cells, long long n, int nbins, double lo, double hi, double* hist,
                                       cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(double) * (size_t)nbins * nbins, s);
    if (e != cudaSuccess || n <= 0) return e;
    long long b = (n + 255) / 256;
    if (b > 16LL * device_sms()) b = 16LL * device_sms();
    k_curv_hist<T><<<(unsigned)b, 256, 0, s>>>(cells, n, nbins, lo, nbins / (hi - lo), hist);
    return cudaGetLastError();
}
template cudaError_t launch_curvature_histogram<float>(const float*, long long, int, double, double, double*,
                                                       cudaStream_t);
template cudaError_t launch_curvature_histogram<double>(const double*, long long, int, double, double, double*,
                                                        cudaStream_t);

}  // namespace pfc
