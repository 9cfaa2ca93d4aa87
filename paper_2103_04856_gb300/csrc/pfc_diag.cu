// pfc_diag.cu -- viability diagnostics of a phase field (Sec. 4.5): the
// discrepancy  h^3 sum |eps/2 |grad u|^2 - W(u)/eps|, the Cahn-Hilliard
// energy  h^3 sum (eps/2 |grad u|^2 + W(u)/eps)  (the diffuse area) and the
// extremes of u.  grad u is the periodic central difference, without xi.
//
// One pass that marches in z (HBM-bound: u is read once, 4 or 8 B/voxel);
// per-thread sums in the arithmetic type, FP64 across warps and blocks,
// combined in a fixed order by the last block to finish (ticket).
#include "pfc_device.cuh"

namespace pfc {

namespace {

constexpr int kDX = 32, kDY = 8;
constexpr int kDiagThreads = kDX * kDY;

__device__ __forceinline__ double fmax_(double a, double b) { return a > b ? a : b; }
__device__ __forceinline__ double fmin_(double a, double b) { return a < b ? a : b; }

// The per-voxel terms |eps/2 |G|^2 - W/eps| and eps/2 |G|^2 + W/eps from
// the raw differences d = u(+) - u(-) (G = d / 2h): kin = ks |d|^2 with
// ks = eps / (8 h^2), and W/eps = q wq q with q = u (1 - u), wq = 1/eps
// (wells 0/1) or q = 1 - u^2, wq = 1/(4 eps) (wells -1/1).
template <typename T>
__device__ __forceinline__ void diag_terms(T dx, T dy, T dz, T u0, T ks, T wq, int well, T& d, T& c)
{
    const T kin = ks * fma_(dx, dx, fma_(dy, dy, dz * dz));
    const T q = well == 0 ? fma_(-u0, u0, u0) : fma_(-u0, u0, T(1));
    const T qw = q * wq;
    const T e = fma_(-qw, q, kin);
    d = e < T(0) ? -e : e;
    c = fma_(qw, q, kin);
}

// FP64 beyond the thread: warp shuffles, one value per warp, one partial per
// block; the last block to arrive (ticket, no waiting) combines the partials
// in block order and writes the five results.  Called by every thread.
__device__ void diag_finish(double sd, double sc, double umax, double umin, int nblocks, int bid, double h3,
                            double* part, unsigned* ticket, double* out)
{
    double v[4] = { sd, sc, umax, umin };
    __shared__ double red[kDiagThreads / 32][4];
    __shared__ int last;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
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

// Any element type and row length.  Block (32 x 8 threads) = one (x, y)
// tile; blockIdx.z = a chunk of zc planes that every thread marches through,
// keeping u(z-1), u(z), u(z+1) of its column in registers: one new load per
// voxel from HBM, the four x/y neighbours from L1/L2.
template <typename T>
__global__ void __launch_bounds__(kDiagThreads) k_diag(const T* __restrict__ u, int nx, int ny, int nz, int zc, T ks,
                                                      T wq, int well, double h3, double* part, unsigned* ticket,
                                                      double* out)
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
            T d, s;
            diag_terms<T>(c[xp] - c[xm], c[yp] - c[ym], up - um, u0, ks, wq, well, d, s);
            sd += d;
            sc += s;
            umax = u0 > umax ? u0 : umax;
            umin = u0 < umin ? u0 : umin;
            um = u0;
            u0 = up;
        }
    }
    const int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    diag_finish((double)sd, (double)sc, (double)umax, (double)umin, nblocks, bid, h3, part, ticket, out);
}

// FP32 rows of a multiple of 4 voxels on a 16-byte aligned field of 2^31
// voxels or more (64-bit offsets; smaller grids take k_diag_rows): each
// thread owns 4 consecutive x voxels (one float4), a warp 128 voxels of a
// row, a block (32 x 8 threads) a tile of 128 x 8 columns.  Persistent grid:
// block b walks the work items b, b + gridDim.x, ... (a tile over a chunk of
// zc planes).  Each thread marches its 4 columns up z, issuing the loads of
// kB planes together (its own float4 from HBM, the y neighbours' float4 from
// L1/L2); the x neighbours are in its own float4 or its lanes' (shuffles),
// and the tile's two edge columns are loaded by the edge lanes.  A quarter
// of the load instructions of one voxel per thread, kB loads in flight.
constexpr int kB = 4;

__global__ void __launch_bounds__(kDiagThreads) k_diag4(const float* __restrict__ u, int nx, int ny, int nz, int zc,
                                                       int tiles_x, int tiles_y, int chunks, float ks, float wq,
                                                       int well, double h3, double* part, unsigned* ticket,
                                                       double* out)
{
    const long pls = (long)nx * ny;
    const int lx = threadIdx.x;
    float sd = 0.f, sc = 0.f, umax = -INFINITY, umin = INFINITY;
    const int items = tiles_x * tiles_y * chunks;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int ch = it % chunks, t = it / chunks;
        const int x4 = (t % tiles_x) * (4 * kDX) + 4 * lx, y = (t / tiles_x) * kDY + threadIdx.y;
        const int z0 = ch * zc, z1 = min(nz, z0 + zc);
        // lanes past a ragged edge work on a valid (clamped) column and count nothing
        const bool live = x4 < nx && y < ny;
        const int xq = min(x4, nx - 4), yl = min(y, ny - 1);
        // whether lane -1 / +1 holds the voxel left of x4 / right of x4 + 3
        const bool sh_l = lx > 0, sh_r = lx < kDX - 1 && x4 + 4 < nx;
        const long ym = (long)(nbr(yl, -1, ny) - yl) * nx, yp = (long)(nbr(yl, 1, ny) - yl) * nx;
        const int xl = nbr(xq, -1, nx) - xq, xr = nbr(xq, 4, nx) - xq;
        const float* col = u + (long)yl * nx + xq;
        float4 um = *reinterpret_cast<const float4*>(col + (long)nbr(z0, -1, nz) * pls);
        float4 u0 = *reinterpret_cast<const float4*>(col + (long)z0 * pls);
        for (int zb = z0; zb < z1; zb += kB) {
            const int n = min(kB, z1 - zb);   // uniform across the block: the shuffles see full warps
            float4 up[kB], vp[kB], vm[kB];
            float el[kB], er[kB];
#pragma unroll
            for (int k = 0; k < kB; ++k) {
                if (k < n) {
                    const int z = zb + k;
                    const float* c = col + (long)z * pls;
                    up[k] = *reinterpret_cast<const float4*>(col + (long)(z + 1 == nz ? 0 : z + 1) * pls);
                    vp[k] = *reinterpret_cast<const float4*>(c + yp);
                    vm[k] = *reinterpret_cast<const float4*>(c + ym);
                    el[k] = sh_l ? 0.f : c[xl];
                    er[k] = sh_r ? 0.f : c[xr];
                }
            }
#pragma unroll
            for (int k = 0; k < kB; ++k) {
                if (k < n) {
                    const float left = __shfl_up_sync(0xffffffffu, u0.w, 1);
                    const float right = __shfl_down_sync(0xffffffffu, u0.x, 1);
                    const float l = sh_l ? left : el[k], r = sh_r ? right : er[k];
                    float d0, c0, d1, c1, d2, c2, d3, c3;
                    diag_terms<float>(u0.y - l, vp[k].x - vm[k].x, up[k].x - um.x, u0.x, ks, wq, well, d0, c0);
                    diag_terms<float>(u0.z - u0.x, vp[k].y - vm[k].y, up[k].y - um.y, u0.y, ks, wq, well, d1, c1);
                    diag_terms<float>(u0.w - u0.y, vp[k].z - vm[k].z, up[k].z - um.z, u0.z, ks, wq, well, d2, c2);
                    diag_terms<float>(r - u0.z, vp[k].w - vm[k].w, up[k].w - um.w, u0.w, ks, wq, well, d3, c3);
                    if (live) {
                        sd += (d0 + d1) + (d2 + d3);
                        sc += (c0 + c1) + (c2 + c3);
                        umax = fmaxf(umax, fmaxf(fmaxf(u0.x, u0.y), fmaxf(u0.z, u0.w)));
                        umin = fminf(umin, fminf(fminf(u0.x, u0.y), fminf(u0.z, u0.w)));
                    }
                    um = u0;
                    u0 = up[k];
                }
            }
        }
    }
    diag_finish((double)sd, (double)sc, (double)umax, (double)umin, gridDim.x, blockIdx.x, h3, part, ticket, out);
}

// The FP32 kernel for grids of fewer than 2^31 voxels (rows of a multiple of
// 4 voxels, 16-byte aligned field).  Each thread owns one float4 of x
// columns in R consecutive rows, a block (32 x 8 threads) a tile of 128 x 8R
// columns; persistent grid over work items (a tile over a chunk of zc
// planes).  The thread marches up z keeping u(z-1) and u(z) of its rows in
// registers and issues the loads of KB planes together: its rows' float4 at
// z+1 (from HBM), the rows below and above its own at z (L1/L2), one voxel
// beyond a warp's edge for the edge lanes; the x neighbours inside the warp
// come by shuffles, the y neighbours between its rows from its own
// registers.  Per load one address instruction (32-bit plane offsets, one
// base pointer per row).  The per-voxel terms are scaled by 1/ks (ks = eps /
// 8h^2), the sums by ks at the end, and the double well is a template
// parameter: about 14 arithmetic instructions per voxel.
template <int WELL>
__device__ __forceinline__ void diag_terms_k(float dx, float dy, float dz, float u0, float wk, float& d, float& c)
{
    const float g2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float q = WELL == 0 ? fmaf(-u0, u0, u0) : fmaf(-u0, u0, 1.f);
    const float qw = q * wk;
    const float e = fmaf(-qw, q, g2);
    d = fabsf(e);
    c = fmaf(qw, q, g2);
}

template <int R, int KB, int WELL>
__global__ void __launch_bounds__(kDiagThreads) k_diag_rows(const float* __restrict__ u, int nx, int ny, int nz,
                                                            int zc, int tiles_x, int chunks, float wk, float ks,
                                                            double h3, double* part, unsigned* ticket, double* out)
{
    static_assert(R >= 1 && R <= 4, "one to four rows per thread");
    const int pls = nx * ny;   // fewer than 2^31 voxels in all
    const int lx = threadIdx.x;
    float sd = 0.f, sc = 0.f, umax = -INFINITY, umin = INFINITY;
    const int items = tiles_x * ((ny + kDY * R - 1) / (kDY * R)) * chunks;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int ch = it % chunks, t = it / chunks;
        const int x4 = (t % tiles_x) * (4 * kDX) + 4 * lx, yb = (t / tiles_x) * (kDY * R) + R * threadIdx.y;
        const int z0 = ch * zc, z1 = min(nz, z0 + zc);
        // lanes and rows past a ragged edge count nothing.  A lane past the
        // row's end works on the columns x4 modulo nx, so that the lane
        // before it finds its right neighbour there; a row past the edge
        // reads the upper neighbour of the row before it instead, which that
        // row then takes as its own
        const int xq = x4 < nx ? x4 : x4 % nx, y0 = min(yb, ny - 1);
        bool live[R];
        int yr[R];
        yr[0] = y0;
        live[0] = x4 < nx && yb < ny;
#pragma unroll
        for (int r = 1; r < R; ++r) {
            yr[r] = yb + r < ny ? yb + r : nbr(yr[r - 1], 1, ny);
            live[r] = x4 < nx && yb + r < ny;
        }
        const float* prow[R];
#pragma unroll
        for (int r = 0; r < R; ++r) prow[r] = u + yr[r] * nx + xq;
        const float* pym = u + nbr(y0, -1, ny) * nx + xq;
        const float* pyp = u + nbr(yr[R - 1], 1, ny) * nx + xq;
        // x neighbours: lane - 1 holds the voxel left of x4, lane + 1 the one
        // right of x4 + 3 (periodic, through the wrapped columns); lanes 0
        // and 31 load the one beyond the warp's edge
        const bool need = lx == 0 || lx == kDX - 1;
        const int eoff = lx == 0 ? nbr(xq, -1, nx) - xq : nbr(xq + 3, 1, nx) - xq;
        float4 m[R], c[R];
        int zo = z0 * pls;
        {
            const int om = nbr(z0, -1, nz) * pls;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                m[r] = *reinterpret_cast<const float4*>(prow[r] + om);
                c[r] = *reinterpret_cast<const float4*>(prow[r] + zo);
            }
        }
        for (int zb = z0; zb < z1; zb += KB) {
            const int n = min(KB, z1 - zb);   // uniform across the block: the shuffles see full warps
            float4 up[KB][R], lo[KB], hi[KB];
            float ev[KB][R];
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                if (k < n) {
                    const int o = zo + k * pls, on = zb + k + 1 == nz ? 0 : o + pls;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        up[k][r] = *reinterpret_cast<const float4*>(prow[r] + on);
                        ev[k][r] = need ? prow[r][o + eoff] : 0.f;
                    }
                    lo[k] = *reinterpret_cast<const float4*>(pym + o);
                    hi[k] = *reinterpret_cast<const float4*>(pyp + o);
                }
            }
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                if (k < n) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const float4 a = c[r];
                        const float4 b = r == 0 ? lo[k] : c[r > 0 ? r - 1 : 0];        // the row below
                        const float4 t4 = r == R - 1 ? hi[k] : c[r + 1 < R ? r + 1 : r];   // the row above
                        const float left = __shfl_up_sync(0xffffffffu, a.w, 1);
                        const float right = __shfl_down_sync(0xffffffffu, a.x, 1);
                        const float l = lx == 0 ? ev[k][r] : left;
                        const float rr = lx == kDX - 1 ? ev[k][r] : right;
                        float d0, c0, d1, c1, d2, c2, d3, c3;
                        diag_terms_k<WELL>(a.y - l, t4.x - b.x, up[k][r].x - m[r].x, a.x, wk, d0, c0);
                        diag_terms_k<WELL>(a.z - a.x, t4.y - b.y, up[k][r].y - m[r].y, a.y, wk, d1, c1);
                        diag_terms_k<WELL>(a.w - a.y, t4.z - b.z, up[k][r].z - m[r].z, a.z, wk, d2, c2);
                        diag_terms_k<WELL>(rr - a.z, t4.w - b.w, up[k][r].w - m[r].w, a.w, wk, d3, c3);
                        if (live[r]) {
                            sd += (d0 + d1) + (d2 + d3);
                            sc += (c0 + c1) + (c2 + c3);
                            umax = fmaxf(umax, fmaxf(fmaxf(a.x, a.y), fmaxf(a.z, a.w)));
                            umin = fminf(umin, fminf(fminf(a.x, a.y), fminf(a.z, a.w)));
                        }
                    }
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        m[r] = c[r];
                        c[r] = up[k][r];
                    }
                }
            }
            zo += n * pls;
        }
    }
    diag_finish((double)sd * ks, (double)sc * ks, (double)umax, (double)umin, gridDim.x, blockIdx.x, h3, part,
                ticket, out);
}

}  // namespace

// The scalar kernel's grid: (x, y) tiles times z chunks, about 4 waves of 8
// blocks per SM.
static dim3 diag_grid(int nx, int ny, int nz, int* zc)
{
    const long tiles = (long)((nx + kDX - 1) / kDX) * ((ny + kDY - 1) / kDY);
    const long target = 32L * device_sms();
    long chunks = (target + tiles - 1) / tiles;
    if (chunks > nz) chunks = nz;
    if (chunks < 1) chunks = 1;
    *zc = (int)((nz + chunks - 1) / chunks);
    chunks = (nz + *zc - 1) / *zc;
    return dim3((nx + kDX - 1) / kDX, (ny + kDY - 1) / kDY, (unsigned)chunks);
}

// The float4 kernel: work items of up to 32 planes (more, shorter items when
// the grid is small, so that each block walks several), one resident wave
// of blocks.
struct Diag4Geom {
    int tiles_x, tiles_y, chunks, zc, blocks;
};
static int diag4_blocks_per_sm()
{
    static int cached = 0;
    if (!cached) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_diag4, kDiagThreads, 0) != cudaSuccess || n < 1) {
            (void)cudaGetLastError();
            n = 2;
        }
        cached = n;
    }
    return cached;
}
static Diag4Geom diag4_geom(int nx, int ny, int nz)
{
    Diag4Geom g;
    g.tiles_x = (nx + 4 * kDX - 1) / (4 * kDX);
    g.tiles_y = (ny + kDY - 1) / kDY;
    const long tiles = (long)g.tiles_x * g.tiles_y;
    const long wave = (long)diag4_blocks_per_sm() * device_sms();
    long chunks = (nz + 31) / 32;
    if (tiles * chunks < 8 * wave) chunks = (8 * wave + tiles - 1) / tiles;
    if (chunks > nz) chunks = nz;
    g.zc = (int)((nz + chunks - 1) / chunks);
    g.chunks = (nz + g.zc - 1) / g.zc;
    const long items = tiles * g.chunks;
    g.blocks = (int)(items < wave ? items : wave);
    return g;
}

// The row kernel: two rows per thread, four planes of loads issued together
// (k_diag_rows<kRows, kPlanes, well>: 121 registers, two blocks per SM);
// grids of fewer than 2^31 voxels.  Measured on a 512^3 field: 131 us
// (4.1 TB/s); one row and four planes 255 us (spills at three blocks per
// SM), two rows and two planes 170 us, four rows and two planes 135 us.
// Staging the planes in a shared-memory ring with cp.async (no registers
// held by loads) hid the latency but issued 20 % more instructions: 144 us.
// Packed FP32 (FFMA2) pairs of voxels: 135-172 us (the pairs of x
// differences need register moves).  Bulk L2 prefetches of each warp's rows
// 4-16 planes ahead: 154-164 us.  Tiles of 256 or 512 columns (warps side by
// side in x, for longer contiguous reads per plane): 133-138 us.  Bands of
// 16 full rows staged plane by plane in shared memory by bulk asynchronous
// copies (one issuing thread, six slots, 16.7 instructions per voxel): 132 us,
// its warps waiting on the copies.
constexpr int kRows = 2, kPlanes = 4;
template <int WELL>
static int diag_rows_blocks_per_sm()
{
    static int cached = 0;
    if (!cached) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_diag_rows<kRows, kPlanes, WELL>, kDiagThreads, 0) !=
                cudaSuccess ||
            n < 1) {
            (void)cudaGetLastError();
            n = 2;
        }
        cached = n;
    }
    return cached;
}
static bool diag_rows_fits(int nx, int ny, int nz) { return (long long)nx * ny * nz < (1LL << 31); }
static Diag4Geom diag_rows_geom(int nx, int ny, int nz, int well)
{
    Diag4Geom g;
    g.tiles_x = (nx + 4 * kDX - 1) / (4 * kDX);
    g.tiles_y = (ny + kDY * kRows - 1) / (kDY * kRows);
    const long tiles = (long)g.tiles_x * g.tiles_y;
    const long wave = (long)(well == 0 ? diag_rows_blocks_per_sm<0>() : diag_rows_blocks_per_sm<1>()) * device_sms();
    long chunks = (nz + 31) / 32;
    if (tiles * chunks < 8 * wave) chunks = (8 * wave + tiles - 1) / tiles;
    if (chunks > nz) chunks = nz;
    g.zc = (int)((nz + chunks - 1) / chunks);
    g.chunks = (nz + g.zc - 1) / g.zc;
    const long items = tiles * g.chunks;
    g.blocks = (int)(items < wave ? items : wave);
    return g;
}

long diag_blocks(int nx, int ny, int nz)
{
    int zc;
    const dim3 g = diag_grid(nx, ny, nz, &zc);
    long a = (long)g.x * g.y * g.z;
    const long b = diag4_geom(nx, ny, nz).blocks;
    if (b > a) a = b;
    for (int well = 0; well < 2; ++well) {
        const long c = diag_rows_geom(nx, ny, nz, well).blocks;
        if (c > a) a = c;
    }
    return a;
}

template <typename T>
cudaError_t launch_diagnostics(const T* u, int nx, int ny, int nz, double h, double eps, int well, double* part,
                               unsigned* ticket, double* out, cudaStream_t s)
{
    const double ks = eps / (8.0 * h * h), wq = well == 0 ? 1.0 / eps : 0.25 / eps;
    if (sizeof(T) == 4 && nx % 4 == 0 && ((uintptr_t)u) % 16 == 0 && diag_rows_fits(nx, ny, nz)) {
        const Diag4Geom g = diag_rows_geom(nx, ny, nz, well);
        const float wk = (float)(wq / ks);
        if (well == 0)
            k_diag_rows<kRows, kPlanes, 0><<<g.blocks, dim3(kDX, kDY), 0, s>>>(
                (const float*)u, nx, ny, nz, g.zc, g.tiles_x, g.chunks, wk, (float)ks, h * h * h, part, ticket, out);
        else
            k_diag_rows<kRows, kPlanes, 1><<<g.blocks, dim3(kDX, kDY), 0, s>>>(
                (const float*)u, nx, ny, nz, g.zc, g.tiles_x, g.chunks, wk, (float)ks, h * h * h, part, ticket, out);
        return cudaGetLastError();
    }
    if (sizeof(T) == 4 && nx % 4 == 0 && ((uintptr_t)u) % 16 == 0) {
        const Diag4Geom g = diag4_geom(nx, ny, nz);
        k_diag4<<<g.blocks, dim3(kDX, kDY), 0, s>>>((const float*)u, nx, ny, nz, g.zc, g.tiles_x, g.tiles_y,
                                                    g.chunks, (float)ks, (float)wq, well, h * h * h, part, ticket, out);
        return cudaGetLastError();
    }
    int zc;
    const dim3 g = diag_grid(nx, ny, nz, &zc);
    k_diag<T><<<g, dim3(kDX, kDY), 0, s>>>(u, nx, ny, nz, zc, (T)ks, (T)wq, well, h * h * h, part, ticket, out);
    return cudaGetLastError();
}
template cudaError_t launch_diagnostics<float>(const float*, int, int, int, double, double, int, double*, unsigned*,
                                               double*, cudaStream_t);
template cudaError_t launch_diagnostics<double>(const double*, int, int, int, double, double, int, double*, unsigned*,
                                                double*, cudaStream_t);

}  // namespace pfc
