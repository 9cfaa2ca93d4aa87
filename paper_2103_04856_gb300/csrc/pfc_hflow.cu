// pfc_hflow.cu -- the paper's generator (Alg. 1, Sec. 4.1): the H^-1 flow of
// F_eps written as an L2 flow on a periodic vector field A through the change
// of variable u = div A + m0 (eq. change_var), a small Gaussian blur of u
// before the energy, and Adam on A.  One step:
//   div    : A (3 fields)  -> u = div A + m0          (plus the mass of u)
//   blur   : u -> k * u     (three periodic 1-D passes, x, y, z)
//   sweep  : k * u -> E, g = dF/du                    (the fused kernel)
//   blur   : g -> k * g     (the blur is symmetric and periodic: self-adjoint)
//   adam   : dG/dA_c = -(k*g)(j+e_c) + (k*g)(j-e_c), over 2h; moments; A update
// The div, blur and Adam kernels are memory-bound: grid-stride loops over the
// voxels (FP32 sums per thread, FP64 only across warps and blocks: FP64 runs
// at a small fraction of the FP32 rate on this GPU); for FP32 rows of up to
// 128 values div and the x pass of the blur share one kernel (shuffles across
// a warp), the y and z passes are register windows along each line, and other
// radii or precisions take shared-memory tiles.  The sweep is the issue-bound
// kernel of pfc_fused_kernel.cuh.  A batch runs every kernel once for up to
// 64 flows on grids of one size (instances along grid y).
#include <cuda_runtime.h>

#include <math.h>
#include <stdio.h>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pfc.h"
#include "pfc_device.cuh"

using namespace pfc;

namespace pfc {
void set_last_error(const char* msg);
}

namespace {

constexpr int kMaxRadius = 32;
constexpr int kThreads = 128;
constexpr int kTileAx = 64;        // blur outputs per tile along the blurred axis

// Reduction slots of the flow's own kernels (the sweep has its own).
enum { H_MASS = 0, H_GMAX, H_GABS, NH };

struct Flow {
    int nx, ny, nz;
    long n;
    double sg;          // 1 / (2h)
    double m0;
    const void* mf;     // null, or m(x) (N values of the arithmetic type, Sec. 5.2)
    double lr, beta1, beta2, adam_eps;
    double* part;       // [blocks][NH] FP64 partials of the flow kernels
    unsigned* ints;     // [0] ticket, [1] Adam step t, [2] trace row
    double* hs;         // [NH] finished sums: mass, max|dG/dA|, mean|dG/dA|
    const double* sweep_scal;   // the sweep's scalars (energy)
    double* trace;      // [cap][5]
    int trace_cap;
};

struct Weights {
    int R;
    float wf[2 * kMaxRadius + 1];
    double wd[2 * kMaxRadius + 1];
};

template <typename T>
__device__ __forceinline__ T wget(const Weights& w, int j);
template <>
__device__ __forceinline__ float wget<float>(const Weights& w, int j) { return w.wf[j]; }
template <>
__device__ __forceinline__ double wget<double>(const Weights& w, int j) { return w.wd[j]; }

template <typename T> __device__ __forceinline__ T pow_(T b, T e);
template <> __device__ __forceinline__ float pow_<float>(float b, float e) { return powf(b, e); }
template <> __device__ __forceinline__ double pow_<double>(double b, double e) { return pow(b, e); }

// Block totals of (sum, max) in the arithmetic type per thread, FP64 across
// warps and blocks; the last block combines all partials in a fixed order
// and runs `fin` with the totals (thread 0).  The blocks of one instance are
// the grid's x dimension (a batch puts its instances along y).
template <typename T, class Fin>
__device__ void flow_finish(const Flow& f, T a0, T a1, Fin fin)
{
    __shared__ double red[2 * (kThreads / 32)];
    __shared__ int last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nblocks = gridDim.x;
    const int bid = blockIdx.x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 = fmax(a1, __shfl_xor_sync(0xffffffffu, a1, o));
    }
    if (lane == 0) { red[2 * wid] = (double)a0; red[2 * wid + 1] = (double)a1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0, s1 = 0;
        for (int w = 0; w < kThreads / 32; ++w) { s0 += red[2 * w]; s1 = fmax(s1, red[2 * w + 1]); }
        double* p = f.part + (size_t)bid * 2;
        p[0] = s0; p[1] = s1;
        __threadfence();
        last = atomicAdd(&f.ints[0], 1u) == (unsigned)nblocks - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s0 = 0, s1 = 0;
    for (int b = threadIdx.x; b < nblocks; b += kThreads) {
        s0 += __ldcg(f.part + (size_t)b * 2);
        s1 = fmax(s1, __ldcg(f.part + (size_t)b * 2 + 1));
    }
    s0 = warp_sum(s0);
    s1 = warp_max(s1);
    __syncthreads();
    if (lane == 0) { red[2 * wid] = s0; red[2 * wid + 1] = s1; }
    __syncthreads();
    if (threadIdx.x != 0) return;
    s0 = 0; s1 = 0;
    for (int w = 0; w < kThreads / 32; ++w) { s0 += red[2 * w]; s1 = fmax(s1, red[2 * w + 1]); }
    fin(s0, s1);
    __threadfence();
    f.ints[0] = 0;
}

// Launch of the pointwise kernels: a 1-D grid of at most 8 blocks per SM
// striding over the flattened voxel index; each thread carries its (x, y, z)
// and advances it by the stride's own (sx, sy, sz) with two carries.
inline long flow_blocks() { return 8L * device_sms(); }
inline dim3 flow_grid(long n)
{
    const long b = (n + kThreads - 1) / kThreads, cap = flow_blocks();
    return dim3((unsigned)(b < cap ? b : cap));
}

// Blocks per instance when n_inst instances share a launch (instances along
// grid y): about two waves in all, so that each block strides over enough
// work to pay for its closing reduction (a fence and a ticket per block).
inline unsigned inst_blocks(long n, int n_inst)
{
    const unsigned b = flow_grid(n).x;
    if (n_inst <= 1) return b;
    const unsigned cap = (unsigned)((2 * flow_blocks() + n_inst - 1) / n_inst);
    return b < cap ? b : cap;
}


// Launch descriptors: one flow (MAXI = 1) or a batch of up to BATCH_MAX
// flows on grids of one size, instance k = blockIdx.y (blockIdx.z / zb for
// the blur), passed by value and read from the constant bank.
template <typename T, int MAXI>
struct DivL {
    Flow f[MAXI];
    const T* A[MAXI];
    T* u[MAXI];
    int want_mass;
};
template <typename T, int MAXI>
struct AdamL {
    Flow f[MAXI];
    const T* gb[MAXI];
    T* A[MAXI];
    T* m[MAXI];
    T* v[MAXI];
    int only_grad;
};
template <typename T, int MAXI>
struct BlurL {
    const T* in[MAXI];
    T* out[MAXI];
    int nx, ny, nz;
    int zb;             // z blocks per instance (tiled kernel)
    int n;              // instances
    int chunk, nchunks; // line pieces per thread (window kernel)
    Weights w;
};

// u = div A + m0 (or + m(x)), periodic central differences (eq.
// change_var); mass of u.
template <typename T, int MAXI>
__global__ void __launch_bounds__(kThreads) k_div(const __grid_constant__ DivL<T, MAXI> L)
{
    const Flow& f = L.f[blockIdx.y];
    const T* __restrict__ A = L.A[blockIdx.y];
    T* __restrict__ u = L.u[blockIdx.y];
    const int want_mass = L.want_mass;
    const long n = f.n, pls = (long)f.nx * f.ny;
    T ms = 0;
    for (Walk w(f.nx, f.ny, (long)blockIdx.x * kThreads + threadIdx.x, (long)gridDim.x * kThreads); w.i < n;
         w.next(f.nx, f.ny)) {
        const long row = w.i - w.x, pl = (long)w.z * pls, col = w.i - pl;
        const T dx = A[row + nbr(w.x, 1, f.nx)] - A[row + nbr(w.x, -1, f.nx)];
        const T dy = A[n + pl + (long)nbr(w.y, 1, f.ny) * f.nx + w.x] - A[n + pl + (long)nbr(w.y, -1, f.ny) * f.nx + w.x];
        const T dz = A[2 * n + (long)nbr(w.z, 1, f.nz) * pls + col] - A[2 * n + (long)nbr(w.z, -1, f.nz) * pls + col];
        const T m = f.mf ? ((const T*)f.mf)[w.i] : (T)f.m0;
        const T v = (T)f.sg * (dx + dy + dz) + m;
        u[w.i] = v;
        ms += v;
    }
    if (!want_mass) return;
    flow_finish<T>(f, ms, T(0), [&](double s0, double) { f.hs[H_MASS] = s0 / (double)f.n; });
}

// One periodic 1-D Gaussian pass along axis AX (0 x, 1 y, 2 z), staged in
// shared memory: a block of 32 x 8 threads loads kTileAx + 2R lines of the
// axis once (each line a coalesced run along x; along x itself, kTileAx + 2R
// consecutive values of 8 rows) and writes kTileAx outputs per line, so each
// input is read about (kTileAx + 2R) / kTileAx times instead of 2R + 1.
// Grid: x = tiles across x (32 wide, or kTileAx wide for AX 0), y = tiles
// along the blurred axis (for AX 0: groups of 8 rows), z = the remaining
// axis (looped when above the grid limit).
// RT > 0: the radius is RT (the paper's blurs: 3 and 6 taps per side), the
// weights sit in registers and the tap loops unroll; RT = 0: any radius.
// Both sum the taps in the same order.
template <typename T, int AX, int MAXI, int RT>
__global__ void __launch_bounds__(256) k_blur(const __grid_constant__ BlurL<T, MAXI> BL)
{
    constexpr int L = kTileAx + 2 * (RT ? RT : kMaxRadius);
    __shared__ T s[AX == 0 ? 8 : L][AX == 0 ? L : 32];
    const int inst = blockIdx.z / BL.zb, zo = blockIdx.z - inst * BL.zb;
    const T* __restrict__ in = BL.in[inst];
    T* __restrict__ out = BL.out[inst];
    const int nx = BL.nx, ny = BL.ny, nz = BL.nz;
    const Weights& w = BL.w;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int R = RT ? RT : w.R;
    T wk[RT ? 2 * RT + 1 : 1];
    if constexpr (RT > 0) {
#pragma unroll
        for (int j = 0; j <= 2 * RT; ++j) wk[j] = wget<T>(w, j);
    }
    auto tap = [&](int j) -> T {
        if constexpr (RT > 0) return wk[j];
        else return wget<T>(w, j);
    };
    const long pls = (long)nx * ny;
    const int n_other = AX == 2 ? ny : nz;
    for (int o = zo; o < n_other; o += BL.zb) {
#if PFC_DEBUG
        // debug builds: the tile starts as NaN, so an output that reads a cell
        // this pass did not load shows up in the results
        for (int i = ty * 32 + tx; i < (int)(sizeof(s) / sizeof(T)); i += 256) (&s[0][0])[i] = T(NAN);
        __syncthreads();
#endif
        if (AX == 0) {
            const int x0 = blockIdx.x * kTileAx, y = blockIdx.y * 8 + ty;
            const long row = (long)o * pls + (long)y * nx;
            if (y < ny)
                for (int k = tx; k < kTileAx + 2 * R; k += 32) s[ty][k] = in[row + nbr(x0, k - R, nx)];
            __syncthreads();
            if (y < ny)
                for (int k = tx; k < kTileAx && x0 + k < nx; k += 32) {
                    T acc = 0;
#pragma unroll
                    for (int j = 0; j <= 2 * (RT ? RT : kMaxRadius); ++j) {
                        if (!RT && j > 2 * R) break;
                        acc += tap(j) * s[ty][k + j];
                    }
                    out[row + x0 + k] = acc;
                }
        } else {
            const int x = blockIdx.x * 32 + tx, c0 = blockIdx.y * kTileAx;
            const int n_ax = AX == 1 ? ny : nz;
            // element (x, axis index c, other index o)
            const long stride = AX == 1 ? (long)nx : pls;
            const long base = AX == 1 ? (long)o * pls + x : (long)o * nx + x;
            if (x < nx)
                for (int k = ty; k < kTileAx + 2 * R; k += 8) s[k][tx] = in[base + (long)nbr(c0, k - R, n_ax) * stride];
            __syncthreads();
            if (x < nx)
                for (int k = ty; k < kTileAx && c0 + k < n_ax; k += 8) {
                    T acc = 0;
#pragma unroll
                    for (int j = 0; j <= 2 * (RT ? RT : kMaxRadius); ++j) {
                        if (!RT && j > 2 * R) break;
                        acc += tap(j) * s[k + j][tx];
                    }
                    out[base + (long)(c0 + k) * stride] = acc;
                }
        }
        __syncthreads();
    }
}

// The y and z passes for the paper's radii (RT = 3 or 6) as a sliding
// window in registers: a thread walks `chunk` outputs along one line (lanes
// on consecutive x, so every load is coalesced), keeping the 2 RT + 1 inputs
// of the current output; each step loads one new input and replaces the
// oldest.  The tap loop is unrolled over a whole window so that slot
// (q + j) % W is a compile-time register: no moves, no shared memory, no
// barriers.  The taps are summed in the same order as in k_blur.
template <typename T, int AX, int MAXI, int RT>
__global__ void __launch_bounds__(256) k_blur_win(const __grid_constant__ BlurL<T, MAXI> BL)
{
    constexpr int W = 2 * RT + 1;
    const int nx = BL.nx, ny = BL.ny, nz = BL.nz;
    const int n_ax = AX == 1 ? ny : nz, n_oth = AX == 1 ? nz : ny;
    const long stride = AX == 1 ? (long)nx : (long)nx * ny;
    long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const long total = (long)nx * BL.nchunks * n_oth * BL.n;
    if (t >= total) return;
    const int x = (int)(t % nx);
    t /= nx;
    const int ch = (int)(t % BL.nchunks);
    t /= BL.nchunks;
    const int o = (int)(t % n_oth);
    const int inst = (int)(t / n_oth);
    const long base = (AX == 1 ? (long)o * nx * ny : (long)o * nx) + x;
    const T* __restrict__ in = BL.in[inst] + base;
    T* __restrict__ out = BL.out[inst] + base;
    const int c0 = ch * BL.chunk, c1 = min(n_ax, c0 + BL.chunk);
    if (c0 >= c1) return;
    T wk[W], win[W];
#pragma unroll
    for (int j = 0; j < W; ++j) {
        wk[j] = wget<T>(BL.w, j);
        win[j] = in[(long)nbr(c0, j - RT, n_ax) * stride];
    }
    int nxt = nbr(c0, RT + 1, n_ax);      // the input entering the window next
    int c = c0;
    for (; c + W <= c1; c += W) {
#pragma unroll
        for (int q = 0; q < W; ++q) {
            T acc = 0;
#pragma unroll
            for (int j = 0; j < W; ++j) acc += wk[j] * win[(q + j) % W];
            out[(long)(c + q) * stride] = acc;
            win[q] = in[(long)nxt * stride];
            nxt = nxt + 1 == n_ax ? 0 : nxt + 1;
        }
    }
    for (; c < c1; ++c) {                 // the rest, window in natural order
        T acc = 0;
#pragma unroll
        for (int j = 0; j < W; ++j) acc += wk[j] * win[j];
        out[(long)c * stride] = acc;
#pragma unroll
        for (int j = 0; j + 1 < W; ++j) win[j] = win[j + 1];
        win[W - 1] = in[(long)nxt * stride];
        nxt = nxt + 1 == n_ax ? 0 : nxt + 1;
    }
}

// FP32 x pass for rows of 4 to 128 values with nx % 4 == 0 (the paper's
// 100^3 grids): the lanes of a row hold x = 4k .. 4k+3 as one float4 each and
// take the taps around their outputs from the neighbouring lanes' registers
// by shuffles, wrapping inside the row (periodic).  32 / (nx/4) rows share a
// warp; a warp covers kRowIt such groups with every load issued before the
// arithmetic.  Taps are summed in the same order as in k_blur.
constexpr int kRowIt = 4;
constexpr int kPrefetch = 3;     // extra ring slots of the float4 window

__device__ __forceinline__ float f4c(const float4& q, int e)
{
    return e == 0 ? q.x : e == 1 ? q.y : e == 2 ? q.z : q.w;
}

template <int MAXI, int RT>
__global__ void __launch_bounds__(256) k_blurx4(const __grid_constant__ BlurL<float, MAXI> BL)
{
    constexpr int NB = (RT + 3) / 4;           // float4 neighbours needed on each side
    constexpr int E = 4 * (2 * NB + 1);        // window: x = 4(k - NB) .. 4(k + NB) + 3
    const int n4 = BL.nx >> 2, rpw = 32 / n4;
    const int lane = threadIdx.x & 31, r = lane / n4, k = lane - r * n4;
    const int rows = BL.ny * BL.nz;            // of this instance (blockIdx.y)
    const int g = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (g * kRowIt * rpw >= rows) return;      // whole warps only: the shuffles need all lanes
    const float* __restrict__ in = BL.in[blockIdx.y];
    float* __restrict__ out = BL.out[blockIdx.y];
    float wk[2 * RT + 1];
#pragma unroll
    for (int j = 0; j <= 2 * RT; ++j) wk[j] = BL.w.wf[j];
    int src[2 * NB + 1];
#pragma unroll
    for (int d = 0; d <= 2 * NB; ++d) {
        int kk = k + d - NB;
        while (kk < 0) kk += n4;
        while (kk >= n4) kk -= n4;
        src[d] = r < rpw ? r * n4 + kk : lane;
    }
    float4 v[kRowIt];
    long off[kRowIt];
#pragma unroll
    for (int it = 0; it < kRowIt; ++it) {
        const int row = (g * kRowIt + it) * rpw + r;
        v[it] = make_float4(0.f, 0.f, 0.f, 0.f);
        off[it] = -1;
        if (r < rpw && row < rows) {
            off[it] = (long)row * BL.nx + 4 * k;
            v[it] = *reinterpret_cast<const float4*>(in + off[it]);
        }
    }
#pragma unroll
    for (int it = 0; it < kRowIt; ++it) {
        float c[E];
#pragma unroll
        for (int d = 0; d <= 2 * NB; ++d)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int ox = 4 * (d - NB) + e;           // x offset from 4k
                if (ox < -RT || ox > 3 + RT) continue;     // never a tap
                const float val = f4c(v[it], e);
                c[4 * d + e] = d == NB ? val : __shfl_sync(0xffffffffu, val, src[d]);
            }
        float o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j <= 2 * RT; ++j) acc += wk[j] * c[4 * NB + e - RT + j];
            o[e] = acc;
        }
        if (off[it] >= 0) *reinterpret_cast<float4*>(out + off[it]) = make_float4(o[0], o[1], o[2], o[3]);
    }
}

// FP32 y and z passes with nx % 4 == 0: k_blur_win with four x-columns per
// thread as one float4 (16-byte loads and stores) and a ring of 2 RT + 1 + D
// float4 in registers: the input loaded after output q is first needed D + 1
// outputs later, so D + 1 loads per thread are in flight.  Instance =
// blockIdx.y; all index arithmetic in 32 bits (the launch checks the sizes).
template <int AX, int MAXI, int RT, int D>
__global__ void __launch_bounds__(256) k_blur_win4(const __grid_constant__ BlurL<float, MAXI> BL)
{
    constexpr int W = 2 * RT + 1, S = W + D;
    const int nx = BL.nx, ny = BL.ny, nz = BL.nz, nx4 = nx >> 2;
    const int n_ax = AX == 1 ? ny : nz, n_oth = AX == 1 ? nz : ny;
    const long stride = AX == 1 ? (long)nx : (long)nx * ny;
    unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (unsigned)(nx4 * BL.nchunks * n_oth)) return;
    const int x4 = (int)(t % (unsigned)nx4);
    t /= (unsigned)nx4;
    const int ch = (int)(t % (unsigned)BL.nchunks);
    const int o = (int)(t / (unsigned)BL.nchunks);
    const long base = (AX == 1 ? (long)o * nx * ny : (long)o * nx) + 4 * x4;
    const float* __restrict__ in = BL.in[blockIdx.y] + base;
    float* __restrict__ out = BL.out[blockIdx.y] + base;
    const int c0 = ch * BL.chunk, c1 = min(n_ax, c0 + BL.chunk);
    if (c0 >= c1) return;
    auto ld = [&](int c) { return *reinterpret_cast<const float4*>(in + (long)c * stride); };
    auto st = [&](int c, float4 q) { *reinterpret_cast<float4*>(out + (long)c * stride) = q; };
    float wk[W];
    float4 win[S];                        // slot s: input c - RT + s (rotating by whole rings)
#pragma unroll
    for (int j = 0; j < W; ++j) wk[j] = BL.w.wf[j];
#pragma unroll
    for (int s = 0; s < S; ++s) win[s] = ld(nbr(c0, s - RT, n_ax));
    int nxt = nbr(c0, S - RT, n_ax);      // the input entering the ring next
    int c = c0;
    for (; c + S <= c1; c += S) {
#pragma unroll
        for (int q = 0; q < S; ++q) {
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int j = 0; j < W; ++j) {
                const float4 s = win[(q + j) % S];
                acc.x += wk[j] * s.x; acc.y += wk[j] * s.y; acc.z += wk[j] * s.z; acc.w += wk[j] * s.w;
            }
            st(c + q, acc);
            win[q] = ld(nxt);
            nxt = nxt + 1 == n_ax ? 0 : nxt + 1;
        }
    }
    for (; c < c1; ++c) {                 // the rest, ring in natural order
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < W; ++j) {
            acc.x += wk[j] * win[j].x; acc.y += wk[j] * win[j].y; acc.z += wk[j] * win[j].z; acc.w += wk[j] * win[j].w;
        }
        st(c, acc);
#pragma unroll
        for (int s = 0; s + 1 < S; ++s) win[s] = win[s + 1];
        win[S - 1] = ld(nxt);
        nxt = nxt + 1 == n_ax ? 0 : nxt + 1;
    }
}

template <int MAXI>
static void k_blurx4_launch(const BlurL<float, MAXI>& BL, int R, dim3 grid, cudaStream_t s)
{
    if (R == 6) k_blurx4<MAXI, 6><<<grid, 256, 0, s>>>(BL);
    else k_blurx4<MAXI, 3><<<grid, 256, 0, s>>>(BL);
}

// Pieces per line for the window kernels: enough threads to fill the GPU,
// no piece shorter than min_chunk outputs when the line holds that many.
static void blur_pieces(int n_ax, int min_chunk, long lines, long want, int* chunk, int* nchunks)
{
    long pieces = (want + lines - 1) / lines;
    const long max_pieces = n_ax >= min_chunk ? n_ax / min_chunk : 1;
    if (pieces > max_pieces) pieces = max_pieces;
    if (pieces < 1) pieces = 1;
    *chunk = (int)((n_ax + pieces - 1) / pieces);
    *nchunks = (n_ax + *chunk - 1) / *chunk;
}

// FP32 with nx % 4 == 0, 16-byte aligned buffers and the paper's radii: the
// float4 kernels (x: shuffles within a warp for rows of up to 128 values;
// y, z: float4 windows).  Other FP32 and FP64 cases: register windows for y
// and z at radii 3 and 6, shared-memory tiles otherwise.
template <typename T, int AX, int MAXI>
static void launch_blur(BlurL<T, MAXI>& BL, int n_inst, cudaStream_t s)
{
    const int nx = BL.nx, ny = BL.ny, nz = BL.nz;
    BL.n = n_inst;
    const int R = BL.w.R;
    const bool paper_r = R == 3 || R == 6;
    bool vec = sizeof(T) == 4 && nx % 4 == 0 && paper_r && (AX != 0 || nx <= 128) &&
               (long)nx * ny * nz < (1L << 31);     // 32-bit indexing inside the instance
    for (int k = 0; vec && k < n_inst; ++k)
        vec = reinterpret_cast<uintptr_t>(BL.in[k]) % 16 == 0 && reinterpret_cast<uintptr_t>(BL.out[k]) % 16 == 0;
    if constexpr (sizeof(T) == 4 && AX == 0) {
        if (vec) {
            const long per_warp = (long)(32 / (nx / 4)) * kRowIt;
            const long warps = ((long)ny * nz + per_warp - 1) / per_warp;
            k_blurx4_launch<MAXI>(BL, R, dim3((unsigned)((warps + 7) / 8), n_inst), s);
            return;
        }
    }
    if constexpr (sizeof(T) == 4 && AX != 0) {
        if (vec) {
            const int n_ax = AX == 1 ? ny : nz, n_oth = AX == 1 ? nz : ny;
            const long lines = (long)(nx / 4) * n_oth;
            // pieces as short as 4 outputs when there are few lines (one flow:
            // the GPU would otherwise sit half idle); the taps are summed in
            // the same order whatever the pieces
            blur_pieces(n_ax, 4, lines * n_inst, 1024L * device_sms(), &BL.chunk, &BL.nchunks);
            const dim3 grid((unsigned)((lines * BL.nchunks + 255) / 256), n_inst);
            if (R == 6) k_blur_win4<AX, MAXI, 6, kPrefetch><<<grid, 256, 0, s>>>(BL);
            else k_blur_win4<AX, MAXI, 3, kPrefetch><<<grid, 256, 0, s>>>(BL);
            return;
        }
    }
    if constexpr (AX != 0) {
        if (paper_r) {
            const int n_ax = AX == 1 ? ny : nz, n_oth = AX == 1 ? nz : ny;
            const long lines = (long)nx * n_oth * n_inst;
            blur_pieces(n_ax, 2 * R + 1, lines, 4096L * device_sms(), &BL.chunk, &BL.nchunks);
            const unsigned blocks = (unsigned)((lines * BL.nchunks + 255) / 256);
            if (R == 6) k_blur_win<T, AX, MAXI, 6><<<blocks, 256, 0, s>>>(BL);
            else k_blur_win<T, AX, MAXI, 3><<<blocks, 256, 0, s>>>(BL);
            return;
        }
    }
    const int n_other = AX == 2 ? ny : nz;
    const int cap = 65535 / n_inst;
    BL.zb = n_other < cap ? n_other : cap;
    const dim3 grid = AX == 0 ? dim3((nx + kTileAx - 1) / kTileAx, (ny + 7) / 8, BL.zb * n_inst)
                              : dim3((nx + 31) / 32, ((AX == 1 ? ny : nz) + kTileAx - 1) / kTileAx, BL.zb * n_inst);
    if constexpr (AX == 0) {
        if (R == 6) { k_blur<T, AX, MAXI, 6><<<grid, dim3(32, 8), 0, s>>>(BL); return; }
        if (R == 3) { k_blur<T, AX, MAXI, 3><<<grid, dim3(32, 8), 0, s>>>(BL); return; }
    }
    k_blur<T, AX, MAXI, 0><<<grid, dim3(32, 8), 0, s>>>(BL);
}

// dG/dA from the blurred gradient gb, then Adam (Kingma and Ba) on A with
// moments m, v; the step counter lives in f.ints[1].  `only_grad`: write
// dG/dA to m and leave A, v alone (pfc_hflow_grad).
template <typename T, int MAXI>
__global__ void __launch_bounds__(kThreads) k_adam(const __grid_constant__ AdamL<T, MAXI> L)
{
    const Flow& f = L.f[blockIdx.y];
    const T* __restrict__ gb = L.gb[blockIdx.y];
    T* __restrict__ A = L.A[blockIdx.y];
    T* __restrict__ m = L.m[blockIdx.y];
    T* __restrict__ v = L.v[blockIdx.y];
    const int only_grad = L.only_grad;
    const long n = f.n, pls = (long)f.nx * f.ny;
    const unsigned t = f.ints[1] + 1;
    const T b1 = (T)f.beta1, b2 = (T)f.beta2;
    const T c1 = T(1) / (T(1) - pow_<T>(b1, (T)t)), c2 = T(1) / (T(1) - pow_<T>(b2, (T)t));
    const T lr = (T)f.lr, ae = (T)f.adam_eps, sg = (T)f.sg;
    T sabs = 0, gmax = 0;
    for (Walk w(f.nx, f.ny, (long)blockIdx.x * kThreads + threadIdx.x, (long)gridDim.x * kThreads); w.i < n;
         w.next(f.nx, f.ny)) {
        const long row = w.i - w.x, pl = (long)w.z * pls, col = w.i - pl;
        T g[3];
        g[0] = sg * (gb[row + nbr(w.x, -1, f.nx)] - gb[row + nbr(w.x, 1, f.nx)]);
        g[1] = sg * (gb[pl + (long)nbr(w.y, -1, f.ny) * f.nx + w.x] - gb[pl + (long)nbr(w.y, 1, f.ny) * f.nx + w.x]);
        g[2] = sg * (gb[(long)nbr(w.z, -1, f.nz) * pls + col] - gb[(long)nbr(w.z, 1, f.nz) * pls + col]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long k = c * n + w.i;
            const T gc = g[c];
            const T ag = gc < T(0) ? -gc : gc;
            sabs += ag;
            gmax = ag > gmax ? ag : gmax;
            if (only_grad) {
                m[k] = gc;
                continue;
            }
            const T mk = b1 * m[k] + (T(1) - b1) * gc;
            const T vk = b2 * v[k] + (T(1) - b2) * gc * gc;
            m[k] = mk;
            v[k] = vk;
            A[k] -= lr * (mk * c1) / (sqrt(vk * c2) + ae);
        }
    }
    flow_finish<T>(f, sabs, gmax, [&](double s0, double s1) {
        f.hs[H_GMAX] = s1;
        f.hs[H_GABS] = s0 / (3.0 * (double)f.n);
        if (only_grad) return;
        f.ints[1] = t;
        const unsigned rowi = f.ints[2];
        if (f.trace && (int)rowi < f.trace_cap) {
            double* r = f.trace + (size_t)rowi * 5;
            r[0] = f.sweep_scal[S_E];
            r[1] = s1;
            r[2] = s0 / (3.0 * (double)f.n);
            r[3] = f.hs[H_MASS];
            r[4] = (double)t;
        }
        f.ints[2] = rowi + 1;
    });
}

// float fields with nx % 4 == 0: the same two kernels on float4 along x (four
// voxels per thread, one 16-byte load per field and neighbour row, the two
// x-neighbours outside the four as scalar loads), a quarter of the load
// instructions of the scalar forms.
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
// Streams touched once per iteration (Adam's A, m, v): evict-first loads and
// stores, so that they do not push the stencils' reused fields out of L2.
__device__ __forceinline__ float4 ld4s(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void st4s(float* p, float4 v) { __stcs(reinterpret_cast<float4*>(p), v); }

template <int MAXI>
__global__ void __launch_bounds__(kThreads) k_div4(const __grid_constant__ DivL<float, MAXI> L)
{
    const Flow& f = L.f[blockIdx.y];
    const float* __restrict__ A = L.A[blockIdx.y];
    float* __restrict__ u = L.u[blockIdx.y];
    const int want_mass = L.want_mass;
    const int nx4 = f.nx >> 2;
    const long n = f.n, n4 = n >> 2, pls = (long)f.nx * f.ny;
    const float sg = (float)f.sg, m0 = (float)f.m0;
    const float* mf = (const float*)f.mf;
    float ms = 0;
    for (Walk w(nx4, f.ny, (long)blockIdx.x * kThreads + threadIdx.x, (long)gridDim.x * kThreads); w.i < n4;
         w.next(nx4, f.ny)) {
        const int x = 4 * w.x;
        const long pl = (long)w.z * pls, row = pl + (long)w.y * f.nx, i = row + x, col = i - pl;
        const float4 a = ld4(A + i);
        const float am = A[row + nbr(x, -1, f.nx)], ap = A[row + nbr(x + 3, 1, f.nx)];
        const float4 yp = ld4(A + n + pl + (long)nbr(w.y, 1, f.ny) * f.nx + x);
        const float4 ym = ld4(A + n + pl + (long)nbr(w.y, -1, f.ny) * f.nx + x);
        const float4 zp = ld4(A + 2 * n + (long)nbr(w.z, 1, f.nz) * pls + col);
        const float4 zm = ld4(A + 2 * n + (long)nbr(w.z, -1, f.nz) * pls + col);
        const float4 m = mf ? ld4(mf + i) : make_float4(m0, m0, m0, m0);
        float4 v;
        v.x = sg * ((a.y - am) + (yp.x - ym.x) + (zp.x - zm.x)) + m.x;
        v.y = sg * ((a.z - a.x) + (yp.y - ym.y) + (zp.y - zm.y)) + m.y;
        v.z = sg * ((a.w - a.y) + (yp.z - ym.z) + (zp.z - zm.z)) + m.z;
        v.w = sg * ((ap - a.z) + (yp.w - ym.w) + (zp.w - zm.w)) + m.w;
        st4(u + i, v);
        ms += (v.x + v.y) + (v.z + v.w);
    }
    if (!want_mass) return;
    flow_finish<float>(f, ms, 0.0f, [&](double s0, double) { f.hs[H_MASS] = s0 / (double)f.n; });
}

// div A + m followed by the x pass of the blur in one kernel, for FP32 rows
// of 4 to 128 values with nx % 4 == 0 (the paper's 100^3 grids): the lanes
// of a row hold x = 4k .. 4k+3 as one float4, take A_x at x - 1 and x + 4
// from their neighbours by shuffles, form the row of div A + m in registers
// and blur it along x as k_blurx4 does (same arithmetic, same tap order as
// k_div4 followed by k_blurx4).  The mass is the mean of div A + m before
// the blur, summed as k_div4 sums it.  Instance = blockIdx.y; blocks stride
// over groups of rows.
constexpr int kDivRowIt = 2;

template <int MAXI, int RT>
__global__ void __launch_bounds__(kThreads)
k_div_blurx4(const __grid_constant__ DivL<float, MAXI> L, const __grid_constant__ Weights w)
{
    constexpr int NB = (RT + 3) / 4;           // float4 neighbours needed on each side (>= 1)
    constexpr int E = 4 * (2 * NB + 1);
    const Flow& f = L.f[blockIdx.y];
    const float* __restrict__ A = L.A[blockIdx.y];
    float* __restrict__ u = L.u[blockIdx.y];
    const int nx = f.nx, ny = f.ny, nz = f.nz, n4 = nx >> 2, rpw = 32 / n4;
    const long n = f.n, pls = (long)nx * ny;
    const int lane = threadIdx.x & 31, r = lane / n4, k = lane - r * n4;
    const int rows = ny * nz;
    const float sg = (float)f.sg, m0 = (float)f.m0;
    const float* mf = (const float*)f.mf;
    float wk[2 * RT + 1];
#pragma unroll
    for (int j = 0; j <= 2 * RT; ++j) wk[j] = w.wf[j];
    int src[2 * NB + 1];
#pragma unroll
    for (int d = 0; d <= 2 * NB; ++d) {
        int kk = k + d - NB;
        while (kk < 0) kk += n4;
        while (kk >= n4) kk -= n4;
        src[d] = r < rpw ? r * n4 + kk : lane;
    }
    float ms = 0.f;
    constexpr int wpb = kThreads / 32;
    for (int g = blockIdx.x * wpb + (threadIdx.x >> 5); g * kDivRowIt * rpw < rows; g += gridDim.x * wpb) {
        float4 ax[kDivRowIt], yp[kDivRowIt], ym[kDivRowIt], zp[kDivRowIt], zm[kDivRowIt], mm[kDivRowIt];
        long off[kDivRowIt];
#pragma unroll
        for (int it = 0; it < kDivRowIt; ++it) {
            const int row = (g * kDivRowIt + it) * rpw + r;
            const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
            ax[it] = yp[it] = ym[it] = zp[it] = zm[it] = zero;
            mm[it] = make_float4(m0, m0, m0, m0);
            off[it] = -1;
            if (r < rpw && row < rows) {
                const int z = row / ny, y = row - z * ny, x = 4 * k;
                const long pl = (long)z * pls, i = pl + (long)y * nx + x, col = i - pl;
                off[it] = i;
                ax[it] = ld4(A + i);
                yp[it] = ld4(A + n + pl + (long)nbr(y, 1, ny) * nx + x);
                ym[it] = ld4(A + n + pl + (long)nbr(y, -1, ny) * nx + x);
                zp[it] = ld4(A + 2 * n + (long)nbr(z, 1, nz) * pls + col);
                zm[it] = ld4(A + 2 * n + (long)nbr(z, -1, nz) * pls + col);
                if (mf) mm[it] = ld4(mf + i);
            }
        }
#pragma unroll
        for (int it = 0; it < kDivRowIt; ++it) {
            const float am = __shfl_sync(0xffffffffu, ax[it].w, src[NB - 1]);
            const float ap = __shfl_sync(0xffffffffu, ax[it].x, src[NB + 1]);
            const float4 a = ax[it], p = yp[it], q = ym[it], zu = zp[it], zd = zm[it], m = mm[it];
            float4 v;
            v.x = sg * ((a.y - am) + (p.x - q.x) + (zu.x - zd.x)) + m.x;
            v.y = sg * ((a.z - a.x) + (p.y - q.y) + (zu.y - zd.y)) + m.y;
            v.z = sg * ((a.w - a.y) + (p.z - q.z) + (zu.z - zd.z)) + m.z;
            v.w = sg * ((ap - a.z) + (p.w - q.w) + (zu.w - zd.w)) + m.w;
            if (off[it] >= 0) ms += (v.x + v.y) + (v.z + v.w);
            float c[E];
#pragma unroll
            for (int d = 0; d <= 2 * NB; ++d)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int ox = 4 * (d - NB) + e;
                    if (ox < -RT || ox > 3 + RT) continue;
                    const float val = f4c(v, e);
                    c[4 * d + e] = d == NB ? val : __shfl_sync(0xffffffffu, val, src[d]);
                }
            float o[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j <= 2 * RT; ++j) acc += wk[j] * c[4 * NB + e - RT + j];
                o[e] = acc;
            }
            if (off[it] >= 0) st4(u + off[it], make_float4(o[0], o[1], o[2], o[3]));
        }
    }
    if (!L.want_mass) return;
    flow_finish<float>(f, ms, 0.0f, [&](double s0, double) { f.hs[H_MASS] = s0 / (double)f.n; });
}

template <int MAXI>
__global__ void __launch_bounds__(kThreads) k_adam4(const __grid_constant__ AdamL<float, MAXI> L)
{
    const Flow& f = L.f[blockIdx.y];
    const float* __restrict__ gb = L.gb[blockIdx.y];
    float* __restrict__ A = L.A[blockIdx.y];
    float* __restrict__ m = L.m[blockIdx.y];
    float* __restrict__ v = L.v[blockIdx.y];
    const int only_grad = L.only_grad;
    const int nx4 = f.nx >> 2;
    const long n = f.n, n4 = n >> 2, pls = (long)f.nx * f.ny;
    const unsigned t = f.ints[1] + 1;
    const float b1 = (float)f.beta1, b2 = (float)f.beta2;
    const float c1 = 1.0f / (1.0f - powf(b1, (float)t)), c2 = 1.0f / (1.0f - powf(b2, (float)t));
    const float lr = (float)f.lr, ae = (float)f.adam_eps, sg = (float)f.sg;
    float sabs = 0, gmax = 0;
    for (Walk w(nx4, f.ny, (long)blockIdx.x * kThreads + threadIdx.x, (long)gridDim.x * kThreads); w.i < n4;
         w.next(nx4, f.ny)) {
        const int x = 4 * w.x;
        const long pl = (long)w.z * pls, row = pl + (long)w.y * f.nx, i = row + x, col = i - pl;
        const float4 c = ld4(gb + i);
        const float gm = gb[row + nbr(x, -1, f.nx)], gp = gb[row + nbr(x + 3, 1, f.nx)];
        const float4 ym = ld4(gb + pl + (long)nbr(w.y, -1, f.ny) * f.nx + x);
        const float4 yp = ld4(gb + pl + (long)nbr(w.y, 1, f.ny) * f.nx + x);
        const float4 zm = ld4(gb + (long)nbr(w.z, -1, f.nz) * pls + col);
        const float4 zp = ld4(gb + (long)nbr(w.z, 1, f.nz) * pls + col);
        float4 m4[3], v4[3], a4[3];     // all state loads in flight before the arithmetic
        if (!only_grad) {
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                const long k = cc * n + i;
                m4[cc] = ld4s(m + k);
                v4[cc] = ld4s(v + k);
                a4[cc] = ld4s(A + k);
            }
        }
        float4 g[3];
        g[0] = make_float4(sg * (gm - c.y), sg * (c.x - c.z), sg * (c.y - c.w), sg * (c.z - gp));
        g[1] = make_float4(sg * (ym.x - yp.x), sg * (ym.y - yp.y), sg * (ym.z - yp.z), sg * (ym.w - yp.w));
        g[2] = make_float4(sg * (zm.x - zp.x), sg * (zm.y - zp.y), sg * (zm.z - zp.z), sg * (zm.w - zp.w));
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            const long k = cc * n + i;
            const float gg[4] = { g[cc].x, g[cc].y, g[cc].z, g[cc].w };
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float ag = fabsf(gg[j]);
                sabs += ag;
                gmax = fmaxf(gmax, ag);
            }
            if (only_grad) {
                st4(m + k, g[cc]);
                continue;
            }
            const float mm[4] = { m4[cc].x, m4[cc].y, m4[cc].z, m4[cc].w };
            const float vv[4] = { v4[cc].x, v4[cc].y, v4[cc].z, v4[cc].w };
            const float aa[4] = { a4[cc].x, a4[cc].y, a4[cc].z, a4[cc].w };
            float mo[4], vo[4], ao[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                mo[j] = b1 * mm[j] + (1.0f - b1) * gg[j];
                vo[j] = b2 * vv[j] + (1.0f - b2) * gg[j] * gg[j];
                ao[j] = aa[j] - lr * (mo[j] * c1) / (sqrtf(vo[j] * c2) + ae);
            }
            st4s(m + k, make_float4(mo[0], mo[1], mo[2], mo[3]));
            st4s(v + k, make_float4(vo[0], vo[1], vo[2], vo[3]));
            st4s(A + k, make_float4(ao[0], ao[1], ao[2], ao[3]));
        }
    }
    flow_finish<float>(f, sabs, gmax, [&](double s0, double s1) {
        f.hs[H_GMAX] = s1;
        f.hs[H_GABS] = s0 / (3.0 * (double)f.n);
        if (only_grad) return;
        f.ints[1] = t;
        const unsigned rowi = f.ints[2];
        if (f.trace && (int)rowi < f.trace_cap) {
            double* r = f.trace + (size_t)rowi * 5;
            r[0] = f.sweep_scal[S_E];
            r[1] = s1;
            r[2] = s0 / (3.0 * (double)f.n);
            r[3] = f.hs[H_MASS];
            r[4] = (double)t;
        }
        f.ints[2] = rowi + 1;
    });
}

long flow_blocks(long n) { return flow_grid(n).x; }

}  // namespace

struct pfc_hflow {
    pfc_problem P;
    pfc_hflow_params H;
    int device = 0;
    long N = 0;
    int esz = 4;
    int tile_y = 16;
    Weights W{};
    void* buf[4] = { nullptr, nullptr, nullptr, nullptr };   // ut, g, two blur temporaries
    double* spart = nullptr;    // sweep partials
    unsigned* sints = nullptr;  // sweep counters
    double* sscal = nullptr;    // sweep scalars
    double* fpart = nullptr;    // flow partials
    unsigned* fints = nullptr;
    double* hs = nullptr;
    double* trace = nullptr;
    int trace_cap = 0;
    int sweep_slots = 0;
    void* cfield = nullptr;     // c(x) (NCF fields), when a(x) is set
    bool cf_on = false;
    void* mfield = nullptr;     // m(x), when set
    bool mf_on = false;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const void* gA = nullptr;
    const void* gm = nullptr;
    const void* gv = nullptr;
    int glen = 0;
    double* gtrace = nullptr;
    bool gcf = false, gmf = false;
};

static pfc_status hfail(pfc_status s, const char* msg)
{
    pfc::set_last_error(msg);
    return s;
}

#define HCU(call)                                                              \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            (void)cudaGetLastError();                                          \
            char b_[256];                                                      \
            snprintf(b_, sizeof b_, "%s: %s", #call, cudaGetErrorString(e_));  \
            return hfail(PFC_ECUDA, b_);                                       \
        }                                                                      \
    } while (0)

static bool is_current(int device)
{
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return cur == device;
}

// p is device (or managed) memory of the current device, where the flow's
// kernels run
static bool dev_ptr(const void* p)
{
    cudaPointerAttributes at;
    int cur = -1;
    if (!p || cudaGetDevice(&cur) != cudaSuccess || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == cur;
}

static void free_flow(pfc_hflow* h)
{
    for (void* b : h->buf) cudaFree(b);
    cudaFree(h->spart);
    cudaFree(h->sints);
    cudaFree(h->sscal);
    cudaFree(h->fpart);
    cudaFree(h->fints);
    cudaFree(h->hs);
    cudaFree(h->trace);
    cudaFree(h->cfield);
    cudaFree(h->mfield);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->cap) cudaStreamDestroy(h->cap);
}

extern "C" pfc_status pfc_hflow_create(const pfc_problem* prob, const pfc_hflow_params* hp, pfc_hflow** out)
{
    if (!out || !prob || !hp) return hfail(PFC_EINVAL, "hflow: problem, params and out are required");
    *out = nullptr;
    const pfc_problem& p = *prob;
    if (p.nx < 1 || p.ny < 1 || p.nz < 1 || (double)p.nx * p.ny * p.nz > 2.0e9)
        return hfail(PFC_EINVAL, "hflow: grid sizes must be >= 1 and hold at most 2e9 voxels");
    if (!(p.h > 0) || !(p.eps > 0) || !(p.xi > 0)) return hfail(PFC_EINVAL, "hflow: h, eps, xi must be > 0");
    if (p.prec != PFC_FP32 && p.prec != PFC_FP64) return hfail(PFC_EINVAL, "hflow: unknown precision");
    if (p.well != PFC_WELL_01 && p.well != PFC_WELL_PM1) return hfail(PFC_EINVAL, "hflow: unknown double well");
    if (p.impl != PFC_IMPL_FUSED) return hfail(PFC_EUNSUPPORTED, "hflow: runs on the fused path");
    if (p.tile_y != 0 && p.tile_y != 8 && p.tile_y != 13 && p.tile_y != 16) return hfail(PFC_EINVAL, "hflow: tile_y must be 0, 8, 13 or 16");
    for (int i = 0; i < 6; ++i)
        if (!isfinite(p.a[i])) return hfail(PFC_EINVAL, "hflow: a coefficient is not finite");
    if (!isfinite(p.mu) || !isfinite(p.theta[0]) || !isfinite(p.theta[1]) || !isfinite(p.theta[2]))
        return hfail(PFC_EINVAL, "hflow: mu and theta must be finite");
    if ((p.proj != 0 && p.proj != 1) || (p.flags & ~PFC_FLAG_NO_DISCRIMINANT_REFINEMENT))
        return hfail(PFC_EINVAL, "hflow: proj 0 or 1, unknown flags");
    if (!isfinite(hp->m0) || !(hp->lr >= 0) || !(hp->beta1 >= 0 && hp->beta1 < 1) || !(hp->beta2 >= 0 && hp->beta2 < 1) ||
        !(hp->adam_eps >= 0) || !(hp->blur_sigma >= 0))
        return hfail(PFC_EINVAL, "hflow: m0 finite, lr >= 0, betas in [0,1), eps >= 0, sigma >= 0 required");
    int R = 0;
    if (hp->blur_sigma > 0) {
        R = hp->blur_radius > 0 ? hp->blur_radius : (int)ceil(3.0 * hp->blur_sigma);
        if (R > kMaxRadius) return hfail(PFC_EINVAL, "hflow: blur radius above 32 taps");
    }
    pfc_hflow* h = new (std::nothrow) pfc_hflow();
    if (!h) return hfail(PFC_ENOMEM, "hflow: host allocation failed");
    h->P = p;
    h->H = *hp;
    h->H.blur_radius = R;
    h->N = (long)p.nx * p.ny * p.nz;
    h->esz = p.prec == PFC_FP64 ? 8 : 4;
    h->tile_y = p.tile_y ? p.tile_y : default_tile_y(p.ny, p.prec == PFC_FP64);
    h->W.R = R;
    if (R > 0) {   // discrete Gaussian, normalised to sum 1
        double s = 0;
        for (int j = -R; j <= R; ++j) s += exp(-(double)j * j / (2.0 * hp->blur_sigma * hp->blur_sigma));
        for (int j = -R; j <= R; ++j) {
            h->W.wd[j + R] = exp(-(double)j * j / (2.0 * hp->blur_sigma * hp->blur_sigma)) / s;
            h->W.wf[j + R] = (float)h->W.wd[j + R];
        }
    }
    cudaGetDevice(&h->device);
    h->sweep_slots = (int)fused_slots(p.nx, p.ny, p.nz, h->tile_y, p.tile_z);
    bool ok = true;
    for (void*& b : h->buf) ok = ok && cudaMalloc(&b, (size_t)h->esz * h->N) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&h->spart, sizeof(double) * NPART * (size_t)h->sweep_slots) == cudaSuccess &&
         cudaMalloc((void**)&h->sints, sizeof(unsigned) * NINTS) == cudaSuccess &&
         cudaMalloc((void**)&h->sscal, sizeof(double) * NSCAL) == cudaSuccess &&
         cudaMalloc((void**)&h->fpart, sizeof(double) * 2 * (size_t)flow_blocks((long)p.nx * p.ny * p.nz)) == cudaSuccess &&
         cudaMalloc((void**)&h->fints, sizeof(unsigned) * 4) == cudaSuccess &&
         cudaMalloc((void**)&h->hs, sizeof(double) * NH) == cudaSuccess &&
         cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) ok = cudaMemsetAsync(h->sints, 0, sizeof(unsigned) * NINTS, h->cap) == cudaSuccess &&
                 cudaMemsetAsync(h->fints, 0, sizeof(unsigned) * 4, h->cap) == cudaSuccess &&
                 cudaMemsetAsync(h->hs, 0, sizeof(double) * NH, h->cap) == cudaSuccess &&
                 cudaStreamSynchronize(h->cap) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        free_flow(h);
        delete h;
        return hfail(PFC_ENOMEM, "hflow: device allocation failed");
    }
    *out = h;
    return PFC_OK;
}

extern "C" void pfc_hflow_destroy(pfc_hflow* h)
{
    if (!h) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    free_flow(h);
    cudaSetDevice(prev);
    delete h;
}

static Flow flow_desc(const pfc_hflow* h)
{
    Flow f;
    f.nx = h->P.nx; f.ny = h->P.ny; f.nz = h->P.nz;
    f.n = h->N;
    f.sg = 1.0 / (2.0 * h->P.h);
    f.m0 = h->H.m0;
    f.mf = h->mf_on ? h->mfield : nullptr;
    f.lr = h->H.lr; f.beta1 = h->H.beta1; f.beta2 = h->H.beta2; f.adam_eps = h->H.adam_eps;
    f.part = h->fpart;
    f.ints = h->fints;
    f.hs = h->hs;
    f.sweep_scal = h->sscal;
    f.trace = h->trace;
    f.trace_cap = h->trace_cap;
    return f;
}

static bool al16(const void* p) { return p == nullptr || ((uintptr_t)p & 15) == 0; }

// u = div A + m into `out` for n_inst instances of one grid size (float4
// path when the rows and every buffer allow it)
template <typename T, int MAXI>
static void launch_div(DivL<T, MAXI>& L, int n_inst, long N, int nx, cudaStream_t s)
{
    bool v4 = sizeof(T) == 4 && nx % 4 == 0;
    for (int k = 0; k < n_inst; ++k) v4 = v4 && al16(L.A[k]) && al16(L.u[k]) && al16(L.f[k].mf);
    if (v4) {
        const dim3 grid(inst_blocks(N / 4, n_inst), n_inst);
        k_div4<MAXI><<<grid, kThreads, 0, s>>>(reinterpret_cast<const DivL<float, MAXI>&>(L));
        return;
    }
    k_div<T, MAXI><<<dim3(inst_blocks(N, n_inst), n_inst), kThreads, 0, s>>>(L);
}

// div A + m and the blur's x pass in one kernel into L.u; false (nothing
// launched) unless FP32, nx % 4 == 0, nx <= 128, radius 3 or 6 and aligned
// buffers
template <typename T, int MAXI>
static bool launch_div_blurx(DivL<T, MAXI>& L, int n_inst, long N, int nx, int ny, int nz, const Weights& w,
                             cudaStream_t s)
{
    if constexpr (sizeof(T) != 4) {
        return false;
    } else {
        if (nx % 4 != 0 || nx > 128 || !(w.R == 3 || w.R == 6) || N >= (1L << 31)) return false;
        for (int k = 0; k < n_inst; ++k)
            if (!al16(L.A[k]) || !al16(L.u[k]) || !al16(L.f[k].mf)) return false;
        const long per_warp = (long)(32 / (nx / 4)) * kDivRowIt;
        const long warps = ((long)ny * nz + per_warp - 1) / per_warp;
        long blocks = (warps + kThreads / 32 - 1) / (kThreads / 32);
        if (blocks > (long)inst_blocks(N, n_inst)) blocks = inst_blocks(N, n_inst);   // <= partials capacity
        const dim3 grid((unsigned)blocks, n_inst);
        const DivL<float, MAXI>& Lf = reinterpret_cast<const DivL<float, MAXI>&>(L);
        if (w.R == 6) k_div_blurx4<MAXI, 6><<<grid, kThreads, 0, s>>>(Lf, w);
        else k_div_blurx4<MAXI, 3><<<grid, kThreads, 0, s>>>(Lf, w);
        return true;
    }
}

// dG/dA and (unless only_grad) the Adam update, n_inst instances
template <typename T, int MAXI>
static void launch_adam(AdamL<T, MAXI>& L, int n_inst, long N, int nx, cudaStream_t s)
{
    bool v4 = sizeof(T) == 4 && nx % 4 == 0;
    for (int k = 0; k < n_inst; ++k) v4 = v4 && al16(L.gb[k]) && al16(L.A[k]) && al16(L.m[k]) && al16(L.v[k]);
    if (v4) {
        const dim3 grid(inst_blocks(N / 4, n_inst), n_inst);
        k_adam4<MAXI><<<grid, kThreads, 0, s>>>(reinterpret_cast<const AdamL<float, MAXI>&>(L));
        return;
    }
    k_adam<T, MAXI><<<dim3(inst_blocks(N, n_inst), n_inst), kThreads, 0, s>>>(L);
}

template <typename T>
static void launch_div(const pfc_hflow* h, const T* A, T* out, int want_mass, cudaStream_t s)
{
    DivL<T, 1> L;
    L.f[0] = flow_desc(h);
    L.A[0] = A;
    L.u[0] = out;
    L.want_mass = want_mass;
    launch_div<T, 1>(L, 1, h->N, h->P.nx, s);
}

template <typename T>
static void launch_adam(const pfc_hflow* h, const T* gb, T* A, T* m, T* v, int only_grad, cudaStream_t s)
{
    AdamL<T, 1> L;
    L.f[0] = flow_desc(h);
    L.gb[0] = gb;
    L.A[0] = A;
    L.m[0] = m;
    L.v[0] = v;
    L.only_grad = only_grad;
    launch_adam<T, 1>(L, 1, h->N, h->P.nx, s);
}

template <typename T, int AX>
static void launch_blur(const T* in, T* out, int nx, int ny, int nz, const Weights& w, cudaStream_t s)
{
    BlurL<T, 1> BL;
    BL.in[0] = in;
    BL.out[0] = out;
    BL.nx = nx; BL.ny = ny; BL.nz = nz;
    BL.w = w;
    launch_blur<T, AX, 1>(BL, 1, s);
}

// in -> k * in through the two temporaries; returns the buffer holding the result
template <typename T>
static cudaError_t blur3(const pfc_hflow* h, T* in, T* t1, T* t2, T** result, cudaStream_t s)
{
    if (h->W.R == 0) {
        *result = in;
        return cudaSuccess;
    }
    launch_blur<T, 0>(in, t1, h->P.nx, h->P.ny, h->P.nz, h->W, s);
    launch_blur<T, 1>(t1, t2, h->P.nx, h->P.ny, h->P.nz, h->W, s);
    launch_blur<T, 2>(t2, t1, h->P.nx, h->P.ny, h->P.nz, h->W, s);
    *result = t1;
    return cudaGetLastError();
}

// ut = k * (div A + m0) into buf[0] (or the returned buffer)
template <typename T>
static cudaError_t field(const pfc_hflow* h, const T* A, T** ut, int want_mass, cudaStream_t s)
{
    T* b0 = (T*)h->buf[0];
    T* b2 = (T*)h->buf[2];
    T* b3 = (T*)h->buf[3];
    if (h->W.R == 0) {
        launch_div<T>(h, A, b0, want_mass, s);
        *ut = b0;
        return cudaGetLastError();
    }
    DivL<T, 1> L;
    L.f[0] = flow_desc(h);
    L.A[0] = A;
    L.u[0] = b3;
    L.want_mass = want_mass;
    if (!launch_div_blurx<T, 1>(L, 1, h->N, h->P.nx, h->P.ny, h->P.nz, h->W, s)) {
        launch_div<T>(h, A, b2, want_mass, s);
        launch_blur<T, 0>(b2, b3, h->P.nx, h->P.ny, h->P.nz, h->W, s);
    }
    launch_blur<T, 1>(b3, b2, h->P.nx, h->P.ny, h->P.nz, h->W, s);
    launch_blur<T, 2>(b2, b0, h->P.nx, h->P.ny, h->P.nz, h->W, s);
    *ut = b0;
    return cudaGetLastError();
}

// one evaluation: E and k * dF/du in a buffer (returned)
template <typename T>
static cudaError_t eval(pfc_hflow* h, const T* A, T** gb, cudaStream_t s)
{
    T* ut = nullptr;
    cudaError_t e = field<T>(h, A, &ut, 1, s);
    if (e != cudaSuccess) return e;
    Inst<T> in{};
    in.u = ut;
    in.out = (T*)h->buf[1];
    in.nx = h->P.nx; in.ny = h->P.ny; in.nz = h->P.nz;
    in.vec = (h->P.nx % (16 / (int)sizeof(T)) == 0);
    in.C = make_coef<T>(h->P.a, h->P.h, h->P.eps, h->P.xi, h->P.well, h->P.mu, h->P.theta, h->P.proj,
                          (h->P.flags & PFC_FLAG_NO_DISCRIMINANT_REFINEMENT) ? 0 : 1);
    in.cf = h->cf_on ? (const T*)h->cfield : nullptr;
    in.inv_N = 1.0 / (double)h->N;
    in.partials = h->spart;
    in.ints = h->sints;
    in.scal = h->sscal;
    e = launch_fused<T>(in, MODE_GRAD, h->tile_y, h->P.tile_z, s);
    if (e != cudaSuccess) return e;
    return blur3<T>(h, (T*)h->buf[1], (T*)h->buf[2], (T*)h->buf[3], gb, s);
}

template <typename T>
static cudaError_t step(pfc_hflow* h, T* A, T* m, T* v, cudaStream_t s)
{
    T* gb = nullptr;
    cudaError_t e = eval<T>(h, A, &gb, s);
    if (e != cudaSuccess) return e;
    launch_adam<T>(h, gb, A, m, v, 0, s);
    return cudaGetLastError();
}

extern "C" pfc_status pfc_hflow_field(pfc_hflow* h, const void* A, void* ut, pfc_stream stream)
{
    if (!h) return hfail(PFC_EINVAL, "hflow: handle is NULL");
    if (!is_current(h->device)) return hfail(PFC_EINVAL, "hflow: the flow's device is not the current device");
    if (!dev_ptr(A) || !dev_ptr(ut)) return hfail(PFC_EINVAL, "hflow: A and ut must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    if (h->P.prec == PFC_FP64) {
        double* r = nullptr;
        HCU(field<double>(h, (const double*)A, &r, 0, s));
        HCU(cudaMemcpyAsync(ut, r, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, s));
    } else {
        float* r = nullptr;
        HCU(field<float>(h, (const float*)A, &r, 0, s));
        HCU(cudaMemcpyAsync(ut, r, sizeof(float) * h->N, cudaMemcpyDeviceToDevice, s));
    }
    return PFC_OK;
}

extern "C" pfc_status pfc_hflow_grad(pfc_hflow* h, const void* A, void* gA, double* G_host, pfc_stream stream)
{
    if (!h) return hfail(PFC_EINVAL, "hflow: handle is NULL");
    if (!is_current(h->device)) return hfail(PFC_EINVAL, "hflow: the flow's device is not the current device");
    if (!dev_ptr(A) || !dev_ptr(gA)) return hfail(PFC_EINVAL, "hflow: A and gA must be device memory");
    if (A == gA) return hfail(PFC_EINVAL, "hflow: gA must not alias A");
    cudaStream_t s = (cudaStream_t)stream;
    if (h->P.prec == PFC_FP64) {
        double* gb = nullptr;
        HCU(eval<double>(h, (const double*)A, &gb, s));
        launch_adam<double>(h, gb, nullptr, (double*)gA, nullptr, 1, s);
    } else {
        float* gb = nullptr;
        HCU(eval<float>(h, (const float*)A, &gb, s));
        launch_adam<float>(h, gb, nullptr, (float*)gA, nullptr, 1, s);
    }
    HCU(cudaGetLastError());
    if (G_host) {
        HCU(cudaMemcpyAsync(G_host, h->sscal + S_E, sizeof(double), cudaMemcpyDeviceToHost, s));
        HCU(cudaStreamSynchronize(s));
        if (!isfinite(*G_host)) return hfail(PFC_ENONFINITE, "hflow: energy is not finite");
    }
    return PFC_OK;
}

extern "C" pfc_status pfc_hflow_run(pfc_hflow* h, void* A, void* m, void* v, int32_t nsteps, int32_t* t,
                                    double* trace_host, pfc_stream stream)
{
    nvtxRangePushA("pfc_hflow_run");
    struct Pop { ~Pop() { nvtxRangePop(); } } pop_;
    if (!h) return hfail(PFC_EINVAL, "hflow: handle is NULL");
    if (!is_current(h->device)) return hfail(PFC_EINVAL, "hflow: the flow's device is not the current device");
    if (!dev_ptr(A) || !dev_ptr(m) || !dev_ptr(v)) return hfail(PFC_EINVAL, "hflow: A, m, v must be device memory");
    if (A == m || A == v || m == v) return hfail(PFC_EINVAL, "hflow: A, m and v must be distinct");
    if (!t || *t < 0 || nsteps < 0) return hfail(PFC_EINVAL, "hflow: nsteps >= 0 and a step counter >= 0 required");
    if (nsteps == 0) return PFC_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (nsteps > h->trace_cap) {
        if (h->gexec) {
            cudaGraphExecDestroy(h->gexec);
            h->gexec = nullptr;
        }
        // only this stream (earlier runs ended with a wait on theirs): a device-wide
        // wait would break a graph capture that another thread has in progress
        HCU(cudaStreamSynchronize(s));
        cudaFree(h->trace);
        h->trace = nullptr;
        h->trace_cap = 0;
        HCU(cudaMalloc((void**)&h->trace, sizeof(double) * 5 * (size_t)nsteps));
        h->trace_cap = nsteps;
    }
    const unsigned tt[2] = { (unsigned)*t, 0u };
    HCU(cudaMemsetAsync(h->fints, 0, sizeof(unsigned), s));
    HCU(cudaMemcpyAsync(h->fints + 1, tt, sizeof tt, cudaMemcpyHostToDevice, s));
    auto enqueue = [&](int cnt, cudaStream_t st) -> cudaError_t {
        for (int i = 0; i < cnt; ++i) {
            cudaError_t e = h->P.prec == PFC_FP64 ? step<double>(h, (double*)A, (double*)m, (double*)v, st)
                                                  : step<float>(h, (float*)A, (float*)m, (float*)v, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    const int G = nsteps >= 32 ? 32 : 0;
    if (G) {
        if (!(h->gexec && h->gA == A && h->gm == m && h->gv == v && h->glen == G && h->gtrace == h->trace &&
              h->gcf == h->cf_on && h->gmf == h->mf_on)) {
            if (h->gexec) {
                cudaGraphExecDestroy(h->gexec);
                h->gexec = nullptr;
            }
            cudaGraph_t graph = nullptr;
            HCU(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = enqueue(G, h->cap);
            cudaError_t e2 = cudaStreamEndCapture(h->cap, &graph);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                (void)cudaGetLastError();
                return hfail(PFC_ECUDA, "hflow: graph capture failed");
            }
            e = cudaGraphInstantiate(&h->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                h->gexec = nullptr;
                (void)cudaGetLastError();
                return hfail(PFC_ECUDA, "hflow: graph instantiation failed");
            }
            h->gA = A; h->gm = m; h->gv = v; h->glen = G; h->gtrace = h->trace;
            h->gcf = h->cf_on; h->gmf = h->mf_on;
        }
        for (int k = 0; k + G <= nsteps; k += G) HCU(cudaGraphLaunch(h->gexec, s));
    }
    const int done = G ? (nsteps / G) * G : 0;
    HCU(enqueue(nsteps - done, s));
    unsigned back[2];
    HCU(cudaMemcpyAsync(back, h->fints + 1, sizeof back, cudaMemcpyDeviceToHost, s));
    if (trace_host) HCU(cudaMemcpyAsync(trace_host, h->trace, sizeof(double) * 5 * (size_t)nsteps, cudaMemcpyDeviceToHost, s));
    HCU(cudaStreamSynchronize(s));
    *t = (int32_t)back[0];
    if (back[1] != (unsigned)nsteps) return hfail(PFC_ECUDA, "hflow: step count mismatch");
    return PFC_OK;
}

extern "C" pfc_status pfc_hflow_set_coefficient_field(pfc_hflow* h, const void* a_field, pfc_stream stream)
{
    if (!h) return hfail(PFC_EINVAL, "hflow: handle is NULL");
    if (!is_current(h->device)) return hfail(PFC_EINVAL, "hflow: the flow's device is not the current device");
    if (!a_field) {
        h->cf_on = false;
        return PFC_OK;
    }
    if (!dev_ptr(a_field)) return hfail(PFC_EINVAL, "hflow: a_field must be device memory");
    if (!h->cfield) HCU(cudaMalloc(&h->cfield, (size_t)h->esz * NCF * h->N));
    cudaStream_t s = (cudaStream_t)stream;
    if (h->P.prec == PFC_FP64)
        HCU(launch_coef_field<double>((const double*)a_field, (double*)h->cfield, h->N, h->P.h, h->P.eps, s));
    else
        HCU(launch_coef_field<float>((const float*)a_field, (float*)h->cfield, h->N, h->P.h, h->P.eps, s));
    h->cf_on = true;
    return PFC_OK;
}

extern "C" pfc_status pfc_hflow_set_mass_field(pfc_hflow* h, const void* m_field, pfc_stream stream)
{
    if (!h) return hfail(PFC_EINVAL, "hflow: handle is NULL");
    if (!is_current(h->device)) return hfail(PFC_EINVAL, "hflow: the flow's device is not the current device");
    if (!m_field) {
        h->mf_on = false;
        return PFC_OK;
    }
    if (!dev_ptr(m_field)) return hfail(PFC_EINVAL, "hflow: m_field must be device memory");
    if (!h->mfield) HCU(cudaMalloc(&h->mfield, (size_t)h->esz * h->N));
    HCU(cudaMemcpyAsync(h->mfield, m_field, (size_t)h->esz * h->N, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    h->mf_on = true;
    return PFC_OK;
}

// ------------------------------------------------------------ batches of flows
//
// Up to BATCH_MAX flows on grids of one size (FP32, fused path) advanced
// together: every kernel of an iteration is one launch over all instances
// (the sweep through the batched fused kernel), so small grids such as the
// paper's 100^3 fill the GPU.  Each instance has its own coefficients, eps,
// h, xi, double well and mass m0; the blur and Adam's settings are shared.

struct pfc_hflow_batch {
    int n = 0;
    int device = 0;
    int nx = 0, ny = 0, nz = 0;
    long N = 0;
    int tile_y = 16;
    std::vector<pfc_problem> P;
    std::vector<double> m0;
    pfc_hflow_params H{};
    Weights W{};
    float* bufs = nullptr;       // [n][4][N]: ut, g, two blur temporaries
    double* spart = nullptr;     // sweep partials [n][slots][NPART]
    unsigned* sints = nullptr;   // [n][NINTS]
    double* sscal = nullptr;     // [n][NSCAL]
    double* fpart = nullptr;     // flow partials [n][2 * blocks]
    unsigned* fints = nullptr;   // [n][4]
    double* hs = nullptr;        // [n][NH]
    double* trace = nullptr;     // [n][cap][5]
    int trace_cap = 0;
    int slots = 0;
    long fblocks = 0;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<const void*> gkey;
    int glen = 0;
    double* gtrace = nullptr;
};

static void free_flow_batch(pfc_hflow_batch* b)
{
    cudaFree(b->bufs);
    cudaFree(b->spart);
    cudaFree(b->sints);
    cudaFree(b->sscal);
    cudaFree(b->fpart);
    cudaFree(b->fints);
    cudaFree(b->hs);
    cudaFree(b->trace);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->cap) cudaStreamDestroy(b->cap);
}

extern "C" pfc_status pfc_hflow_batch_create(const pfc_problem* probs, const double* m0, int32_t n_inst,
                                             const pfc_hflow_params* hp, pfc_hflow_batch** out)
{
    if (!out || !probs || !m0 || !hp) return hfail(PFC_EINVAL, "hflow batch: problems, m0, params and out are required");
    *out = nullptr;
    if (n_inst < 1 || n_inst > BATCH_MAX) return hfail(PFC_EINVAL, "hflow batch: between 1 and 64 instances");
    for (int k = 0; k < n_inst; ++k) {
        const pfc_problem& p = probs[k];
        if (p.nx != probs[0].nx || p.ny != probs[0].ny || p.nz != probs[0].nz)
            return hfail(PFC_EINVAL, "hflow batch: every instance must have the grid size of the first");
        if (p.nx < 1 || p.ny < 1 || p.nz < 1 || (double)p.nx * p.ny * p.nz > 2.0e9)
            return hfail(PFC_EINVAL, "hflow batch: grid sizes must be >= 1 and hold at most 2e9 voxels");
        if (!(p.h > 0) || !(p.eps > 0) || !(p.xi > 0) || !isfinite(p.h) || !isfinite(p.eps) || !isfinite(p.xi))
            return hfail(PFC_EINVAL, "hflow batch: h, eps, xi must be finite and > 0");
        for (int i = 0; i < 6; ++i)
            if (!isfinite(p.a[i])) return hfail(PFC_EINVAL, "hflow batch: a coefficient is not finite");
        if (p.well != PFC_WELL_01 && p.well != PFC_WELL_PM1) return hfail(PFC_EINVAL, "hflow batch: unknown double well");
        if (p.prec != PFC_FP32 || p.impl != PFC_IMPL_FUSED)
            return hfail(PFC_EUNSUPPORTED, "hflow batch: FP32 on the fused path only");
        if (p.mu != 0.0 || p.proj != 0)
            return hfail(PFC_EUNSUPPORTED, "hflow batch: no orientation term or projected M in batches");
        if (!isfinite(m0[k])) return hfail(PFC_EINVAL, "hflow batch: m0 must be finite");
    }
    if (!(hp->lr >= 0) || !(hp->beta1 >= 0 && hp->beta1 < 1) || !(hp->beta2 >= 0 && hp->beta2 < 1) ||
        !(hp->adam_eps >= 0) || !(hp->blur_sigma >= 0))
        return hfail(PFC_EINVAL, "hflow batch: lr >= 0, betas in [0,1), eps >= 0, sigma >= 0 required");
    int R = 0;
    if (hp->blur_sigma > 0) {
        R = hp->blur_radius > 0 ? hp->blur_radius : (int)ceil(3.0 * hp->blur_sigma);
        if (R > kMaxRadius) return hfail(PFC_EINVAL, "hflow batch: blur radius above 32 taps");
    }
    pfc_hflow_batch* b = new (std::nothrow) pfc_hflow_batch();
    if (!b) return hfail(PFC_ENOMEM, "hflow batch: host allocation failed");
    b->n = n_inst;
    b->nx = probs[0].nx; b->ny = probs[0].ny; b->nz = probs[0].nz;
    b->N = (long)b->nx * b->ny * b->nz;
    b->P.assign(probs, probs + n_inst);
    b->m0.assign(m0, m0 + n_inst);
    b->H = *hp;
    b->H.blur_radius = R;
    b->W.R = R;
    if (R > 0) {
        double s = 0;
        for (int j = -R; j <= R; ++j) s += exp(-(double)j * j / (2.0 * hp->blur_sigma * hp->blur_sigma));
        for (int j = -R; j <= R; ++j) {
            b->W.wd[j + R] = exp(-(double)j * j / (2.0 * hp->blur_sigma * hp->blur_sigma)) / s;
            b->W.wf[j + R] = (float)b->W.wd[j + R];
        }
    }
    b->tile_y = probs[0].tile_y ? probs[0].tile_y : default_tile_y(b->ny, false);
    cudaGetDevice(&b->device);
    const long long units = (long long)((b->nx + 31) / 32) * ((b->ny + b->tile_y - 1) / b->tile_y) * b->nz * n_inst;
    b->slots = (int)fused_grid(units, probs[0].tile_z);
    b->fblocks = flow_blocks(b->N);
    const size_t n = (size_t)n_inst;
    bool ok = cudaMalloc((void**)&b->bufs, sizeof(float) * 4 * (size_t)b->N * n) == cudaSuccess &&
              cudaMalloc((void**)&b->spart, sizeof(double) * NPART * (size_t)b->slots * n) == cudaSuccess &&
              cudaMalloc((void**)&b->sints, sizeof(unsigned) * NINTS * n) == cudaSuccess &&
              cudaMalloc((void**)&b->sscal, sizeof(double) * NSCAL * n) == cudaSuccess &&
              cudaMalloc((void**)&b->fpart, sizeof(double) * 2 * (size_t)b->fblocks * n) == cudaSuccess &&
              cudaMalloc((void**)&b->fints, sizeof(unsigned) * 4 * n) == cudaSuccess &&
              cudaMalloc((void**)&b->hs, sizeof(double) * NH * n) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) ok = cudaMemsetAsync(b->sints, 0, sizeof(unsigned) * NINTS * n, b->cap) == cudaSuccess &&
                 cudaMemsetAsync(b->fints, 0, sizeof(unsigned) * 4 * n, b->cap) == cudaSuccess &&
                 cudaMemsetAsync(b->hs, 0, sizeof(double) * NH * n, b->cap) == cudaSuccess &&
                 cudaStreamSynchronize(b->cap) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        free_flow_batch(b);
        delete b;
        return hfail(PFC_ENOMEM, "hflow batch: device allocation failed");
    }
    *out = b;
    return PFC_OK;
}

extern "C" void pfc_hflow_batch_destroy(pfc_hflow_batch* b)
{
    if (!b) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    free_flow_batch(b);
    cudaSetDevice(prev);
    delete b;
}

static Flow flow_desc_batch(const pfc_hflow_batch* b, int k)
{
    Flow f;
    f.nx = b->nx; f.ny = b->ny; f.nz = b->nz;
    f.n = b->N;
    f.sg = 1.0 / (2.0 * b->P[k].h);
    f.m0 = b->m0[k];
    f.mf = nullptr;
    f.lr = b->H.lr; f.beta1 = b->H.beta1; f.beta2 = b->H.beta2; f.adam_eps = b->H.adam_eps;
    f.part = b->fpart + (size_t)k * 2 * b->fblocks;
    f.ints = b->fints + (size_t)k * 4;
    f.hs = b->hs + (size_t)k * NH;
    f.sweep_scal = b->sscal + (size_t)k * NSCAL;
    f.trace = b->trace ? b->trace + (size_t)k * 5 * b->trace_cap : nullptr;
    f.trace_cap = b->trace_cap;
    return f;
}

static float* bbuf(const pfc_hflow_batch* b, int k, int which) { return b->bufs + ((size_t)k * 4 + which) * b->N; }

// the blur over every instance: in[k] -> out[k]
template <int AX>
static void batch_blur(const pfc_hflow_batch* b, int from, int to, cudaStream_t s)
{
    BlurL<float, BATCH_MAX> BL;
    for (int k = 0; k < b->n; ++k) {
        BL.in[k] = bbuf(b, k, from);
        BL.out[k] = bbuf(b, k, to);
    }
    BL.nx = b->nx; BL.ny = b->ny; BL.nz = b->nz;
    BL.w = b->W;
    launch_blur<float, AX, BATCH_MAX>(BL, b->n, s);
}

// ut[k] = k * (div A[k] + m0[k]) into buffer 0 of every instance
static cudaError_t batch_field(const pfc_hflow_batch* b, const float* const* A, int want_mass, cudaStream_t s)
{
    DivL<float, BATCH_MAX> L;
    for (int k = 0; k < b->n; ++k) {
        L.f[k] = flow_desc_batch(b, k);
        L.A[k] = A[k];
        L.u[k] = bbuf(b, k, b->W.R ? 3 : 0);
    }
    L.want_mass = want_mass;
    if (b->W.R && launch_div_blurx<float, BATCH_MAX>(L, b->n, b->N, b->nx, b->ny, b->nz, b->W, s)) {
        batch_blur<1>(b, 3, 2, s);
        batch_blur<2>(b, 2, 0, s);
        return cudaGetLastError();
    }
    for (int k = 0; k < b->n; ++k) L.u[k] = bbuf(b, k, b->W.R ? 2 : 0);
    launch_div<float, BATCH_MAX>(L, b->n, b->N, b->nx, s);
    if (b->W.R) {
        batch_blur<0>(b, 2, 3, s);
        batch_blur<1>(b, 3, 2, s);
        batch_blur<2>(b, 2, 0, s);
    }
    return cudaGetLastError();
}

// one iteration of Alg. 1 for every instance
static cudaError_t batch_step(const pfc_hflow_batch* b, float* const* A, float* const* m, float* const* v,
                              cudaStream_t s)
{
    cudaError_t e = batch_field(b, A, 1, s);
    if (e != cudaSuccess) return e;
    std::vector<Inst<float>> in(b->n);
    for (int k = 0; k < b->n; ++k) {
        const pfc_problem& P = b->P[k];
        Inst<float>& I = in[k];
        I = Inst<float>{};
        I.u = bbuf(b, k, 0);
        I.out = bbuf(b, k, 1);
        I.nx = b->nx; I.ny = b->ny; I.nz = b->nz;
        I.vec = b->nx % 4 == 0;
        I.C = make_coef<float>(P.a, P.h, P.eps, P.xi, P.well, 0.0, nullptr, 0,
                               (P.flags & PFC_FLAG_NO_DISCRIMINANT_REFINEMENT) ? 0 : 1);
        I.inv_N = 1.0 / (double)b->N;
        I.partials = b->spart + (size_t)k * b->slots * NPART;
        I.ints = b->sints + (size_t)k * NINTS;
        I.scal = b->sscal + (size_t)k * NSCAL;
    }
    e = launch_fused_batch(in.data(), b->n, b->tile_y, b->P[0].tile_z, s, MODE_GRAD);
    if (e != cudaSuccess) return e;
    int gbuf = 1;
    if (b->W.R) {   // the blur of g: 1 -> 2 -> 3 -> 2
        batch_blur<0>(b, 1, 2, s);
        batch_blur<1>(b, 2, 3, s);
        batch_blur<2>(b, 3, 2, s);
        gbuf = 2;
    }
    AdamL<float, BATCH_MAX> L;
    for (int k = 0; k < b->n; ++k) {
        L.f[k] = flow_desc_batch(b, k);
        L.gb[k] = bbuf(b, k, gbuf);
        L.A[k] = A[k];
        L.m[k] = m[k];
        L.v[k] = v[k];
    }
    L.only_grad = 0;
    launch_adam<float, BATCH_MAX>(L, b->n, b->N, b->nx, s);
    return cudaGetLastError();
}

static pfc_status check_vec_list(const void* const* p, int n, const char* name)
{
    if (!p) return hfail(PFC_EINVAL, "hflow batch: a pointer array is NULL");
    for (int k = 0; k < n; ++k)
        if (!dev_ptr(p[k])) {
            char b_[128];
            snprintf(b_, sizeof b_, "hflow batch: %s[%d] must be device memory", name, k);
            return hfail(PFC_EINVAL, b_);
        }
    return PFC_OK;
}

extern "C" pfc_status pfc_hflow_batch_field(pfc_hflow_batch* b, const void* const* A, void* const* ut,
                                            pfc_stream stream)
{
    if (!b) return hfail(PFC_EINVAL, "hflow batch: handle is NULL");
    if (!is_current(b->device)) return hfail(PFC_EINVAL, "hflow batch: the batch's device is not the current device");
    pfc_status st;
    if ((st = check_vec_list(A, b->n, "A")) || (st = check_vec_list(ut, b->n, "ut"))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    HCU(batch_field(b, (const float* const*)A, 0, s));
    for (int k = 0; k < b->n; ++k)
        HCU(cudaMemcpyAsync(ut[k], bbuf(b, k, 0), sizeof(float) * b->N, cudaMemcpyDeviceToDevice, s));
    return PFC_OK;
}

extern "C" pfc_status pfc_hflow_batch_run(pfc_hflow_batch* b, void* const* A, void* const* m, void* const* v,
                                          int32_t nsteps, int32_t* t, double* trace_host, pfc_stream stream)
{
    nvtxRangePushA("pfc_hflow_batch_run");
    struct Pop { ~Pop() { nvtxRangePop(); } } pop_;
    if (!b) return hfail(PFC_EINVAL, "hflow batch: handle is NULL");
    if (!is_current(b->device)) return hfail(PFC_EINVAL, "hflow batch: the batch's device is not the current device");
    pfc_status st;
    if ((st = check_vec_list(A, b->n, "A")) || (st = check_vec_list(m, b->n, "m")) ||
        (st = check_vec_list(v, b->n, "v")))
        return st;
    for (int k = 0; k < b->n; ++k)
        if (A[k] == m[k] || A[k] == v[k] || m[k] == v[k])
            return hfail(PFC_EINVAL, "hflow batch: A, m and v of an instance must be distinct");
    if (!t || *t < 0 || nsteps < 0) return hfail(PFC_EINVAL, "hflow batch: nsteps >= 0 and a step counter >= 0 required");
    if (nsteps == 0) return PFC_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (nsteps > b->trace_cap) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        HCU(cudaStreamSynchronize(s));   // this stream only (a device-wide wait breaks other threads' captures)
        cudaFree(b->trace);
        b->trace = nullptr;
        b->trace_cap = 0;
        HCU(cudaMalloc((void**)&b->trace, sizeof(double) * 5 * (size_t)nsteps * b->n));
        b->trace_cap = nsteps;
    }
    std::vector<unsigned> ti((size_t)4 * b->n, 0u);
    for (int k = 0; k < b->n; ++k) ti[(size_t)4 * k + 1] = (unsigned)*t;
    HCU(cudaMemcpyAsync(b->fints, ti.data(), sizeof(unsigned) * ti.size(), cudaMemcpyHostToDevice, s));
    HCU(cudaMemsetAsync(b->sints, 0, sizeof(unsigned) * NINTS * b->n, s));
    float* const* Af = (float* const*)A;
    float* const* mf = (float* const*)m;
    float* const* vf = (float* const*)v;
    auto enqueue = [&](int cnt, cudaStream_t st2) -> cudaError_t {
        for (int i = 0; i < cnt; ++i) {
            cudaError_t e = batch_step(b, Af, mf, vf, st2);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    const int G = nsteps >= 32 ? 32 : 0;
    if (G) {
        std::vector<const void*> key;
        for (int k = 0; k < b->n; ++k) {
            key.push_back(A[k]);
            key.push_back(m[k]);
            key.push_back(v[k]);
        }
        if (!(b->gexec && b->gkey == key && b->glen == G && b->gtrace == b->trace)) {
            if (b->gexec) {
                cudaGraphExecDestroy(b->gexec);
                b->gexec = nullptr;
            }
            cudaGraph_t graph = nullptr;
            HCU(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = enqueue(G, b->cap);
            cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                (void)cudaGetLastError();
                return hfail(PFC_ECUDA, "hflow batch: graph capture failed");
            }
            e = cudaGraphInstantiate(&b->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                b->gexec = nullptr;
                (void)cudaGetLastError();
                return hfail(PFC_ECUDA, "hflow batch: graph instantiation failed");
            }
            b->gkey = key;
            b->glen = G;
            b->gtrace = b->trace;
        }
        for (int k = 0; k + G <= nsteps; k += G) HCU(cudaGraphLaunch(b->gexec, s));
    }
    const int done = G ? (nsteps / G) * G : 0;
    HCU(enqueue(nsteps - done, s));
    std::vector<unsigned> back((size_t)4 * b->n);
    HCU(cudaMemcpyAsync(back.data(), b->fints, sizeof(unsigned) * back.size(), cudaMemcpyDeviceToHost, s));
    if (trace_host)
        for (int k = 0; k < b->n; ++k)
            HCU(cudaMemcpyAsync(trace_host + (size_t)k * 5 * nsteps, b->trace + (size_t)k * 5 * b->trace_cap,
                                sizeof(double) * 5 * (size_t)nsteps, cudaMemcpyDeviceToHost, s));
    HCU(cudaStreamSynchronize(s));
    for (int k = 0; k < b->n; ++k)
        if (back[(size_t)4 * k + 2] != (unsigned)nsteps) return hfail(PFC_ECUDA, "hflow batch: step count mismatch");
    *t = (int32_t)back[1];
    return PFC_OK;
}
