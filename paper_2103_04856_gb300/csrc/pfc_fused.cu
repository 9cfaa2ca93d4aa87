// pfc_fused.cu -- the fused forward + adjoint stencil sweep.
//
// One CTA owns an output tile of 32 x TY columns (x, y) and marches through a
// chunk of z planes.  For every plane m it
//   1. evaluates eq. Feps and the local reverse mode (pfc_device.cuh) on the
//      tile plus a one-column halo ring, from a ring of u planes in shared
//      memory that cp.async keeps PD planes ahead;
//   2. keeps the z-direction adjoint terms of its own column in registers
//      (first/second z differences and the z parts of the xz / yz mixed
//      differences), so that only five x/y fields per plane go through shared
//      memory;
//   3. one plane later, gathers the transposed stencil (the exact gradient of
//      the discrete sum) for the tile and writes either g or the descent
//      update u - tau g.
// Nothing but u is read from HBM and nothing but the result is written; the
// cotangents are recomputed per tile instead of stored.  The energy and the
// gradient sums are reduced per CTA in FP64 and combined by the last CTA of
// the problem (pfc_device.cuh, grid_finish).
//
// EXT (the extended sweep): 1 = the orientation term of Sec. 5.2 and
// coefficients read per voxel from a field c(x) (each thread loads the six
// coefficients of its column one plane ahead of their use); 2 = the same
// with the tangent-projected M = -eps P Hess u P.
#include <type_traits>

#include "pfc_device.cuh"

namespace pfc {

constexpr int TX = 32;      // output columns per tile in x
constexpr int UXP = 40;     // u tile row in shared memory: x0-4 .. x0+35
constexpr int NBUF = 8;     // ring of u planes
constexpr int PD = 3;       // planes in flight ahead of the plane being consumed

// Thread layout of a tile (TY rows of 32 output columns, plus a one-column
// halo ring whose cotangents the gather needs):
//   warps 0 .. TY-1 : interior rows, lane = x          (these also gather)
//   warps TY, TY+1  : the halo rows above and below the tile
//   then the left and right halo columns (TY+2 lanes each): one warp for
//   both when 2 (TY+2) <= 32 (lanes 0..TY+1 left, the next TY+2 right),
//   else one warp each
// so every warp but the halo-column ones reads contiguous shared memory.
// The SM's four schedulers hold the warps round-robin, and each has a
// quarter of the register file: TY = 13 (16 warps, 4 per scheduler) may use
// 128 registers per thread, TY = 16 (20 warps, 5 per scheduler) only 96.
template <int TY>
struct Tile {
    static constexpr int EX = TX + 2;             // extended (halo) columns in x
    static constexpr int EY = TY + 2;
    static constexpr int NEXT = EX * EY;
    static constexpr bool MERGED = 2 * (TY + 2) <= 32;
    static constexpr int NT = (TY + (MERGED ? 3 : 4)) * 32;
    static constexpr int UY = TY + 4;             // u rows: y0-2 .. y0+TY+1
    static constexpr int PLANE = UY * UXP;
};

__device__ __forceinline__ int wrapi(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ void cp_async16(void* s, const void* g)
{
    unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_elem(float* s, const float* g)
{
    unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double* s, const double* g)
{
    unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename T, int TY, int MODE, int MAXI, int EXT = 0>
__global__ void __launch_bounds__(Tile<TY>::NT, 1)
k_fused(const __grid_constant__ Launch<T, MAXI> L)
{
    using TL = Tile<TY>;
    constexpr int EX = TL::EX, NEXT = TL::NEXT, NT = TL::NT, UY = TL::UY, PLANE = TL::PLANE;
    constexpr int VEC = 16 / (int)sizeof(T);
    constexpr int NCH = UXP / VEC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* us = reinterpret_cast<T*>(smem_raw);            // [NBUF][UY][UXP]
    T* fs = us + NBUF * PLANE;                          // [2][5][NEXT]
    float* scr = reinterpret_cast<float*>(fs + 2 * 5 * NEXT);   // [NPART][NT]
    __shared__ double tot[NPART];

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    int ex, ey;                                   // extended column of this thread
    bool active = true;
    if (warp < TY) { ey = warp + 1; ex = lane + 1; }
    else if (warp == TY) { ey = 0; ex = lane + 1; }
    else if (warp == TY + 1) { ey = TY + 1; ex = lane + 1; }
    else if (TL::MERGED) {   // both halo columns; lanes past them duplicate the last row, never publish
        const bool left = lane < TY + 2;
        ex = left ? 0 : EX - 1;
        ey = left ? lane : (lane - (TY + 2) < TY + 2 ? lane - (TY + 2) : TY + 1);
        active = lane < 2 * (TY + 2);
    } else {   // one halo column per warp; lanes past the last row duplicate it and never publish
        ex = warp == TY + 2 ? 0 : EX - 1;
        ey = lane < TY + 2 ? lane : TY + 1;
        active = lane < TY + 2;
    }
    const bool rowwarp = warp < TY;               // the warps that gather
    // warps whose threads copy u planes (vector path: one 16-byte chunk per
    // thread; element path: every warp)
    constexpr int LOADWARPS = (UY * NCH + 31) / 32;
    const int uc = (ey + 1) * UXP + ex + 3;       // this column in a u plane
    const int fc = ey * EX + ex;                  // this column in a field plane

    // per-thread sums of the problem being processed, in the arithmetic type
    // (a few hundred terms each), combined in FP64 across threads and CTAs
    T se = 0, su = 0, sg = 0, sag = 0, gmax = 0, sout = 0;
    int cur = -1;                                 // problem the sums belong to
    auto flush = [&]() {
        const T v[NPART] = { se, su, sg, sag, gmax, sout };
        block_sums<NT>(v, scr, tot);
        const Inst<T>& pin = L.inst[cur];
        finish_problem(pin, (int)blockIdx.x - pin.first_block, MODE, tot);
        se = su = sg = sag = gmax = sout = 0;
    };

    // this CTA's share of the work units
    const long long W = L.units;
    long long U = (long long)blockIdx.x * W / L.grid;
    const long long Uend = ((long long)blockIdx.x + 1) * W / L.grid;
    while (U < Uend) {
        // ---- the run: one column tile of one problem, a contiguous z range
        int k = 0;
        if (MAXI > 1) {
            int hi = L.n - 1;
            while (k < hi) {
                const int mid = (k + hi + 1) >> 1;
                if (L.inst[mid].unit_base <= U) k = mid; else hi = mid - 1;
            }
        }
        if (k != cur) {
            if (cur >= 0) flush();
            cur = k;
        }
        const Inst<T>& in = L.inst[k];
        const int nx = in.nx, ny = in.ny, nz = in.nz;
        const long long rel = U - in.unit_base;
        const int ct = (int)(rel / nz);
        const int z0 = (int)(rel - (long long)ct * nz);
        const long long run_end = min(Uend, in.unit_base + (long long)(ct + 1) * nz);
        const int zend = z0 + (int)(run_end - U);      // exclusive
        U = run_end;
        const int x0 = (ct % in.tiles_x) * TX, y0 = (ct / in.tiles_x) * TY;
        const int plast = zend + 1;                    // last u plane needed
        const size_t plane_g = (size_t)nx * ny;
        const int gx = x0 + ex - 1, gy = y0 + ey - 1;
        const bool interior = warp < TY && gx < nx && gy < ny;
        const bool loader = !in.vec || warp < LOADWARPS;

        // ---- loads: every u plane of the tile, periodic in x, y and z
        int ld_off = -1, ld_dst = 0;
        if (in.vec && tid < UY * NCH) {
            const int r = tid / NCH, c = tid - (tid / NCH) * NCH;
            ld_off = wrapi(y0 - 2 + r, ny) * nx + wrapi(x0 - 4 + c * VEC, nx);
            ld_dst = r * UXP + c * VEC;
        }
        int pz = wrapi(z0 - 2, nz);                // planes are issued in increasing order
        auto issue = [&](int p) {
            if (!loader) return;                   // warp-uniform: only loading warps copy, commit and wait
            if (p <= plast) {
                T* dst = us + (p & (NBUF - 1)) * PLANE;
                const T* src = in.u + (size_t)pz * plane_g;
                if (in.vec) {
                    if (ld_off >= 0) cp_async16(dst + ld_dst, src + ld_off);
                } else {
                    for (int i = tid; i < PLANE; i += NT) {
                        const int r = i / UXP, c = i - (i / UXP) * UXP;
                        cp_async_elem(dst + i, src + wrapi(y0 - 2 + r, ny) * nx + wrapi(x0 - 4 + c, nx));
                    }
                }
            }
            cp_async_commit();   // one group per plane slot, empty past the run
            pz = pz + 1 == nz ? 0 : pz + 1;
        };

#if PFC_DEBUG
        // debug builds: every shared value starts as NaN, so a read of a cell
        // that no load or publish of this run wrote shows up in the results
        for (int i = tid; i < NBUF * PLANE + 2 * 5 * NEXT; i += NT) us[i] = T(NAN);
        __syncthreads();
#endif
        const double cind = (MODE == MODE_STEP) ? in.scal[S_C] : 0.0;
        const T cin = (T)cind;

        // EXT: c(x) of this thread's (wrapped) column, one plane ahead
        const T* cfp = nullptr;
        size_t cf_stride = 0;
        T ccn[NCF];
        if constexpr (EXT) {
            if (in.cf) {
                cfp = in.cf + (size_t)wrapi(gy, ny) * nx + wrapi(gx, nx);
                cf_stride = plane_g * nz;
            }
        }
        auto load_c = [&](int m) {
            if constexpr (EXT) {
                if (cfp) {
                    const T* q = cfp + (size_t)wrapi(m, nz) * plane_g;
#pragma unroll
                    for (int k = 0; k < NCF; ++k) ccn[k] = __ldg(q + k * cf_stride);
                }
            }
        };
        load_c(z0 - 1);

        // ---- per-column state carried from plane to plane
        T accC = 0, zdn = 0, hxz2 = 0, hyz2 = 0, hxz1 = 0, hyz1 = 0;
        T fx1 = 0, fx2 = 0, fy1 = 0, fy2 = 0, fxy = 0, cpend = 0;

        T* optr = in.out + (size_t)z0 * plane_g + (size_t)gy * nx + gx;   // planes gathered in order
        auto gather = [&](int kz) {   // row warps; lanes past a ragged edge only skip the store
            const T* F = fs + (kz & 1) * 5 * NEXT;
            const int c = fc;
            const T gv = cpend + F[c - 1] + F[NEXT + c + 1] + F[2 * NEXT + c - EX] + F[3 * NEXT + c + EX]
                       + (F[4 * NEXT + c - 1 - EX] - F[4 * NEXT + c - 1 + EX])
                       - (F[4 * NEXT + c + 1 - EX] - F[4 * NEXT + c + 1 + EX]);
            const T g = interior ? gv : T(0);
            const T ag = g < T(0) ? -g : g;
            sg += g;
            sag += ag;
            gmax = ag > gmax ? ag : gmax;
            if (MODE == MODE_GRAD) {
                if (interior) *optr = g;
            } else {
                const T u0 = us[(kz & (NBUF - 1)) * PLANE + uc] + cin;
                const T v = fma_(-in.tau, g, u0);
                if (interior) *optr = v;
                su += interior ? u0 : T(0);
                sout += interior ? v : T(0);
            }
            optr += plane_g;
        };

        for (int p = z0 - 2; p <= z0 + PD - 1; ++p) issue(p);

        // One plane m of the march.  GATHER: write plane m-2; PUBLISH: plane
        // m-1 is complete, publish its x/y fields; OWN: plane m is in the
        // run (its energy counts).  All three are compile-time constants, so
        // the steady state (all true) has no phase tests.
        auto plane = [&](int m, auto GATHER, auto PUBLISH, auto OWN) {
            constexpr bool kGather = decltype(GATHER)::value, kPublish = decltype(PUBLISH)::value;
            (void)kPublish;
            constexpr bool kOwn = decltype(OWN)::value;
            // EXT: this plane's coefficients; start the next plane's loads
            Coef<T> Cv;
            if constexpr (EXT) {
                Cv = in.C;
                if (cfp) {
                    Cv.c1 = ccn[0]; Cv.c2 = ccn[1]; Cv.c3 = ccn[2];
                    Cv.c4 = ccn[3]; Cv.c5 = ccn[4]; Cv.c6 = ccn[5];
                }
                load_c(m + 1);
            }
            if (loader) cp_async_wait<PD - 1>();
            __syncthreads();
            if constexpr (kGather && MODE != MODE_ENERGY) {
                if (rowwarp) gather(m - 2);
            }
            issue(m + 1 + PD);
            if constexpr (MODE == MODE_ENERGY && !kOwn) return;
            const T* pm = us + ((m - 1) & (NBUF - 1)) * PLANE + uc;
            const T* p0 = us + (m & (NBUF - 1)) * PLANE + uc;
            const T* pp = us + ((m + 1) & (NBUF - 1)) * PLANE + uc;
            const T u0 = p0[0];
            const T dx = p0[1] - p0[-1];
            const T dy = p0[UXP] - p0[-UXP];
            const T dz = pp[0] - pm[0];
            const T hxx = (p0[1] + p0[-1]) - T(2) * u0;
            const T hyy = (p0[UXP] + p0[-UXP]) - T(2) * u0;
            const T hzz = (pp[0] + pm[0]) - T(2) * u0;
            const T hxy = (p0[UXP + 1] - p0[UXP - 1]) - (p0[-UXP + 1] - p0[-UXP - 1]);
            const T hxz = (pp[1] - pp[-1]) - (pm[1] - pm[-1]);
            const T hyz = (pp[UXP] - pp[-UXP]) - (pm[UXP] - pm[-UXP]);
            Cot<T> ctv;
            const Coef<T>& CC = [&]() -> const Coef<T>& {
                if constexpr (EXT) return Cv;
                else return in.C;
            }();
            // FP64 re-evaluation of D from the exact float inputs (float path only)
            auto refine = [&]() -> T {
                if constexpr (EXT == 2) return discriminant_fp64_proj_at<T>(in.C.R, pm, p0, pp, UXP);
                else return discriminant_fp64_at<T>(in.C.R, in.C.well, pm, p0, pp, UXP, cind);
            };
            if constexpr (MODE == MODE_ENERGY) {
                const T e = voxel_eval<T, false, EXT != 0, EXT == 2>(CC, u0 + cin, dx, dy, dz, hxx, hyy, hzz, hxy, hxz, hyz, ctv, refine);
                se += interior ? e : T(0);
                return;
            } else {
                const T e = voxel_eval<T, true, EXT != 0, EXT == 2>(CC, u0 + cin, dx, dy, dz, hxx, hyy, hzz, hxy, hxz, hyz, ctv, refine);
                if constexpr (kOwn) se += interior ? e : T(0);
                // transposed-stencil pieces of this voxel (see the gather):
                //   x/y first+second differences read from the left/right neighbour,
                //   z pieces from the planes below/above, the centre term stays here
                const T X1 = ctv.dx + ctv.hxx, X2 = ctv.hxx - ctv.dx;
                const T Y1 = ctv.dy + ctv.hyy, Y2 = ctv.hyy - ctv.dy;
                const T zd = ctv.dz + ctv.hzz, zu = ctv.hzz - ctv.dz;
                const T cpart = ctv.u - T(2) * (ctv.hxx + ctv.hyy + ctv.hzz);
                if constexpr (kPublish) {   // plane m-1 is complete
                    cpend = accC + zu;
                    const T dxz = hxz2 - ctv.hxz, dyz = hyz2 - ctv.hyz;
                    T* F = fs + ((m - 1) & 1) * 5 * NEXT + fc;
                    if (active) {
                        F[0] = fx1 + dxz;
                        F[NEXT] = fx2 - dxz;
                        F[2 * NEXT] = fy1 + dyz;
                        F[3 * NEXT] = fy2 - dyz;
                        F[4 * NEXT] = fxy;
                    }
                }
                accC = cpart + zdn;
                zdn = zd;
                hxz2 = hxz1; hyz2 = hyz1;
                hxz1 = ctv.hxz; hyz1 = ctv.hyz;
                fx1 = X1; fx2 = X2; fy1 = Y1; fy2 = Y2; fxy = ctv.hxy;
            }
        };
        using Y = std::true_type;
        using N = std::false_type;
        plane(z0 - 1, N{}, N{}, N{});
        plane(z0, N{}, N{}, Y{});
        if (zend - z0 == 1) {
            plane(z0 + 1, N{}, Y{}, N{});
        } else {
            plane(z0 + 1, N{}, Y{}, Y{});
#pragma unroll 1
            for (int m = z0 + 2; m < zend; ++m) plane(m, Y{}, Y{}, Y{});
            plane(zend, Y{}, Y{}, N{});
        }
        if (MODE != MODE_ENERGY) {
            __syncthreads();
            if (rowwarp) gather(zend - 1);
        }
        cp_async_wait<0>();
        __syncthreads();   // the ring and the field planes are reused by the next run
    }
    if (cur >= 0) flush();
}

// ------------------------------------------------------------ small kernels

template <typename T>
__global__ void k_add_offset(T* __restrict__ out, const T* __restrict__ in, long n, const double* c)
{
    const T off = (T)(*c);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        out[i] = in[i] + off;
}

// Batched form: blockIdx.y selects the problem; out[i] += its offset.
struct OffsetLaunch {
    int n;
    float* out[BATCH_MAX];
    const double* c[BATCH_MAX];
    long len[BATCH_MAX];
    int vec[BATCH_MAX];      // 1: out is 16-byte aligned (float4 accesses, scalar tail)
};
__global__ void k_add_offset_batch(const __grid_constant__ OffsetLaunch L)
{
    const int k = blockIdx.y;
    const float off = (float)(*L.c[k]);
    float* out = L.out[k];
    const long n = L.len[k];
    const long t0 = blockIdx.x * (long)blockDim.x + threadIdx.x, stride = (long)gridDim.x * blockDim.x;
    long done = 0;
    if (L.vec[k]) {
        float4* o4 = reinterpret_cast<float4*>(out);
        const long n4 = n >> 2;
        for (long i = t0; i < n4; i += stride) {
            float4 v = o4[i];
            v.x += off; v.y += off; v.z += off; v.w += off;
            o4[i] = v;
        }
        done = n4 << 2;
    }
    for (long i = done + t0; i < n; i += stride) out[i] += off;
}

// Diffuse principal curvatures (Sec. 3.1, eqs. kepsa/kepsb) per voxel.
template <typename T>
__global__ void k_curvatures(const T* __restrict__ u, T* __restrict__ k1, T* __restrict__ k2, int nx,
                             int ny, int nz, Coef<T> C, T eps)
{
    const long n = (long)nx * ny * nz;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long)nx * ny));
        auto at = [&](int dx, int dy, int dz) {
            return u[((long)wrapi(z + dz, nz) * ny + wrapi(y + dy, ny)) * nx + wrapi(x + dx, nx)];
        };
        const T u0 = at(0, 0, 0);
        const T dx = at(1, 0, 0) - at(-1, 0, 0), dy = at(0, 1, 0) - at(0, -1, 0), dz = at(0, 0, 1) - at(0, 0, -1);
        const T hxx = at(1, 0, 0) + at(-1, 0, 0) - T(2) * u0;
        const T hyy = at(0, 1, 0) + at(0, -1, 0) - T(2) * u0;
        const T hzz = at(0, 0, 1) + at(0, 0, -1) - T(2) * u0;
        const T hxy = at(1, 1, 0) - at(1, -1, 0) - at(-1, 1, 0) + at(-1, -1, 0);
        const T hxz = at(1, 0, 1) - at(1, 0, -1) - at(-1, 0, 1) + at(-1, 0, -1);
        const T hyz = at(0, 1, 1) - at(0, 1, -1) - at(0, -1, 1) + at(0, -1, -1);
        const T Gx = dx * C.sg, Gy = dy * C.sg, Gz = dz * C.sg;
        const T rho = Gx * Gx + Gy * Gy + Gz * Gz + C.xi2;
        T Mxx, Myy, Mzz, Mxy, Mxz, Myz;
        if (C.proj) {   // M = P K P, K = -eps Hess u, P = I - G G^T / rho
            const T Kxx = C.kd * hxx, Kyy = C.kd * hyy, Kzz = C.kd * hzz;
            const T Kxy = C.ko * hxy, Kxz = C.ko * hxz, Kyz = C.ko * hyz;
            const T kx = Kxx * Gx + Kxy * Gy + Kxz * Gz, ky = Kxy * Gx + Kyy * Gy + Kyz * Gz;
            const T kz = Kxz * Gx + Kyz * Gy + Kzz * Gz;
            const T s = Gx * kx + Gy * ky + Gz * kz;
            const T ir = T(1) / rho, s2 = s * ir * ir;
            Mxx = Kxx - T(2) * ir * Gx * kx + s2 * Gx * Gx;
            Myy = Kyy - T(2) * ir * Gy * ky + s2 * Gy * Gy;
            Mzz = Kzz - T(2) * ir * Gz * kz + s2 * Gz * Gz;
            Mxy = Kxy - ir * (Gx * ky + kx * Gy) + s2 * Gx * Gy;
            Mxz = Kxz - ir * (Gx * kz + kx * Gz) + s2 * Gx * Gz;
            Myz = Kyz - ir * (Gy * kz + ky * Gz) + s2 * Gy * Gz;
        } else {
            const T wp = C.well == 0 ? T(2) * u0 * (T(1) - u0) * (T(1) - T(2) * u0) : u0 * u0 * u0 - u0;
            const T wr = wp * C.inv_eps / rho;
            Mxx = C.kd * hxx + wr * Gx * Gx; Myy = C.kd * hyy + wr * Gy * Gy; Mzz = C.kd * hzz + wr * Gz * Gz;
            Mxy = C.ko * hxy + wr * Gx * Gy; Mxz = C.ko * hxz + wr * Gx * Gz; Myz = C.ko * hyz + wr * Gy * Gz;
        }
        const T Tr = Mxx + Myy + Mzz;
        const T S = Mxx * Mxx + Myy * Myy + Mzz * Mzz + T(2) * (Mxy * Mxy + Mxz * Mxz + Myz * Myz);
        const T D = T(2) * S - Tr * Tr;
        const T root = sqrt_(D > T(0) ? D : T(0));
        const T den = T(2) * eps * sqrt_(rho);
        k1[i] = (Tr + root) / den;
        k2[i] = (Tr - root) / den;
    }
}

// ------------------------------------------------------------ host side

template <typename T>
Coef<T> make_coef(const double a[6], double h, double eps, double xi, int well, double mu, const double* theta,
                  int proj)
{
    const double h3 = h * h * h;
    Coef<T> C;
    C.c1 = (T)((a[0] + a[2] - a[1]) / (2.0 * eps) * h3);
    C.c2 = (T)(a[1] / (2.0 * eps) * h3);
    C.c3 = (T)((a[0] - a[2]) / (2.0 * eps) * h3);
    C.c4 = (T)((a[3] + a[4]) / 2.0 * h3);
    C.c5 = (T)((a[3] - a[4]) / 2.0 * h3);
    C.c6 = (T)(a[5] * eps * h3);
    C.kd = (T)(-eps / (h * h));
    C.ko = (T)(-eps / (4.0 * h * h));
    C.sg = (T)(1.0 / (2.0 * h));
    C.inv_eps = (T)(1.0 / eps);
    C.xi = (T)xi;
    C.xi2 = (T)(xi * xi);
    C.inv_xi = (T)(1.0 / xi);
    C.well = well;
    C.R.kd = -eps / (h * h);
    C.R.ko = -eps / (4.0 * h * h);
    C.R.sg = 1.0 / (2.0 * h);
    C.R.inv_eps = 1.0 / eps;
    C.R.xi2 = xi * xi;
    C.c7 = (T)(eps * mu * h3);
    C.th0 = (T)(theta ? theta[0] : 0.0);
    C.th1 = (T)(theta ? theta[1] : 0.0);
    C.th2 = (T)(theta ? theta[2] : 0.0);
    C.proj = proj ? 1 : 0;
    C.sym = (C.c3 == T(0) && C.c5 == T(0)) ? 1 : 0;
    return C;
}
template Coef<float> make_coef<float>(const double*, double, double, double, int, double, const double*, int);
template Coef<double> make_coef<double>(const double*, double, double, double, int, double, const double*, int);

// c(x) from a(x): the coefficients of eq. Feps (times h^3) per voxel, in FP64
// then rounded to the arithmetic type, exactly as make_coef does for a constant a.
template <typename T>
__global__ void k_coef_field(const T* __restrict__ a, T* __restrict__ c, long n, double h3, double eps)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double a20 = a[i], a11 = a[n + i], a02 = a[2 * n + i];
        const double a10 = a[3 * n + i], a01 = a[4 * n + i], a00 = a[5 * n + i];
        c[i] = (T)((a20 + a02 - a11) / (2.0 * eps) * h3);
        c[n + i] = (T)(a11 / (2.0 * eps) * h3);
        c[2 * n + i] = (T)((a20 - a02) / (2.0 * eps) * h3);
        c[3 * n + i] = (T)((a10 + a01) / 2.0 * h3);
        c[4 * n + i] = (T)((a10 - a01) / 2.0 * h3);
        c[5 * n + i] = (T)(a00 * eps * h3);
    }
}

template <typename T>
cudaError_t launch_coef_field(const T* a_field, T* c_field, long n, double h, double eps, cudaStream_t s)
{
    const long b = (n + 255) / 256;
    k_coef_field<T><<<(unsigned)(b < 4096 ? b : 4096), 256, 0, s>>>(a_field, c_field, n, h * h * h, eps);
    return cudaGetLastError();
}
template cudaError_t launch_coef_field<float>(const float*, float*, long, double, double, cudaStream_t);
template cudaError_t launch_coef_field<double>(const double*, double*, long, double, double, cudaStream_t);

int fused_threads(int tile_y) { return tile_y == 8 ? Tile<8>::NT : tile_y == 13 ? Tile<13>::NT : Tile<16>::NT; }

size_t fused_smem_bytes(int elem_size, int tile_y)
{
    const int plane = tile_y == 8 ? Tile<8>::PLANE : tile_y == 13 ? Tile<13>::PLANE : Tile<16>::PLANE;
    const int next = tile_y == 8 ? Tile<8>::NEXT : tile_y == 13 ? Tile<13>::NEXT : Tile<16>::NEXT;
    const int nt = tile_y == 8 ? Tile<8>::NT : tile_y == 13 ? Tile<13>::NT : Tile<16>::NT;
    return (size_t)elem_size * ((size_t)NBUF * plane + 2 * 5 * (size_t)next) + sizeof(float) * NPART * (size_t)nt;
}

template <typename T, int TY, int MODE, int MAXI, int EXT = 0>
static cudaError_t launch_one(const Launch<T, MAXI>& L, int blocks, cudaStream_t s)
{
    const size_t smem = fused_smem_bytes(sizeof(T), TY);
    static bool attr_done = false;   // per instantiation; idempotent, so a race is harmless
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_fused<T, TY, MODE, MAXI, EXT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    k_fused<T, TY, MODE, MAXI, EXT><<<blocks, Tile<TY>::NT, smem, s>>>(L);
    return cudaGetLastError();
}

static int sm_count_current()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        (void)cudaGetLastError();
        n = 152;
    }
    return n;
}

long long fused_grid(long long units, int max_run)
{
    long long G = sm_count_current();                   // one CTA per SM
    if (max_run > 0 && (units + max_run - 1) / max_run > G) G = (units + max_run - 1) / max_run;
    return G < units ? G : units;
}

long long fused_slots(int nx, int ny, int nz, int tile_y, int max_run)
{
    const long long tx = (nx + TX - 1) / TX;
    const long long a = fused_grid(tx * ((ny + tile_y - 1) / tile_y) * nz, max_run);
    const long long b = fused_grid(tx * ((ny + EXT_TILE_Y - 1) / EXT_TILE_Y) * nz, max_run);
    return a > b ? a : b;
}

// Split the launch's work units evenly over G CTAs and record, per problem,
// the first CTA that holds a partial of it and how many do.
template <typename T, int MAXI>
static void plan(Launch<T, MAXI>& L, int tile_y, int max_run)
{
    long long W = 0;
    for (int k = 0; k < L.n; ++k) {
        Inst<T>& in = L.inst[k];
        in.tiles_x = (in.nx + TX - 1) / TX;
        in.tiles_y = (in.ny + tile_y - 1) / tile_y;
        in.unit_base = W;
        W += (long long)in.tiles_x * in.tiles_y * in.nz;
    }
    const long long G = fused_grid(W, max_run);
    L.units = W;
    L.grid = (int)G;
    for (int k = 0; k < L.n; ++k) {
        Inst<T>& in = L.inst[k];
        const long long a = in.unit_base, b = a + (long long)in.tiles_x * in.tiles_y * in.nz - 1;
        const int c0 = (int)(((a + 1) * G - 1) / W), c1 = (int)(((b + 1) * G - 1) / W);
        in.first_block = c0;
        in.nblocks = c1 - c0 + 1;
    }
}

template <typename T, int TY, int EXT = 0>
static cudaError_t launch_mode(const Inst<T>& in, int mode, int max_run, cudaStream_t s)
{
    Launch<T, 1> L;
    L.n = 1;
    L.inst[0] = in;
    plan(L, TY, max_run);
    switch (mode) {
    case MODE_ENERGY: return launch_one<T, TY, MODE_ENERGY, 1, EXT>(L, L.grid, s);
    case MODE_GRAD: return launch_one<T, TY, MODE_GRAD, 1, EXT>(L, L.grid, s);
    case MODE_STEP: return launch_one<T, TY, MODE_STEP, 1, EXT>(L, L.grid, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_fused(const Inst<T>& in, int mode, int tile_y, int max_run, cudaStream_t s)
{
    if (in.C.proj) return launch_mode<T, EXT_TILE_Y, 2>(in, mode, max_run, s);
    if (needs_ext(in)) return launch_mode<T, EXT_TILE_Y, 1>(in, mode, max_run, s);
    if (tile_y == 8) return launch_mode<T, 8>(in, mode, max_run, s);
    if (tile_y == 13) return launch_mode<T, 13>(in, mode, max_run, s);
    return launch_mode<T, 16>(in, mode, max_run, s);
}
template cudaError_t launch_fused<float>(const Inst<float>&, int, int, int, cudaStream_t);
template cudaError_t launch_fused<double>(const Inst<double>&, int, int, int, cudaStream_t);

// Batches of up to BATCH_MAX problems go in one launch (their descriptors
// travel as kernel parameters); larger batches take one launch per group.
// MODE_STEP (descent steps) or MODE_GRAD (energies and gradients).
cudaError_t launch_fused_batch(const Inst<float>* insts, int n_inst, int tile_y, int max_run, cudaStream_t s,
                               int mode)
{
    if (mode != MODE_STEP && mode != MODE_GRAD) return cudaErrorInvalidValue;
    thread_local Launch<float, BATCH_MAX> L;   // host staging (per thread); the launch copies it
    for (int g0 = 0; g0 < n_inst; g0 += BATCH_MAX) {
        const int cnt = n_inst - g0 < BATCH_MAX ? n_inst - g0 : BATCH_MAX;
        L.n = cnt;
        for (int k = 0; k < cnt; ++k) L.inst[k] = insts[g0 + k];
        plan(L, tile_y, max_run);
        cudaError_t e;
        if (mode == MODE_STEP)
            e = tile_y == 8    ? launch_one<float, 8, MODE_STEP, BATCH_MAX>(L, L.grid, s)
                : tile_y == 13 ? launch_one<float, 13, MODE_STEP, BATCH_MAX>(L, L.grid, s)
                               : launch_one<float, 16, MODE_STEP, BATCH_MAX>(L, L.grid, s);
        else
            e = tile_y == 8    ? launch_one<float, 8, MODE_GRAD, BATCH_MAX>(L, L.grid, s)
                : tile_y == 13 ? launch_one<float, 13, MODE_GRAD, BATCH_MAX>(L, L.grid, s)
                               : launch_one<float, 16, MODE_GRAD, BATCH_MAX>(L, L.grid, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_add_offset(T* out, const T* in, long n, const double* c, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_add_offset<T><<<(int)blocks, 256, 0, s>>>(out, in, n, c);
    return cudaGetLastError();
}
template cudaError_t launch_add_offset<float>(float*, const float*, long, const double*, cudaStream_t);
template cudaError_t launch_add_offset<double>(double*, const double*, long, const double*, cudaStream_t);

cudaError_t launch_add_offset_batch(const Inst<float>* insts, int n_inst, cudaStream_t s)
{
    thread_local OffsetLaunch L;   // host staging (per thread)
    for (int g0 = 0; g0 < n_inst; g0 += BATCH_MAX) {
        const int cnt = n_inst - g0 < BATCH_MAX ? n_inst - g0 : BATCH_MAX;
        L.n = cnt;
        for (int k = 0; k < cnt; ++k) {
            const Inst<float>& in = insts[g0 + k];
            L.out[k] = in.out;
            L.c[k] = in.scal + S_C;
            L.len[k] = (long)in.nx * in.ny * in.nz;
            L.vec[k] = ((uintptr_t)in.out & 15) == 0;
        }
        int bx = (152 * 8 + cnt - 1) / cnt;
        if (bx < 8) bx = 8;
        k_add_offset_batch<<<dim3(bx, cnt), 256, 0, s>>>(L);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_curvatures(const T* u, T* k1, T* k2, int nx, int ny, int nz, const Coef<T>& C, double eps,
                              cudaStream_t s)
{
    const long n = (long)nx * ny * nz;
    long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_curvatures<T><<<(int)blocks, 256, 0, s>>>(u, k1, k2, nx, ny, nz, C, (T)eps);
    return cudaGetLastError();
}
template cudaError_t launch_curvatures<float>(const float*, float*, float*, int, int, int, const Coef<float>&,
                                              double, cudaStream_t);
template cudaError_t launch_curvatures<double>(const double*, double*, double*, int, int, int,
                                               const Coef<double>&, double, cudaStream_t);

}  // namespace pfc
