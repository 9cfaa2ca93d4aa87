// pfc_fused_kernel.cuh -- the fused forward + adjoint stencil sweep.
//
// One CTA owns an output tile of 32 x TY columns (x, y) and marches through a
// chunk of z planes.  For every plane m it
//   1. evaluates eq. Feps and the local reverse mode (pfc_device.cuh) on the
//      tile plus a one-column halo ring, from a ring of u planes in shared
//      memory that cp.async keeps PD planes ahead (each thread keeps the
//      stencil values of its column from the two planes below in registers,
//      so it reads only the plane above and four corners per plane);
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
//
// The template and its launch are shared by pfc_fused.cu (every sweep) and
// pfc_fused_sym.cu (the sweep for polynomials symmetric in kappa1, kappa2,
// whose sqrt(D+) terms have weight zero), so that the two sets of
// instantiations compile as separate translation units.
#pragma once

#include <type_traits>

#include "pfc_device.cuh"

namespace pfc {

constexpr int TX = 32;      // output columns per tile in x
constexpr int ULX = 40;     // u tile row loaded into shared memory: x0-4 .. x0+35
// the row's pitch in shared memory: 44 words, so that a halo-column warp,
// whose lanes read down a column (a stride of one pitch), meets 8 banks
// (12 i mod 32) instead of 4 (8 i mod 32 at a pitch of 40)
constexpr int UXP = 44;
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
// The row warps and the halo warps run separate compile-time instantiations
// of a run (no role tests in the march); the halo warps, which do not
// gather, also copy the u planes.
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
// CTA barrier for code whose warps take different (warp-uniform) paths: the
// row and halo warps run separate instantiations of the run body, each with
// the same sequence of barriers
__device__ __forceinline__ void bar_cta() { asm volatile("barrier.sync 0;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// SYM: every problem of the launch has c3 = c5 = 0 (FP32, EXT = 0 only): the
// sqrt(D+) terms, whose weight is exactly zero then, are not compiled in.
// HALO: the problem is a z-slab whose planes beyond its ends come from
// in.halo (instantiated only for slab launches, in pfc_fused_slab.cu: the
// check costs the other launches registers they do not have).
// UNI (batched launches, EXT = 0): every problem of the launch has the
// coefficients L.C0 and the step size L.tau0; per-voxel arithmetic takes them
// as constant-bank operands, where in.C at the run-time problem index costs a
// load per use (pfc_fused_uni.cu).
template <typename T, int TY, int MODE, int MAXI, int EXT = 0, bool SYM = false, bool HALO = false, bool UNI = false>
__global__ void __launch_bounds__(Tile<TY>::NT, 1)
k_fused(const __grid_constant__ Launch<T, MAXI> L)
{
    static_assert(!SYM || (EXT == 0 && sizeof(T) == 4), "the symmetric sweep is FP32 without extensions");
    using TL = Tile<TY>;
    constexpr int EX = TL::EX, NEXT = TL::NEXT, NT = TL::NT, UY = TL::UY, PLANE = TL::PLANE;
    constexpr int VEC = 16 / (int)sizeof(T);
    constexpr int NCH = ULX / VEC;
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
    // the halo warps copy the u planes (vector path: 16-byte chunks dealt
    // round-robin over their threads; element path: every warp)
    constexpr int HT = NT - TY * 32;
    constexpr int NLD = (UY * NCH + HT - 1) / HT;
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
        finish_problem(pin, (int)blockIdx.x - pin.first_block, MODE, tot, MAXI > 1);
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
        const bool interior0 = warp < TY && gx < nx && gy < ny;
        // batch steps: an instance whose scalars became non-finite in an
        // earlier step of the chain is retired (the flag is written only by
        // the finish of a launch, after every CTA has read it): its runs
        // write NaN and add nothing to its sums
        if constexpr (MAXI > 1 && MODE == MODE_STEP) {
            if (__ldcg(&in.ints[I_NONFINITE])) {
                if (interior0) {
                    T* o = in.out + (size_t)z0 * plane_g + (size_t)gy * nx + gx;
                    for (int z = z0; z < zend; ++z, o += plane_g) *o = T(NAN);
                }
                continue;
            }
        }

        using Y = std::true_type;
        using N = std::false_type;
        // The rest of the run, instantiated once for the row warps (ROLE =
        // true: they gather and write the tile) and once for the halo warps
        // (they evaluate the halo ring and copy the u planes), so that
        // neither path tests the warp's role
        auto body = [&](auto ROLE) {
            constexpr bool kRow = decltype(ROLE)::value;
            const bool interior = kRow && gx < nx && gy < ny;
            const T wI = interior ? T(1) : T(0);      // weight of this column's terms in the sums
            const bool loader = !in.vec || !kRow;
            // ---- loads: every u plane of the tile, periodic in x, y and z
            int ld_off[NLD], ld_dst[NLD];
#pragma unroll
            for (int j = 0; j < NLD; ++j) {
                ld_off[j] = -1; ld_dst[j] = 0;
                const int i = tid - TY * 32 + j * HT;
                if (!kRow && in.vec && i < UY * NCH) {
                    const int r = i / NCH, c = i - (i / NCH) * NCH;
                    ld_off[j] = wrapi(y0 - 2 + r, ny) * nx + wrapi(x0 - 4 + c * VEC, nx);
                    ld_dst[j] = r * UXP + c * VEC;
                }
            }
            int pz = wrapi(z0 - 2, nz);                // planes are issued in increasing order
            auto issue = [&](int p) {
                if (!loader) return;                   // warp-uniform: only loading warps copy, commit and wait
                if (p <= plast) {
                    T* dst = us + (p & (NBUF - 1)) * PLANE;
                    // a z-slab takes the planes beyond its ends from its halo buffer
                    const T* src = (HALO && (p < 0 || p >= nz)) ? in.halo + (size_t)(p < 0 ? p + 2 : p - nz + 2) * plane_g
                                                               : in.u + (size_t)pz * plane_g;
                    if (in.vec) {
#pragma unroll
                        for (int j = 0; j < NLD; ++j)
                            if (ld_off[j] >= 0) cp_async16(dst + ld_dst[j], src + ld_off[j]);
                    } else {
                        for (int i = tid; i < UY * ULX; i += NT) {
                            const int r = i / ULX, c = i - (i / ULX) * ULX;
                            cp_async_elem(dst + r * UXP + c, src + wrapi(y0 - 2 + r, ny) * nx + wrapi(x0 - 4 + c, nx));
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
            bar_cta();
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
            // stencil pieces of this column carried up the march: u and the x/y
            // first differences of plane m-1, and u, the differences and the x/y
            // neighbour sums of plane m, so that plane m+1 is the only one whose
            // five-point cross is read from shared memory
            T um_ = 0, dxm_ = 0, dym_ = 0, u0_ = 0, dx0_ = 0, dy0_ = 0, sx0_ = 0, sy0_ = 0;
            T umm_ = 0;   // u of plane m-2, the plane the row warps gather at plane m

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
                    const T u0 = (sizeof(T) == 4 ? umm_ : us[(kz & (NBUF - 1)) * PLANE + uc]) + cin;
                    const T v = fma_(UNI ? -L.tau0 : -in.tau, g, u0);
                    if (interior) *optr = v;
                    su = fma_(wI, u0, su);
                    sout = fma_(wI, v, sout);
                }
                optr += plane_g;
            };

            for (int p = z0 - 2; p <= z0 + PD - 1; ++p) issue(p);

            // One plane m of the march.  GATHER: write plane m-2; PUBLISH: plane
            // m-1 is complete, publish its x/y fields; OWN: plane m is in the
            // run (its energy counts).  All three are compile-time constants, so
            // the steady state (all true) has no phase tests.
            auto plane = [&](int m, auto GATHER, auto PUBLISH, auto OWN, auto FIRST) {
                constexpr bool kGather = decltype(GATHER)::value, kPublish = decltype(PUBLISH)::value;
                (void)kPublish;
                constexpr bool kOwn = decltype(OWN)::value, kFirst = decltype(FIRST)::value;
                // EXT: this plane's coefficients; start the next plane's loads
                Coef<T> Cv;
                if constexpr (EXT) {
                    Cv = in.C;
                    if (cfp) {
                        Cv.c1 = ccn[0]; Cv.c2 = ccn[1]; Cv.c3 = ccn[2];
                        Cv.c4 = ccn[3]; Cv.c5 = ccn[4]; Cv.c6 = ccn[5];
                        Cv.c1x2 = T(2) * ccn[0]; Cv.c2x2 = T(2) * ccn[1]; Cv.c6x2 = T(2) * ccn[5];
                    }
                    load_c(m + 1);
                }
                if (loader) cp_async_wait<PD - 1>();
                bar_cta();
                if constexpr (kGather && MODE != MODE_ENERGY && kRow) gather(m - 2);
                issue(m + 1 + PD);
                if constexpr (MODE == MODE_ENERGY && !kOwn) return;
                const T* p0 = us + (m & (NBUF - 1)) * PLANE + uc;
                const T* pp = us + ((m + 1) & (NBUF - 1)) * PLANE + uc;
                if constexpr (kFirst || sizeof(T) == 8) {   // the run's first evaluated plane: planes m-1 and m from shared memory
                    const T* q = us + ((m - 1) & (NBUF - 1)) * PLANE + uc;
                    um_ = q[0]; dxm_ = q[1] - q[-1]; dym_ = q[UXP] - q[-UXP];
                    u0_ = p0[0]; dx0_ = p0[1] - p0[-1]; dy0_ = p0[UXP] - p0[-UXP];
                    sx0_ = p0[1] + p0[-1]; sy0_ = p0[UXP] + p0[-UXP];
                }
                const T up = pp[0];
                const T dxp = pp[1] - pp[-1], dyp = pp[UXP] - pp[-UXP];
                const T sxp = pp[1] + pp[-1], syp = pp[UXP] + pp[-UXP];
                const T u0 = u0_;
                const T dx = dx0_;
                const T dy = dy0_;
                const T dz = up - um_;
                const T hxx = sx0_ - T(2) * u0;
                const T hyy = sy0_ - T(2) * u0;
                const T hzz = (up + um_) - T(2) * u0;
                const T hxy = (p0[UXP + 1] - p0[UXP - 1]) - (p0[-UXP + 1] - p0[-UXP - 1]);
                const T hxz = dxp - dxm_;
                const T hyz = dyp - dym_;
                umm_ = um_; um_ = u0_; dxm_ = dx0_; dym_ = dy0_;
                u0_ = up; dx0_ = dxp; dy0_ = dyp; sx0_ = sxp; sy0_ = syp;
                Cot<T> ctv;
                const Coef<T>& CC = [&]() -> const Coef<T>& {
                    if constexpr (EXT) return Cv;
                    else if constexpr (UNI) return L.C0;
                    else return in.C;
                }();
                // re-evaluation of D from the exact float inputs (float path only):
                // double-float for eq. Meps, FP64 for the projected form
                auto refine = [&]() -> T {
                    const T* pm = us + ((m - 1) & (NBUF - 1)) * PLANE + uc;
                    // (R and the well are the problem's: a coefficient field changes only
                    // c1 .. c6, and a reference to the per-plane copy Cv would put it in
                    // local memory)
                    if constexpr (EXT == 2) return discriminant_fp64_proj_at<T>(in.C.R, pm, p0, pp, UXP);
                    else if constexpr (EXT == 1) return discriminant_df_at<T>(in.C.R, in.C.well, pm, p0, pp, UXP, cind);
                    else return discriminant_df_at<T>(CC.R, CC.well, pm, p0, pp, UXP, cind);
                };
                if constexpr (MODE == MODE_ENERGY) {
                    const T e = voxel_eval<T, false, EXT != 0, EXT == 2, SYM>(CC, u0 + cin, dx, dy, dz, hxx, hyy, hzz, hxy, hxz, hyz, ctv, refine);
                    if constexpr (kRow) se = fma_(wI, e, se);
                    return;
                } else {
                    const T e = voxel_eval<T, true, EXT != 0, EXT == 2, SYM, SYM>(CC, u0 + cin, dx, dy, dz, hxx, hyy, hzz, hxy, hxz, hyz, ctv, refine);
                    if constexpr (kOwn && kRow) se = fma_(wI, e, se);
                    // transposed-stencil pieces of this voxel (see the gather):
                    //   x/y first+second differences read from the left/right neighbour,
                    //   z pieces from the planes below/above, the centre term stays here
                    //   (SYM: ctv.dx, dy, dz come without the stencil scale sg, which
                    //   the FMAs below apply: 2 % faster there, 1 % slower in the
                    //   general sweep, which keeps the scaled form)
                    T X1, X2, Y1, Y2, zd, zu;
                    if constexpr (SYM) {
                        const T sgv = CC.sg;
                        X1 = fma_(sgv, ctv.dx, ctv.hxx); X2 = fma_(-sgv, ctv.dx, ctv.hxx);
                        Y1 = fma_(sgv, ctv.dy, ctv.hyy); Y2 = fma_(-sgv, ctv.dy, ctv.hyy);
                        zd = fma_(sgv, ctv.dz, ctv.hzz); zu = fma_(-sgv, ctv.dz, ctv.hzz);
                    } else {
                        X1 = ctv.dx + ctv.hxx; X2 = ctv.hxx - ctv.dx;
                        Y1 = ctv.dy + ctv.hyy; Y2 = ctv.hyy - ctv.dy;
                        zd = ctv.dz + ctv.hzz; zu = ctv.hzz - ctv.dz;
                    }
                    const T cpart = ctv.u - T(2) * (ctv.hxx + ctv.hyy + ctv.hzz);
                    if constexpr (kPublish) {   // plane m-1 is complete
                        cpend = accC + zu;
                        const T dxz = hxz2 - ctv.hxz, dyz = hyz2 - ctv.hyz;
                        T* F = fs + ((m - 1) & 1) * 5 * NEXT + fc;
                        if (kRow || active) {
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
            using EF = std::integral_constant<bool, MODE == MODE_ENERGY>;   // energy runs start loading at z0
            plane(z0 - 1, N{}, N{}, N{}, Y{});
            plane(z0, N{}, N{}, Y{}, EF{});
            if (zend - z0 == 1) {
                plane(z0 + 1, N{}, Y{}, N{}, N{});
            } else {
                plane(z0 + 1, N{}, Y{}, Y{}, N{});
                int m = z0 + 2;
                if constexpr (sizeof(T) == 4) {   // two planes per trip: the carried values alternate registers
#pragma unroll 1
                    for (; m + 1 < zend; m += 2) { plane(m, Y{}, Y{}, Y{}, N{}); plane(m + 1, Y{}, Y{}, Y{}, N{}); }
                }
#pragma unroll 1
                for (; m < zend; ++m) plane(m, Y{}, Y{}, Y{}, N{});
                plane(zend, Y{}, Y{}, N{}, N{});
            }
            if (MODE != MODE_ENERGY) {
                bar_cta();
                if constexpr (kRow) gather(zend - 1);
            }
            cp_async_wait<0>();
            bar_cta();   // the ring and the field planes are reused by the next run
        };
        if (warp < TY) body(Y{}); else body(N{});
    }
    if (cur >= 0) flush();
}

size_t fused_smem_bytes(int elem_size, int tile_y);

// One launch of k_fused (sets the dynamic shared-memory limit once per
// instantiation; idempotent, so a race between threads is harmless).
template <typename T, int TY, int MODE, int MAXI, int EXT = 0, bool SYM = false, bool HALO = false, bool UNI = false>
static cudaError_t launch_kernel(const Launch<T, MAXI>& L, int blocks, cudaStream_t s)
{
    const size_t smem = fused_smem_bytes(sizeof(T), TY);
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_fused<T, TY, MODE, MAXI, EXT, SYM, HALO, UNI>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    k_fused<T, TY, MODE, MAXI, EXT, SYM, HALO, UNI><<<blocks, Tile<TY>::NT, smem, s>>>(L);
    return cudaGetLastError();
}

// Batched launches whose problems share L.C0 and L.tau0 (pfc_fused_uni.cu);
// sym: the SYM instantiation.
cudaError_t launch_fused_uni(const Launch<float, BATCH_MAX>& L, int tile_y, int mode, bool sym, cudaStream_t s);

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

// The sweep of a z-slab (in.halo set): every tile height and extension, the
// general instantiation (pfc_fused_slab.cu).
template <typename T>
cudaError_t launch_fused_halo(const Inst<T>& in, int mode, int tile_y, int max_run, cudaStream_t s);

// The FP32 sweep for launches whose problems all have c3 = c5 = 0 (pfc_fused_sym.cu).
template <int MAXI>
cudaError_t launch_fused_sym(const Launch<float, MAXI>& L, int tile_y, int mode, cudaStream_t s);

}  // namespace pfc
