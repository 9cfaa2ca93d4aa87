// pfc_device.cuh -- per-voxel arithmetic of the phase-field energy (Song,
// arXiv 2103.04856, Sec. 3.2 eq. Feps) and its local reverse mode, plus the
// block / grid reductions shared by the fused and the plain kernels.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pfc_internal.h"

namespace pfc {

// ------------------------------------------------------------ type helpers

__device__ __forceinline__ float  rcp_(float x)  { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ float  rsqrt_(float x)  { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float  sqrt_(float x)  { return sqrtf(x); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float  fma_(float a, float b, float c)    { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
// max that returns NaN when either operand is NaN (fmaxf drops a NaN operand)
__device__ __forceinline__ float fmax_nan_(float a, float b) {
    float r;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ double fmax_nan_(double a, double b) { return (a != a || b != b) ? a + b : fmax(a, b); }

// Smooth positive part P(D) = xi log(1 + exp(D/xi)) of Sec. 4.1 and its
// derivative P'(D) = logistic(D/xi).
// float: outside |D| < 64 xi the correction term is below xi*1.6e-28 and is
// dropped (P = D^+ exactly; the neglected sqrt(P) on the negative side is
// below sqrt(xi)*1.3e-14); inside, the overflow-free form is used.
__device__ __forceinline__ void softplus_(float D, const Coef<float>& C, float& P, float& Pp)
{
    float ad = fabsf(D);
    if (ad > 64.0f * C.xi) {
        P = D > 0.0f ? D : 0.0f;
        Pp = D > 0.0f ? 1.0f : 0.0f;
    } else {
        float ex = __expf(-ad * C.inv_xi);
        float inv = __fdividef(1.0f, 1.0f + ex);
        P = fmaxf(D, 0.0f) + C.xi * log1pf(ex);
        Pp = D >= 0.0f ? inv : ex * inv;
    }
}
__device__ __forceinline__ void softplus_(double D, const Coef<double>& C, double& P, double& Pp)
{
    double ex = exp(-fabs(D) * C.inv_xi);
    double inv = 1.0 / (1.0 + ex);
    P = fmax(D, 0.0) + C.xi * log1p(ex);
    Pp = D >= 0.0 ? inv : ex * inv;
}

// Cotangents of one voxel's density with respect to its ten stencil values.
template <typename T>
struct Cot {
    T u;                    // through W'(u)
    T dx, dy, dz;           // first differences u(+) - u(-)
    T hxx, hyy, hzz;        // second differences u(+) - 2u + u(-)
    T hxy, hxz, hyz;        // 4-point mixed differences
};

// ------------------------------------------------------------ double-float

// An unevaluated sum hi + lo of two floats (|lo| <= ulp(hi) / 2): about 44
// significant bits from FP32 operations, far cheaper on this GPU than FP64
// (whose pipe runs at 1/64 of the FP32 rate).  The error-free transformations
// are Knuth's two-sum and the product error from one FMA; the _rn intrinsics
// keep the compiler from contracting or reordering them.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return { s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)) };
}
__device__ __forceinline__ DF df_fast_two_sum(float a, float b)   // |a| >= |b| or a == 0
{
    const float s = __fadd_rn(a, b);
    return { s, __fsub_rn(b, __fsub_rn(s, a)) };
}
__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const DF s = df_two_sum(a.hi, b.hi), t = df_two_sum(a.lo, b.lo);
    const DF r = df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return df_fast_two_sum(r.hi, __fadd_rn(t.lo, r.lo));
}
__device__ __forceinline__ DF df_neg(DF a) { return { -a.hi, -a.lo }; }
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ DF df_mul(DF a, DF b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.hi, -p)));
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ DF df_scale2(DF a) { return { __fmul_rn(2.0f, a.hi), __fmul_rn(2.0f, a.lo) }; }   // exact
__device__ __forceinline__ DF df_div(DF a, DF b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const DF r = df_sub(a, df_mul(DF{ q1, 0.0f }, b));
    return df_fast_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}

// D of eq. Meps's M in double-float from the 19 raw stencil values of the
// voxel (exact floats in three u planes: pm, p0, pp point at the voxel,
// `pitch` is the row pitch) plus the offset c the loads add: differences
// of the inputs are exact (two-sum), every later operation keeps about 44
// bits, so the cancellation in 2S - T^2 no longer loses the result.  Kept out
// of line: it runs for few voxels and must not add registers to the float
// hot path.
template <typename T>
__device__ __noinline__ T discriminant_df_at(const CoefD& R, int well, const T* pm, const T* p0, const T* pp, int pitch,
                                             double c)
{
    const float ch = (float)c;
    const DF cdf = { ch, (float)(c - (double)ch) };
    const float uc = (float)p0[0];
    const DF u0 = df_add(DF{ uc, 0.0f }, cdf);
    auto f = [](T v) { return (float)v; };
    auto diff = [&](const T* p, int o) { return df_two_sum(f(p[o]), -f(p[-o])); };                  // u(+) - u(-)
    auto lap = [&](const T* p, int o) { return df_sub(df_two_sum(f(p[o]), f(p[-o])), DF{ 2.0f * uc, 0.0f }); };
    const DF kd = { R.kd_h, R.kd_l }, ko = { R.ko_h, R.ko_l }, sg = { R.sg_h, R.sg_l };
    const DF Gx = df_mul(diff(p0, 1), sg), Gy = df_mul(diff(p0, pitch), sg);
    const DF Gz = df_mul(df_two_sum(f(pp[0]), -f(pm[0])), sg);
    const DF hxx = lap(p0, 1), hyy = lap(p0, pitch);
    const DF hzz = df_sub(df_two_sum(f(pp[0]), f(pm[0])), DF{ 2.0f * uc, 0.0f });
    const DF hxy = df_sub(df_two_sum(f(p0[pitch + 1]), -f(p0[pitch - 1])), df_two_sum(f(p0[-pitch + 1]), -f(p0[-pitch - 1])));
    const DF hxz = df_sub(df_two_sum(f(pp[1]), -f(pp[-1])), df_two_sum(f(pm[1]), -f(pm[-1])));
    const DF hyz = df_sub(df_two_sum(f(pp[pitch]), -f(pp[-pitch])), df_two_sum(f(pm[pitch]), -f(pm[-pitch])));
    const DF rho = df_add(df_add(df_mul(Gx, Gx), df_mul(Gy, Gy)), df_add(df_mul(Gz, Gz), DF{ R.xi2_h, R.xi2_l }));
    DF w;   // W'(u) / eps
    const DF one = { 1.0f, 0.0f };
    if (well == 0) {
        const DF t = df_sub(u0, df_mul(u0, u0));                       // u (1 - u)
        w = df_mul(df_scale2(t), df_sub(one, df_scale2(u0)));
    } else {
        w = df_sub(df_mul(df_mul(u0, u0), u0), u0);
    }
    const DF wr = df_div(df_mul(w, DF{ R.ie_h, R.ie_l }), rho);        // (W'/eps) / rho
    const DF wx = df_mul(wr, Gx), wy = df_mul(wr, Gy), wz = df_mul(wr, Gz);
    const DF Mxx = df_add(df_mul(kd, hxx), df_mul(wx, Gx)), Myy = df_add(df_mul(kd, hyy), df_mul(wy, Gy));
    const DF Mzz = df_add(df_mul(kd, hzz), df_mul(wz, Gz));
    const DF Mxy = df_add(df_mul(ko, hxy), df_mul(wx, Gy)), Mxz = df_add(df_mul(ko, hxz), df_mul(wx, Gz));
    const DF Myz = df_add(df_mul(ko, hyz), df_mul(wy, Gz));
    const DF Tr = df_add(df_add(Mxx, Myy), Mzz);
    const DF dg = df_add(df_add(df_mul(Mxx, Mxx), df_mul(Myy, Myy)), df_mul(Mzz, Mzz));
    const DF od = df_add(df_add(df_mul(Mxy, Mxy), df_mul(Mxz, Mxz)), df_mul(Myz, Myz));
    const DF S = df_add(dg, df_scale2(od));
    const DF D = df_sub(df_scale2(S), df_mul(Tr, Tr));
    return (T)__fadd_rn(D.hi, D.lo);
}

// rho^4 D of the tangent-projected M, in FP64 from the exact raw stencil
// values: rho^2 M = rho^2 K - rho (G k^T + k G^T) + s G G^T needs no division.
template <typename T>
__device__ __noinline__ T discriminant_fp64_proj_at(const CoefD& R, const T* pm, const T* p0, const T* pp, int pitch)
{
    auto d = [](T v) { return (double)v; };
    const double u0 = d(p0[0]);
    const double Gx = (d(p0[1]) - d(p0[-1])) * R.sg, Gy = (d(p0[pitch]) - d(p0[-pitch])) * R.sg;
    const double Gz = (d(pp[0]) - d(pm[0])) * R.sg;
    const double Kxx = R.kd * ((d(p0[1]) + d(p0[-1])) - 2.0 * u0);
    const double Kyy = R.kd * ((d(p0[pitch]) + d(p0[-pitch])) - 2.0 * u0);
    const double Kzz = R.kd * ((d(pp[0]) + d(pm[0])) - 2.0 * u0);
    const double Kxy = R.ko * ((d(p0[pitch + 1]) - d(p0[pitch - 1])) - (d(p0[-pitch + 1]) - d(p0[-pitch - 1])));
    const double Kxz = R.ko * ((d(pp[1]) - d(pp[-1])) - (d(pm[1]) - d(pm[-1])));
    const double Kyz = R.ko * ((d(pp[pitch]) - d(pp[-pitch])) - (d(pm[pitch]) - d(pm[-pitch])));
    const double rho = fma(Gx, Gx, fma(Gy, Gy, fma(Gz, Gz, R.xi2)));
    const double kx = Kxx * Gx + Kxy * Gy + Kxz * Gz, ky = Kxy * Gx + Kyy * Gy + Kyz * Gz;
    const double kz = Kxz * Gx + Kyz * Gy + Kzz * Gz;
    const double s = Gx * kx + Gy * ky + Gz * kz;
    const double r2 = rho * rho;
    const double Mxx = r2 * Kxx - 2.0 * rho * Gx * kx + s * Gx * Gx;
    const double Myy = r2 * Kyy - 2.0 * rho * Gy * ky + s * Gy * Gy;
    const double Mzz = r2 * Kzz - 2.0 * rho * Gz * kz + s * Gz * Gz;
    const double Mxy = r2 * Kxy - rho * (Gx * ky + kx * Gy) + s * Gx * Gy;
    const double Mxz = r2 * Kxz - rho * (Gx * kz + kx * Gz) + s * Gx * Gz;
    const double Myz = r2 * Kyz - rho * (Gy * kz + ky * Gz) + s * Gy * Gz;
    const double Tr = Mxx + Myy + Mzz;
    const double S = Mxx * Mxx + Myy * Myy + Mzz * Mzz + 2.0 * (Mxy * Mxy + Mxz * Mxz + Myz * Myz);
    // the cancellation is resolved; divide in FP64 (rho^4 can be below float's range)
    return (T)((2.0 * S - Tr * Tr) / (r2 * r2));
}

// No refinement available (the plain path evaluates voxels from stored
// derivatives): D keeps its FP32 value.
struct NoRefine {
    __device__ __forceinline__ float operator()() const { return 0.0f; }
};
template <class R>
struct refines {
    static constexpr bool value = true;
};
template <>
struct refines<NoRefine> {
    static constexpr bool value = false;
};

// Forward (eq. Meps, Sec. 3.1 invariants, eq. Feps) and, if GRAD, local
// reverse mode of one voxel.  Inputs are the raw stencil values:
//   dx = u(x+1) - u(x-1), hxx = u(x+1) - 2u + u(x-1),
//   hxy = u(x+1,y+1) - u(x+1,y-1) - u(x-1,y+1) + u(x-1,y-1), etc.
//
// float only: D is the difference of two O(||M||^2) numbers, so its FP32
// error is about 2^-22 (2S + T^2).  Only the sqrt(D+) terms, of weight
// a3 = c3 T + c5 q (zero for polynomials symmetric in kappa1, kappa2), see
// that error, and it matters only where it is more than 2^-6 of max(|D|, xi):
// there `refine()` recomputes D from the exact float inputs in double-float
// (eq. Meps) or FP64 (the projected form) arithmetic (about one voxel in 10^4
// on noise fields, many more on fields that are blowing up; the kernel's CTAs
// wait for the slowest warp at every plane, so the test is kept tight).
//
// ORIENT adds the orientation term of Sec. 5.2, c7 (theta . G)^2, and its
// cotangent 2 c7 (theta . G) theta on G.
//
// PROJ replaces eq. Meps by the tangent-projected M = P K P, K = -eps Hess u,
// P = I - G G^T / rho (no double-well term): with k = K G and
// s = G.k, M = K - (G m^T + m G^T)/rho, m = k - (s / 2rho) G.
//
// SKIPD (p symmetric in kappa1, kappa2: c3 = c5 = 0 for every voxel the
// caller evaluates): a3 = c3 T + c5 q is exactly 0 and r enters only through
// a3 r, c3 r and c5 r, which stay exact zeros with r = r' = 0; D, P and
// sqrt(P) are then not computed, with the same result bits.
//
// RAWD: ct.dx, ct.dy, ct.dz are returned without the stencil scale sg =
// 1/(2h) (the caller folds it into the FMAs that combine them with the
// second-difference cotangents).
template <typename T, bool GRAD, bool ORIENT = false, bool PROJ = false, bool SKIPD = false, bool RAWD = false,
          class Refine = NoRefine>
__device__ __forceinline__ T voxel_eval(const Coef<T>& C, T u0, T dx, T dy, T dz, T hxx, T hyy,
                                        T hzz, T hxy, T hxz, T hyz, Cot<T>& ct, const Refine& refine = Refine())
{
    static_assert(!(SKIPD && (ORIENT || PROJ)), "the symmetric shortcut is for the plain energy only");
    const T Gx = dx * C.sg, Gy = dy * C.sg, Gz = dz * C.sg;
    const T g2 = fma_(Gx, Gx, fma_(Gy, Gy, Gz * Gz));
    const T rho = g2 + C.xi2;
    const T iq = rsqrt_(rho);
    const T q = rho * iq;
    const T irho = sizeof(T) == 4 ? iq * iq : rcp_(rho);
    T wpp = T(0), wr = T(0);
    T Mxx, Myy, Mzz, Mxy, Mxz, Myz;
    // PROJ only: K = -eps Hess u and k = K G
    T Kxx = T(0), Kyy = T(0), Kzz = T(0), Kxy = T(0), Kxz = T(0), Kyz = T(0);
    T kx = T(0), ky = T(0), kz = T(0), sk = T(0);
    if (PROJ) {
        Kxx = C.kd * hxx; Kyy = C.kd * hyy; Kzz = C.kd * hzz;
        Kxy = C.ko * hxy; Kxz = C.ko * hxz; Kyz = C.ko * hyz;
        kx = fma_(Kxx, Gx, fma_(Kxy, Gy, Kxz * Gz));
        ky = fma_(Kxy, Gx, fma_(Kyy, Gy, Kyz * Gz));
        kz = fma_(Kxz, Gx, fma_(Kyz, Gy, Kzz * Gz));
        sk = fma_(Gx, kx, fma_(Gy, ky, Gz * kz));
        const T hs = T(0.5) * sk * irho;
        const T mx = fma_(-hs, Gx, kx), my = fma_(-hs, Gy, ky), mz = fma_(-hs, Gz, kz);
        Mxx = fma_(-T(2) * irho * Gx, mx, Kxx);
        Myy = fma_(-T(2) * irho * Gy, my, Kyy);
        Mzz = fma_(-T(2) * irho * Gz, mz, Kzz);
        Mxy = Kxy - irho * fma_(Gx, my, mx * Gy);
        Mxz = Kxz - irho * fma_(Gx, mz, mx * Gz);
        Myz = Kyz - irho * fma_(Gy, mz, my * Gz);
    } else {
        // W'(u)/eps and W''(u)/eps for the chosen double well
        T wp;
        if (C.well == 0) {
            const T t = u0 - u0 * u0;                       // u (1 - u)
            wp = T(2) * t * (T(1) - T(2) * u0);
            wpp = T(2) - T(12) * t;                         // 2 (1 - 6u + 6u^2)
        } else {
            wp = u0 * u0 * u0 - u0;
            wpp = T(3) * u0 * u0 - T(1);
        }
        wr = wp * C.inv_eps * irho;                         // (W'/eps) / rho
        // M = -eps Hess u + (W'/eps) G G^T / rho
        const T wx = wr * Gx, wy = wr * Gy, wz = wr * Gz;
        Mxx = fma_(C.kd, hxx, wx * Gx);
        Myy = fma_(C.kd, hyy, wy * Gy);
        Mzz = fma_(C.kd, hzz, wz * Gz);
        Mxy = fma_(C.ko, hxy, wx * Gy);
        Mxz = fma_(C.ko, hxz, wx * Gz);
        Myz = fma_(C.ko, hyz, wy * Gz);
    }
    const T Tr = Mxx + Myy + Mzz;
    const T off = fma_(Mxy, Mxy, fma_(Mxz, Mxz, Myz * Myz));
    const T S = fma_(Mxx, Mxx, fma_(Myy, Myy, fma_(Mzz, Mzz, T(2) * off)));
    const T t2 = Tr * Tr;
    T a3 = T(0);                                        // c3 T + c5 q
    T r = T(0), rs = T(0), Pp = T(0);
    if constexpr (!SKIPD) {
        a3 = fma_(C.c3, Tr, C.c5 * q);
        // D = 2S - T^2 with the rounding error of T^2 put back (two-product)
        const T t2e = fma_(Tr, Tr, -t2);
        T D = fma_(T(2), S, -t2) - t2e;
        if (sizeof(T) == 4 && refines<Refine>::value) {
            const T scale = fma_(T(2), S, t2);
            // a non-finite D comes from invariants that overflowed FP32, which the
            // refinement cannot recover: the NaN-propagating max keeps it out
            if (a3 != T(0) && scale > C.rthr * fmax_nan_(fabs(D), C.xi)) D = (T)refine();
        }
        T P;
        softplus_(D, C, P, Pp);
        // float: one reciprocal square root gives both sqrt(P) and 1/(2 sqrt(P))
        rs = (sizeof(T) == 4 && P > T(0)) ? rsqrt_(P) : T(0);
        r = sizeof(T) == 4 ? P * rs : sqrt_(P);
    }
    // SKIPD: the a3 r term is an exact zero (written out: the compiler may not drop a3 * 0)
    T e = SKIPD ? fma_(C.c1, S, fma_(C.c2, t2, fma_(C.c4 * q, Tr, C.c6 * g2)))
                : fma_(C.c1, S, fma_(C.c2, t2, fma_(a3, r, fma_(C.c4 * q, Tr, C.c6 * g2))));
    T tg = T(0);
    if (ORIENT) {
        tg = fma_(C.th0, Gx, fma_(C.th1, Gy, C.th2 * Gz));
        e = fma_(C.c7 * tg, tg, e);
    }
    if (!GRAD) return e;

    // local reverse mode: e(S, T, r(D(S,T)), q(G), |G|^2), M(Hess, w(u), G)
    // dr/dD, 0 where r = 0
    T dT, dq, s2;   // de/dT, de/dq, 2 de/dS
    if constexpr (SKIPD) {
        // r = r' = 0: the same values as below with k = 0 and r = 0
        dT = fma_(C.c2x2, Tr, C.c4 * q);
        dq = C.c4 * Tr;
        s2 = C.c1x2;
    } else {
        const T rp = sizeof(T) == 4 ? T(0.5) * Pp * rs : (r > T(0) ? T(0.5) * Pp / r : T(0));
        const T k = a3 * rp;                                 // de/dD
        const T dS = fma_(T(2), k, C.c1);
        dT = fma_(C.c2x2, Tr, fma_(C.c3, r, fma_(C.c4, q, -T(2) * Tr * k)));
        dq = fma_(C.c4, Tr, C.c5 * r);
        s2 = T(2) * dS;
    }
    // Lambda = de/dM = 2 dS M + dT I
    const T Lxx = fma_(s2, Mxx, dT), Lyy = fma_(s2, Myy, dT), Lzz = fma_(s2, Mzz, dT);
    const T Lxy = s2 * Mxy, Lxz = s2 * Mxz, Lyz = s2 * Myz;
    const T LGx = fma_(Lxx, Gx, fma_(Lxy, Gy, Lxz * Gz));
    const T LGy = fma_(Lxy, Gx, fma_(Lyy, Gy, Lyz * Gz));
    const T LGz = fma_(Lxz, Gx, fma_(Lyz, Gy, Lzz * Gz));
    const T GLG = fma_(Gx, LGx, fma_(Gy, LGy, Gz * LGz));
    if (PROJ) {
        // dE/dK = P L P = L - (G n^T + n G^T)/rho, n = LG - (G.LG / 2rho) G;
        // dE/dG through P: -2 B G / rho + 2 (G^T B G) G / rho^2 with
        // B G = L P k + K P (LG) and G^T B G = 2 (LG.k - s G.LG / rho)
        const T hl = T(0.5) * GLG * irho;
        const T nx = fma_(-hl, Gx, LGx), ny = fma_(-hl, Gy, LGy), nz = fma_(-hl, Gz, LGz);
        const T Pxx = fma_(-T(2) * irho * Gx, nx, Lxx);
        const T Pyy = fma_(-T(2) * irho * Gy, ny, Lyy);
        const T Pzz = fma_(-T(2) * irho * Gz, nz, Lzz);
        const T Pxy = Lxy - irho * fma_(Gx, ny, nx * Gy);
        const T Pxz = Lxz - irho * fma_(Gx, nz, nx * Gz);
        const T Pyz = Lyz - irho * fma_(Gy, nz, ny * Gz);
        const T si = sk * irho, gi = GLG * irho;
        const T pkx = fma_(-si, Gx, kx), pky = fma_(-si, Gy, ky), pkz = fma_(-si, Gz, kz);      // P k
        const T plx = fma_(-gi, Gx, LGx), ply = fma_(-gi, Gy, LGy), plz = fma_(-gi, Gz, LGz);  // P LG
        const T BGx = fma_(Lxx, pkx, fma_(Lxy, pky, Lxz * pkz)) + fma_(Kxx, plx, fma_(Kxy, ply, Kxz * plz));
        const T BGy = fma_(Lxy, pkx, fma_(Lyy, pky, Lyz * pkz)) + fma_(Kxy, plx, fma_(Kyy, ply, Kyz * plz));
        const T BGz = fma_(Lxz, pkx, fma_(Lyz, pky, Lzz * pkz)) + fma_(Kxz, plx, fma_(Kyz, ply, Kzz * plz));
        const T GBG = T(2) * fma_(LGx, kx, fma_(LGy, ky, fma_(LGz, kz, -si * GLG)));
        const T al = -T(2) * irho;
        const T be = fma_(T(2) * GBG * irho, irho, fma_(dq, iq, C.c6x2));
        ct.u = T(0);
        ct.dx = RAWD ? fma_(al, BGx, be * Gx) : C.sg * fma_(al, BGx, be * Gx);
        ct.dy = RAWD ? fma_(al, BGy, be * Gy) : C.sg * fma_(al, BGy, be * Gy);
        ct.dz = RAWD ? fma_(al, BGz, be * Gz) : C.sg * fma_(al, BGz, be * Gz);
        if (ORIENT) {
            const T ot = RAWD ? T(2) * C.c7 * tg : T(2) * C.c7 * tg * C.sg;
            ct.dx = fma_(ot, C.th0, ct.dx);
            ct.dy = fma_(ot, C.th1, ct.dy);
            ct.dz = fma_(ot, C.th2, ct.dz);
        }
        ct.hxx = C.kd * Pxx;
        ct.hyy = C.kd * Pyy;
        ct.hzz = C.kd * Pzz;
        ct.hxy = C.ko2 * Pxy;
        ct.hxz = C.ko2 * Pxz;
        ct.hyz = C.ko2 * Pyz;
        return e;
    }
    ct.u = wpp * C.inv_eps * GLG * irho;
    const T al = T(2) * wr;
    const T be = fma_(-al * GLG, irho, fma_(dq, iq, C.c6x2));
    ct.dx = RAWD ? fma_(al, LGx, be * Gx) : C.sg * fma_(al, LGx, be * Gx);
    ct.dy = RAWD ? fma_(al, LGy, be * Gy) : C.sg * fma_(al, LGy, be * Gy);
    ct.dz = RAWD ? fma_(al, LGz, be * Gz) : C.sg * fma_(al, LGz, be * Gz);
    if (ORIENT) {
        const T ot = RAWD ? T(2) * C.c7 * tg : T(2) * C.c7 * tg * C.sg;
        ct.dx = fma_(ot, C.th0, ct.dx);
        ct.dy = fma_(ot, C.th1, ct.dy);
        ct.dz = fma_(ot, C.th2, ct.dz);
    }
    ct.hxx = C.kd * Lxx;
    ct.hyy = C.kd * Lyy;
    ct.hzz = C.kd * Lzz;
    ct.hxy = C.ko2 * Lxy;                                     // Hess_cd feeds M_cd and M_dc
    ct.hxz = C.ko2 * Lxz;
    ct.hyz = C.ko2 * Lyz;
    return e;
}

// ------------------------------------------------------------ grid walks

// Neighbour index along one axis: i + d wrapped into [0, n) (periodic),
// without a division when |d| < n.
__device__ __forceinline__ int nbr(int i, int d, int n)
{
    int j = i + d;
    if (j < 0) j += n;
    if (j >= n) j -= n;
    if (j >= 0 && j < n) return j;
    const int r = (i + d) % n;
    return r < 0 ? r + n : r;
}

// A thread's position in a grid-stride loop over the flattened voxel index
// i = (z ny + y) nx + x: the coordinates advance by the stride's own (sx, sy,
// sz) with two carries instead of two divisions per voxel.
struct Walk {
    int x, y, z;            // coordinates of voxel i
    int sx, sy, sz;         // the grid stride as (x, y, z) steps
    long i, stride;
    __device__ Walk(int nx, int ny, long i0, long s) : i(i0), stride(s)
    {
        const long pls = (long)nx * ny;
        z = (int)(i0 / pls); y = (int)((i0 - (long)z * pls) / nx); x = (int)(i0 - (long)z * pls - (long)y * nx);
        sz = (int)(s / pls); sy = (int)((s - (long)sz * pls) / nx); sx = (int)(s - (long)sz * pls - (long)sy * nx);
    }
    __device__ void next(int nx, int ny)
    {
        i += stride;
        x += sx;
        int c = x >= nx;
        x -= c ? nx : 0;
        y += sy + c;
        c = y >= ny;
        y -= c ? ny : 0;
        z += sz + c;
    }
};

// ------------------------------------------------------------ accumulators

// Kahan-compensated running sum in the arithmetic type (per thread, <= a
// few hundred terms), handed to FP64 for everything beyond one thread.
template <typename T>
struct KSum {
    T s = T(0), c = T(0);
    __device__ __forceinline__ void add(T v)
    {
        T y = v - c;
        T t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide reduction of NPART values (sum, except P_GMAX: max); result in
// red[0..NPART) of shared scratch `red` (>= 32*NPART doubles) for thread 0.
// Fixed tree: deterministic for a fixed block size.
__device__ __forceinline__ void block_reduce_parts(double v[NPART], double* red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NPART; ++i) v[i] = (i == P_GMAX) ? warp_max(v[i]) : warp_sum(v[i]);
    __syncthreads();  // red may still be read by a previous use
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NPART; ++i) red[wid * NPART + i] = v[i];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int i = 0; i < NPART; ++i) {
            double x = lane < nw ? red[lane * NPART + i] : 0.0;
            v[i] = (i == P_GMAX) ? warp_max(x) : warp_sum(x);
        }
    }
}

// The problem's scalars from its FP64 totals s[NPART] (sums over every voxel,
// except s[P_GMAX], a max): energy, mean of the gradient (the multiplier),
// max and mean |g|; after a step also the mass, the target mass (set by the
// first step of a run), the offset c = target - mean(v) that the next step's
// loads add, and a trace row.  `retire` (batch steps): an instance already
// flagged non-finite was not evaluated; it only records a NaN trace row.
// One thread.
__device__ __forceinline__ void set_scalars(const double s[NPART], double inv_N, int mode, double* sc, unsigned* ints,
                                            double* trace, int trace_cap, bool retire = false)
{
    if (retire && mode == MODE_STEP && ints[I_NONFINITE]) {
        const unsigned cnt = ints[I_COUNTER];
        if (trace && (int)cnt < trace_cap)
            for (int i = 0; i < 5; ++i) trace[(size_t)cnt * 5 + i] = NAN;
        ints[I_COUNTER] = cnt + 1;
        return;
    }
    const double E = s[P_E];
    bool bad = !isfinite(E);
    if (mode == MODE_ENERGY) {
        sc[S_E] = E;
    } else {
        const double lam = s[P_G] * inv_N;
        sc[S_E] = E;
        sc[S_LAMBDA] = lam;
        sc[S_GMAX] = s[P_GMAX];
        sc[S_GMEAN] = s[P_AG] * inv_N;
        bad = bad || !isfinite(lam);
        if (mode == MODE_STEP) {
            const double mass = s[P_U] * inv_N;
            const unsigned cnt = ints[I_COUNTER];
            if (cnt == 0) sc[S_TARGET] = mass;   // conserve the mass of the first field
            sc[S_MASS] = mass;
            sc[S_C] = sc[S_TARGET] - s[P_OUT] * inv_N;
            bad = bad || !isfinite(mass) || !isfinite(sc[S_C]);
            if (trace && (int)cnt < trace_cap) {
                double* row = trace + (size_t)cnt * 5;
                row[0] = E; row[1] = mass; row[2] = lam; row[3] = s[P_GMAX]; row[4] = sc[S_GMEAN];
            }
            ints[I_COUNTER] = cnt + 1;
        }
    }
    if (bad) ints[I_NONFINITE] = 1;
}

// Publish one CTA's totals `tot` (shared, NPART doubles) as partial `slot`
// of a problem; the last CTA to arrive (atomic ticket, no waiting) combines
// all partials of the problem in a fixed order and writes its scalars (or,
// for a z-slab, its totals to in.sums_out).
template <typename T>
__device__ void finish_problem(const Inst<T>& in, int slot, int mode, const double* tot, bool retire = false)
{
    __shared__ int am_last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NPART; ++i) in.partials[(size_t)slot * NPART + i] = tot[i];
        __threadfence();
        const unsigned t = atomicAdd(&in.ints[I_TICKET], 1u);
        am_last = (t == (unsigned)in.nblocks - 1u);
    }
    __syncthreads();
    if (!am_last || threadIdx.x >= 32) return;
    __threadfence();
    const int lane = threadIdx.x;
    double s[NPART];
#pragma unroll
    for (int i = 0; i < NPART; ++i) s[i] = 0.0;
    for (int b = lane; b < in.nblocks; b += 32) {
#pragma unroll
        for (int i = 0; i < NPART; ++i) {
            const double x = __ldcg(&in.partials[(size_t)b * NPART + i]);
            s[i] = (i == P_GMAX) ? fmax(s[i], x) : s[i] + x;
        }
    }
#pragma unroll
    for (int i = 0; i < NPART; ++i) s[i] = (i == P_GMAX) ? warp_max(s[i]) : warp_sum(s[i]);
    if (lane != 0) return;
    if (in.sums_out) {
#pragma unroll
        for (int i = 0; i < NPART; ++i) in.sums_out[i] = s[i];
    } else {
        set_scalars(s, in.inv_N, mode, in.scal, in.ints, in.trace, in.trace_cap, retire);
    }
    __threadfence();
    in.ints[I_TICKET] = 0;   // ready for the next launch on this problem
}

// Grid-stride kernels (plain path): reduce each thread's FP64 values over the
// block, then publish them as partial blockIdx.x.
template <typename T>
__device__ void grid_finish(const Inst<T>& in, int slot, int mode, double v[NPART], double* red)
{
    __shared__ double tot[NPART];
    block_reduce_parts(v, red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int i = 0; i < NPART; ++i) tot[i] = v[i];
    __syncthreads();
    finish_problem(in, slot, mode, tot);
}

// Block totals of per-thread FP32 sums for the fused sweep: every thread
// stores its NPART values, then warp i adds column i (compensated, 20 terms
// per lane) and finishes in FP64 across lanes.  Few FP64 operations: the
// FP64 pipe is slow on this GPU.  `scr` holds NPART * NT floats.
template <int NT>
__device__ __forceinline__ void block_sums(const float v[NPART], float* scr, double* tot)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NPART; ++i) scr[i * NT + tid] = v[i];
    __syncthreads();
    if (warp < NPART) {
        const float* col = scr + warp * NT;
        double r;
        if (warp == P_GMAX) {
            float m = 0.0f;
            for (int j = lane; j < NT; j += 32) m = fmaxf(m, col[j]);
            r = warp_max((double)m);
        } else {
            KSum<float> k;
            for (int j = lane; j < NT; j += 32) k.add(col[j]);
            r = warp_sum(k.get());
        }
        if (lane == 0) tot[warp] = r;
    }
    __syncthreads();
}

// FP64 sweep: per-thread FP64 sums, plain FP64 block reduction.
template <int NT>
__device__ __forceinline__ void block_sums(const double v[NPART], float*, double* tot)
{
    __shared__ double red[32 * NPART];
    double w[NPART];
#pragma unroll
    for (int i = 0; i < NPART; ++i) w[i] = v[i];
    block_reduce_parts(w, red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int i = 0; i < NPART; ++i) tot[i] = w[i];
    __syncthreads();
}

}  // namespace pfc
