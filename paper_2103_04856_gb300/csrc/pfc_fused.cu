// pfc_fused.cu -- launches of the fused forward + adjoint stencil sweep
// (pfc_fused_kernel.cuh) and the small kernels around it.
#include <atomic>
#include <cstring>

#include "pfc_fused_kernel.cuh"

namespace pfc {

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

// The scalars of a z-slab step from every slab's FP64 sums, combined by one
// thread in rank order (so every slab given the same rows computes the same
// offset c, bit for bit).
__global__ void k_slab_finish(const double* __restrict__ rows, int nslabs, double inv_N, int mode, double* scal,
                              unsigned* ints, double* out5)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s[NPART];
    for (int i = 0; i < NPART; ++i) s[i] = 0.0;
    for (int r = 0; r < nslabs; ++r)
        for (int i = 0; i < NPART; ++i) {
            const double x = rows[(size_t)r * SLAB_NSUMS + i];
            s[i] = i == P_GMAX ? fmax(s[i], x) : s[i] + x;
        }
    set_scalars(s, inv_N, mode, scal, ints, nullptr, 0);
    if (out5) {
        out5[0] = scal[S_E];
        out5[1] = scal[S_MASS];
        out5[2] = scal[S_LAMBDA];
        out5[3] = scal[S_GMAX];
        out5[4] = scal[S_GMEAN];
    }
}

cudaError_t launch_slab_finish(const double* rows, int nslabs, double inv_N, int mode, double* scal, unsigned* ints,
                               double* out5, cudaStream_t s)
{
    k_slab_finish<<<1, 32, 0, s>>>(rows, nslabs, inv_N, mode, scal, ints, out5);
    return cudaGetLastError();
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
                  int proj, int refine)
{
    const double h3 = h * h * h;
    Coef<T> C;
    memset(&C, 0, sizeof C);   // padding too: batched launches compare coefficient sets bytewise
    C.c1 = (T)((a[0] + a[2] - a[1]) / (2.0 * eps) * h3);
    C.c2 = (T)(a[1] / (2.0 * eps) * h3);
    C.c3 = (T)((a[0] - a[2]) / (2.0 * eps) * h3);
    C.c4 = (T)((a[3] + a[4]) / 2.0 * h3);
    C.c5 = (T)((a[3] - a[4]) / 2.0 * h3);
    C.c6 = (T)(a[5] * eps * h3);
    C.c1x2 = T(2) * C.c1;
    C.c2x2 = T(2) * C.c2;
    C.c6x2 = T(2) * C.c6;
    C.kd = (T)(-eps / (h * h));
    C.ko = (T)(-eps / (4.0 * h * h));
    C.ko2 = T(2) * C.ko;
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
    auto split = [](double v, float& hi, float& lo) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    };
    split(C.R.kd, C.R.kd_h, C.R.kd_l);
    split(C.R.ko, C.R.ko_h, C.R.ko_l);
    split(C.R.sg, C.R.sg_h, C.R.sg_l);
    split(C.R.inv_eps, C.R.ie_h, C.R.ie_l);
    split(C.R.xi2, C.R.xi2_h, C.R.xi2_l);
    C.c7 = (T)(eps * mu * h3);
    C.th0 = (T)(theta ? theta[0] : 0.0);
    C.th1 = (T)(theta ? theta[1] : 0.0);
    C.th2 = (T)(theta ? theta[2] : 0.0);
    C.proj = proj ? 1 : 0;
    C.sym = (C.c3 == T(0) && C.c5 == T(0)) ? 1 : 0;
    // the refinement test is scale > rthr max(|D|, xi): 2^16 = 2^22 / 2^6, or never
    C.rthr = refine ? T(65536) : T(INFINITY);
    return C;
}
template Coef<float> make_coef<float>(const double*, double, double, double, int, double, const double*, int, int);
template Coef<double> make_coef<double>(const double*, double, double, double, int, double, const double*, int, int);

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

int device_sms()
{
    static std::atomic<int> cache[64];   // 0: not queried yet
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        dev = -1;
    }
    if (dev >= 0 && dev < 64) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int n = 0;
    if (dev < 0 || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        (void)cudaGetLastError();
        return 1;   // no device to ask: the launch that follows reports the error
    }
    if (dev < 64) cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

long long fused_grid(long long units, int max_run)
{
    long long G = device_sms();                   // one CTA per SM
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

template <typename T, int TY, int EXT = 0>
static cudaError_t launch_mode(const Inst<T>& in, int mode, int max_run, cudaStream_t s)
{
    Launch<T, 1> L;
    L.n = 1;
    L.inst[0] = in;
    plan(L, TY, max_run);
    if constexpr (EXT == 0 && std::is_same<T, float>::value) {
        if (in.C.sym) return launch_fused_sym<1>(L, TY, mode, s);
    }
    switch (mode) {
    case MODE_ENERGY: return launch_kernel<T, TY, MODE_ENERGY, 1, EXT>(L, L.grid, s);
    case MODE_GRAD: return launch_kernel<T, TY, MODE_GRAD, 1, EXT>(L, L.grid, s);
    case MODE_STEP: return launch_kernel<T, TY, MODE_STEP, 1, EXT>(L, L.grid, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_fused(const Inst<T>& in, int mode, int tile_y, int max_run, cudaStream_t s)
{
    if (in.halo) return launch_fused_halo<T>(in, mode, tile_y, max_run, s);
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
// When every problem of a group has the same coefficients and step size, the
// launch's per-voxel arithmetic reads them at fixed constant-bank offsets
// (UNI) instead of loading them from the run's problem descriptor at every
// use (measured: a 256^3 problem 5 % faster).  Splitting a group with two
// coefficient sets into two such launches measured 19 % slower on the four
// 128^3 validation problems (each CTA's runs halve, and a launch gap is
// added), so only single-set groups take it.
// MODE_STEP (descent steps) or MODE_GRAD (energies and gradients).
constexpr int kUniGroups = 1;

cudaError_t launch_fused_batch(const Inst<float>* insts, int n_inst, int tile_y, int max_run, cudaStream_t s,
                               int mode)
{
    if (mode != MODE_STEP && mode != MODE_GRAD) return cudaErrorInvalidValue;
    thread_local Launch<float, BATCH_MAX> L;   // host staging (per thread); the launch copies it
    for (int g0 = 0; g0 < n_inst; g0 += BATCH_MAX) {
        const int cnt = n_inst - g0 < BATCH_MAX ? n_inst - g0 : BATCH_MAX;
        // sets of equal coefficients (bitwise: make_coef clears the padding) and step size
        int set[BATCH_MAX], rep[kUniGroups + 1], nsets = 0;
        bool ext = false;
        for (int k = 0; k < cnt && nsets <= kUniGroups; ++k) {
            const Inst<float>& in = insts[g0 + k];
            ext = ext || needs_ext(in);
            int j = 0;
            while (j < nsets && !(memcmp(&insts[g0 + rep[j]].C, &in.C, sizeof(Coef<float>)) == 0 &&
                                  insts[g0 + rep[j]].tau == in.tau))
                ++j;
            if (j == nsets) rep[nsets++] = k;
            set[k] = j;
        }
        if (!ext && nsets <= kUniGroups) {
            for (int j = 0; j < nsets; ++j) {
                L.n = 0;
                for (int k = 0; k < cnt; ++k)
                    if (set[k] == j) L.inst[L.n++] = insts[g0 + k];
                L.C0 = insts[g0 + rep[j]].C;
                L.tau0 = insts[g0 + rep[j]].tau;
                plan(L, tile_y, max_run);
                cudaError_t e = launch_fused_uni(L, tile_y, mode, L.C0.sym != 0, s);
                if (e != cudaSuccess) return e;
            }
            continue;
        }
        L.n = cnt;
        for (int k = 0; k < cnt; ++k) L.inst[k] = insts[g0 + k];
        plan(L, tile_y, max_run);
        bool sym = true;
        for (int k = 0; k < cnt; ++k) sym = sym && L.inst[k].C.sym && !needs_ext(L.inst[k]);
        cudaError_t e;
        if (sym)
            e = launch_fused_sym<BATCH_MAX>(L, tile_y, mode, s);
        else if (mode == MODE_STEP)
            e = tile_y == 8    ? launch_kernel<float, 8, MODE_STEP, BATCH_MAX>(L, L.grid, s)
                : tile_y == 13 ? launch_kernel<float, 13, MODE_STEP, BATCH_MAX>(L, L.grid, s)
                               : launch_kernel<float, 16, MODE_STEP, BATCH_MAX>(L, L.grid, s);
        else
            e = tile_y == 8    ? launch_kernel<float, 8, MODE_GRAD, BATCH_MAX>(L, L.grid, s)
                : tile_y == 13 ? launch_kernel<float, 13, MODE_GRAD, BATCH_MAX>(L, L.grid, s)
                               : launch_kernel<float, 16, MODE_GRAD, BATCH_MAX>(L, L.grid, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_add_offset(T* out, const T* in, long n, const double* c, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long blocks = (n + 255) / 256;
    if (blocks > 16L * device_sms()) blocks = 16L * device_sms();
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
        int bx = (8 * device_sms() + cnt - 1) / cnt;
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
    if (blocks > 16L * device_sms()) blocks = 16L * device_sms();
    k_curvatures<T><<<(int)blocks, 256, 0, s>>>(u, k1, k2, nx, ny, nz, C, (T)eps);
    return cudaGetLastError();
}
template cudaError_t launch_curvatures<float>(const float*, float*, float*, int, int, int, const Coef<float>&,
                                              double, cudaStream_t);
template cudaError_t launch_curvatures<double>(const double*, double*, double*, int, int, int,
                                               const Coef<double>&, double, cudaStream_t);

}  // namespace pfc
