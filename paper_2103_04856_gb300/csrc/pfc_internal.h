// pfc_internal.h -- types shared by the kernels and the C ABI of the
// phase-field curvature-energy library (not part of the public interface).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pfc {

enum Mode { MODE_ENERGY = 0, MODE_GRAD = 1, MODE_STEP = 2 };

// Per-block FP64 partial sums written by every CTA and combined by the last.
enum Part { P_E = 0, P_U, P_G, P_AG, P_GMAX, P_OUT, NPART };

// Device scalar slots of one problem.
//  S_E      energy of the evaluated field
//  S_MASS   mean of the evaluated field
//  S_LAMBDA mean of the gradient (Lagrange multiplier of the mass constraint)
//  S_GMAX   max |g|;  S_GMEAN mean |g|
//  S_C      offset added to the stored field on load (lazy mass projection)
//  S_TARGET mass to keep, set from the first evaluated field of a run
enum Scal { S_E = 0, S_MASS, S_LAMBDA, S_GMAX, S_GMEAN, S_C, S_TARGET, NSCAL = 8 };
enum Ints { I_TICKET = 0, I_COUNTER, I_NONFINITE, NINTS = 4 };

// The same scale factors in FP64, and as float pairs hi + lo (about 44
// significant bits), for re-evaluating the discriminant D = 2||M||^2 -
// (Tr M)^2 of a float voxel where FP32 cancellation would matter (see
// voxel_eval): eq. Meps in double-float arithmetic, the projected form in FP64.
struct CoefD {
    double kd, ko, sg, inv_eps, xi2;
    float kd_h, kd_l, ko_h, ko_l, sg_h, sg_l, ie_h, ie_l, xi2_h, xi2_l;
};

// Coefficients of eq. Feps (times h^3, so that summing the per-voxel density
// gives E directly) and the stencil scale factors, in the arithmetic type.
template <typename T>
struct Coef {
    T c1, c2, c3, c4, c5, c6;
    T c1x2, c2x2, c6x2;   // 2 c1, 2 c2, 2 c6 (exact doublings, formed once on the host)
    T kd;       // -eps / h^2     : d M_cc / d (u+ - 2u + u-)
    T ko;       // -eps / (4 h^2) : d M_cd / d (4-point mixed difference)
    T ko2;      // 2 ko: Hess_cd feeds both M_cd and M_dc
    T sg;       // 1 / (2h)       : d G_c / d (u+ - u-)
    T inv_eps;  // 1 / eps
    T xi, xi2, inv_xi;
    int well;   // 0: u^2(1-u)^2, 1: (1-s^2)^2/4
    CoefD R;
    // orientation term of Sec. 5.2, eps mu (theta . grad u)^2: c7 = eps mu h^3
    T c7, th0, th1, th2;
    int proj;   // 1: tangent-projected M = -eps P Hess u P instead of eq. Meps
    // 1: c3 = c5 = 0 in the arithmetic type (p symmetric in kappa1, kappa2), so
    // the weight c3 T + c5 q of the sqrt(D+) terms is exactly zero
    int sym;
    // FP32 voxels whose D = 2S - T^2 may have lost its accuracy to
    // cancellation recompute it (double-float; FP64 for the projected M)
    // where 2S + T^2 > rthr max(|D|, xi) and D is finite (voxel_eval):
    // rthr = 2^16, or infinity to never refine
    T rthr;
};

// Coefficient fields: c(x) = (c1..c6)(a(x)) as 6 component planes of N
// values each, built from a user's a(x) (Sec. 5.2) by launch_coef_field.
constexpr int NCF = 6;

// One problem as seen by a fused launch.
template <typename T>
struct Inst {
    const T* u;          // field read (stored field; the true field is u + scal[S_C] in MODE_STEP)
    T* out;              // g (MODE_GRAD) or next stored field (MODE_STEP)
    int nx, ny, nz;
    int zc;              // planes per z-chunk
    int tiles_x, tiles_y, chunks_z;
    int vec;             // 1: 16-byte chunked loads are legal
    int first_block;     // plain path: unused; fused: first CTA holding a partial of this problem
    int nblocks;         // number of FP64 partial slots (CTAs) of this problem in the launch
    long long unit_base; // fused: first work unit (one plane of one column tile) of this problem
    Coef<T> C;
    const T* cf;         // null, or the coefficient field c(x) [NCF][nz][ny][nx] replacing C.c1..c6
    T tau;
    double inv_N;
    double* partials;    // [nblocks][NPART]
    unsigned* ints;      // [NINTS]
    double* scal;        // [NSCAL]
    double* trace;       // [trace_cap][5] or null
    int trace_cap;
    // z-slab of a larger periodic grid: null, or 4 planes of nx*ny values
    // (the two planes below the slab, then the two above) read instead of
    // wrapping around z
    const T* halo;
    // null, or NPART doubles receiving this launch's FP64 sums for the
    // problem (the scalars are then set by a later combine over all slabs)
    double* sums_out;
};

// Problems of one fused launch, passed by value as a kernel parameter (the
// descriptors are read from the constant bank, uniformly per CTA).
constexpr int BATCH_MAX = 64;
// Work is split in units of one z-plane of one 32 x TY column tile,
// enumerated problem by problem, tile by tile, plane by plane; CTA b of G
// takes units [b W / G, (b+1) W / G).
template <typename T, int MAXI>
struct Launch {
    int n;
    int grid;            // G
    long long units;     // W
    // launches whose problems share one coefficient set and step size
    // (k_fused<..., UNI = true>) read them here, at a fixed offset of the
    // constant bank, instead of from inst[k] at a run-time index
    Coef<T> C0;
    T tau0;
    Inst<T> inst[MAXI];
};

template <typename T>
Coef<T> make_coef(const double a[6], double h, double eps, double xi, int well, double mu = 0.0,
                  const double* theta = nullptr, int proj = 0, int refine = 1);

// Automatic tile height: FP64 8 rows; FP32 the one of 16 and 13 rows that
// pads the grid's rows least (16 on a tie: its tiles hold more rows), except
// for general polynomials (not symmetric in kappa1, kappa2), whose 16-row
// instantiation keeps more values in local memory than the 13-row one: a row
// of it costs 4 % more (a 256^3 problem, pfc_run: 0.2354 ms per step at 16
// rows, 0.2295 ms at 13 with 260 rows), so they take 13 rows unless 16 pads
// more than 4 % less.
inline int default_tile_y(int ny, bool fp64, bool general = false)
{
    if (fp64) return 8;
    const int pad16 = (ny + 15) / 16 * 16, pad13 = (ny + 12) / 13 * 13;
    if (general) return pad13 < 1.04 * pad16 ? 13 : 16;
    return pad13 < pad16 ? 13 : 16;
}

// The extended sweep (orientation term, c(x), projected M) runs with 8-row tiles.
template <typename T>
inline bool needs_ext(const Inst<T>& in) { return in.cf != nullptr || in.C.c7 != T(0) || in.C.proj != 0; }
constexpr int EXT_TILE_Y = 8;
// c(x) from a(x) (both [6][n], the arithmetic type; a in the paper's order)
template <typename T>
cudaError_t launch_coef_field(const T* a_field, T* c_field, long n, double h, double eps, cudaStream_t s);

// Streaming multiprocessors of the current device (queried once per device
// ordinal and cached; launch grids are sized in multiples of it).
int device_sms();

// fused kernels (pfc_fused.cu)
// max_run > 0 caps the planes one CTA processes per problem (more CTAs);
// 0 = one CTA per SM with equal shares.  Partial slots needed per problem:
// at most fused_grid(units of the launch, max_run).
template <typename T>
cudaError_t launch_fused(const Inst<T>& in, int mode, int tile_y, int max_run, cudaStream_t s);
// `insts`: host array of descriptors (copied into the launch parameters);
// mode MODE_STEP or MODE_GRAD
cudaError_t launch_fused_batch(const Inst<float>* insts, int n_inst, int tile_y, int max_run, cudaStream_t s,
                               int mode = MODE_STEP);
long long fused_grid(long long units, int max_run);
// partial slots a single problem can need: both the requested tile height and
// the extended sweep's
long long fused_slots(int nx, int ny, int nz, int tile_y, int max_run);
template <typename T>
cudaError_t launch_add_offset(T* out, const T* in, long n, const double* c, cudaStream_t s);
// out += scal[S_C] for every problem of a batch (host descriptors), in place
cudaError_t launch_add_offset_batch(const Inst<float>* insts, int n_inst, cudaStream_t s);
// z-slabs: combine nslabs rows of FP64 sums (stride PFC_SLAB_NSUMS = 8,
// written by the slabs' sweeps) in rank order into the scalars of one slab;
// out5 (may be null) receives E, mass, lambda, max|g|, mean|g|
constexpr int SLAB_NSUMS = 8;
cudaError_t launch_slab_finish(const double* rows, int nslabs, double inv_N, int mode, double* scal, unsigned* ints,
                               double* out5, cudaStream_t s);
template <typename T>
cudaError_t launch_curvatures(const T* u, T* k1, T* k2, int nx, int ny, int nz, const Coef<T>& C,
                              double eps, cudaStream_t s);
size_t fused_smem_bytes(int elem_size, int tile_y);
int fused_threads(int tile_y);

// viability diagnostics (pfc_diag.cu): part holds 4 doubles per block
// (diag_blocks), *ticket starts at 0 and is left at 0, out receives 5 doubles
long diag_blocks(int nx, int ny, int nz);
template <typename T>
cudaError_t launch_diagnostics(const T* u, int nx, int ny, int nz, double h, double eps, int well, double* part,
                               unsigned* ticket, double* out, cudaStream_t s);

// curvature-diagram cells (pfc_surface.cu): block_counts holds
// surface_blocks(n) values, offsets surface_blocks(n) + 1 (the total last);
// cells receive min(total, cap) records (area, kappa1, kappa2)
long surface_blocks(long n);
template <typename T>
cudaError_t launch_surface_cells(const T* u, const T* k1, const T* k2, int nx, int ny, int nz, double h, double level,
                                 unsigned* block_counts, long long* offsets, T* cells, long long cap, cudaStream_t s);
template <typename T>
cudaError_t launch_curvature_histogram(const T* cells, long long n, int nbins, double lo, double hi, double* hist,
                                       cudaStream_t s);

// plain unfused path (pfc_plain.cu)
template <typename T>
struct PlainBufs {
    T* d[9];     // grad u (3) and Hess u (xx yy zz xy xz yz)
    T* ct[10];   // cotangents: ubar, dx dy dz, hxx hyy hzz hxy hxz hyz
    T* e;        // per-voxel energy density
    T* g;        // gradient
};
template <typename T>
cudaError_t launch_plain(const T* u, T* out, const PlainBufs<T>& b, int nx, int ny, int nz,
                         const Coef<T>& C, int mode, T tau, double inv_N, double* partials,
                         int nblocks, unsigned* ints, double* scal, double* trace, int trace_cap,
                         cudaStream_t s);
int plain_blocks(long n);

}  // namespace pfc
