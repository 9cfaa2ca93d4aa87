/*
 * pfc.h -- C ABI of the GB300 phase-field curvature-energy library.
 *
 * What it computes (Song, "Generation of tubular and membranous shape textures
 * with curvature functionals", arXiv 2103.04856):
 *
 *   F_eps(u) = h^3 * sum over voxels of
 *       c1 ||M||^2 + c2 (Tr M)^2 + c3 Tr M sqrt(D+) + c4 |grad u| Tr M
 *     + c5 |grad u| sqrt(D+) + c6 |grad u|^2                          (Sec. 3.2, eq. Feps)
 *   with M = -eps Hess u + (W'(u)/eps) n (x) n                        (Sec. 2.3, eq. Meps)
 *        D = 2 ||M||^2 - (Tr M)^2, sqrt(D+) its smoothed square root   (Sec. 3.1, eqs. kepsa/kepsb)
 *        c1 = (a20+a02-a11)/(2 eps), c2 = a11/(2 eps), c3 = (a20-a02)/(2 eps),
 *        c4 = (a10+a01)/2, c5 = (a10-a01)/2, c6 = a00 eps.
 *   Derivatives are periodic central finite differences on a grid of spacing h;
 *   |grad u| is regularised as sqrt(|grad u|^2 + xi^2) and x+ as
 *   xi log(1 + exp(x/xi)) (Sec. 4.1, implementation details).  The gradient is
 *   the exact derivative dE/du_i of that discrete sum.  Descent steps remove the
 *   mean of the gradient, which keeps the mass (mean of u) fixed (Sec. 4.1,
 *   mass-preserving flow).
 *
 * Conventions for every entry point:
 *  - Fields are caller-owned device arrays u[(z*ny + y)*nx + x] (torch shape
 *    (nz, ny, nx), contiguous), of float (PFC_FP32) or double (PFC_FP64) as the
 *    problem says, on the current CUDA device.  The library never frees them.
 *    A base address that is not 16-byte aligned, or nx not a multiple of
 *    16/sizeof(element), selects a slower element-wise load path (not an error).
 *  - The stream is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    enqueued on it in order; entry points with a host output wait for it.
 *  - Errors are returned as pfc_status; pfc_last_error() gives a message for
 *    the calling thread.  On PFC_ECUDA the CUDA error has been consumed.
 *  - A context is not thread-safe: one thread (or external locking) per context.
 *    Different contexts may be driven from different threads on different
 *    streams at the same time (their graph captures are thread-local, and no
 *    call but the create and destroy functions waits for the whole device).
 */
#ifndef PFC_H
#define PFC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st* pfc_stream;   /* same type as cudaStream_t */

typedef enum {
    PFC_OK = 0,
    PFC_EINVAL = -1,        /* bad argument: null pointer, size, parameter, host pointer */
    PFC_ENOMEM = -2,        /* device or host allocation failed                          */
    PFC_ECUDA = -3,         /* a CUDA call failed                                        */
    PFC_ENONFINITE = -4,    /* energy, mass or multiplier became NaN or infinite         */
    PFC_ETIMEOUT = -5,      /* a bounded device wait gave up                             */
    PFC_EUNSUPPORTED = -6   /* valid request the library does not implement            */
} pfc_status;

enum { PFC_WELL_01 = 0,     /* W(u) = u^2 (1-u)^2, wells 0 and 1                         */
       PFC_WELL_PM1 = 1 };  /* W(s) = (1-s^2)^2 / 4, wells -1 and 1 (Sec. 2.3)           */
enum { PFC_FP32 = 0, PFC_FP64 = 1 };
enum { PFC_IMPL_FUSED = 0,  /* one fused forward+adjoint stencil sweep                   */
       PFC_IMPL_PLAIN = 1 };/* unfused passes that store grad u, Hess u and cotangents   */

typedef struct {
    int32_t nx, ny, nz;     /* grid size, each >= 1                                      */
    int32_t well;           /* PFC_WELL_*                                                */
    int32_t prec;           /* PFC_FP32 or PFC_FP64: element type of every field         */
    int32_t impl;           /* PFC_IMPL_*                                                */
    double h;               /* grid spacing > 0                                          */
    double eps;             /* interface width > 0 (eq. Meps)                            */
    double xi;              /* regularisation > 0 (Sec. 4.1; 1e-6 in the paper)          */
    double a[6];            /* a20 a11 a02 a10 a01 a00 of eq. F, kappa1 >= kappa2         */
    int32_t tile_y;         /* 0 = automatic (FP64: 8; FP32: 16 or 13, whichever pads ny less; a batch:
                               by padded rows of all instances times the measured cost of a row); else 8, 13 or 16 */
    int32_t tile_z;         /* 0 = automatic; else planes per CTA z-chunk (>= 1)         */
    /* Orientation term of Sec. 5.2: eps mu (theta . grad u)^2 joins the
     * integrand (grad u the central-difference gradient).  mu = 0 (with any
     * theta) is the plain eq. Feps.  theta (x, y, z) is used as given; the
     * paper takes it of unit norm.  Fused path only (PFC_EUNSUPPORTED on the
     * plain path and in batches); it runs the extended sweep (8-row tiles). */
    double mu;
    double theta[3];
    /* 1: the tangent-projected M = -eps P Hess u P, P = I - n (x) n (the form
     * eq. Meps takes on the tanh profile, Sec. 3.1, with no double-well term)
     * replaces eq. Meps in the energy, its gradient and the curvatures; 0:
     * eq. Meps.  Fused path only; runs the extended sweep. */
    int32_t proj;
    /* PFC_FLAG_* bits; 0 for the default behaviour. */
    uint32_t flags;
} pfc_problem;

/* FP32 only: D = 2||M||^2 - (Tr M)^2 is the difference of two numbers of
 * size ||M||^2, so its FP32 rounding error is about 2^-22 (2||M||^2 + (Tr
 * M)^2).  Where that error is more than 2^-6 of max(|D|, xi) and the sqrt(D+)
 * terms carry weight (c3 Tr M + c5 |grad u| != 0), the sweep recomputes D from
 * the exact stencil inputs in double-float arithmetic (pairs of floats, about
 * 44 bits; FP64 for the projected M) (Sec. 3.1 invariants); a non-finite D
 * (invariants that overflowed FP32) is left as it is.  This flag turns
 * that refinement off (for measuring what it changes); it has no effect on
 * FP64 problems or on polynomials symmetric in kappa1, kappa2. */
#define PFC_FLAG_NO_DISCRIMINANT_REFINEMENT 1u

typedef struct pfc_ctx pfc_ctx;

/* Validates the problem and allocates the context's device scratch
 * (ping-pong field, FP64 block partials, scalars; the plain path adds 21
 * fields).  The current CUDA device at this call is the context's device. */
pfc_status pfc_create(const pfc_problem* prob, pfc_ctx** out);
void pfc_destroy(pfc_ctx* ctx);

/* E = F_eps(u) (eq. Feps).  E_host receives it; the stream is synchronised. */
pfc_status pfc_energy(pfc_ctx* ctx, const void* u, double* E_host, pfc_stream stream);

/* E and g = dE/du (same layout and type as u).  g must not alias u.
 * E_host may be NULL (then nothing is synchronised). */
pfc_status pfc_energy_and_grad(pfc_ctx* ctx, const void* u, void* g, double* E_host,
                               pfc_stream stream);

/* One mass-projected descent step: lambda = mean(g),
 * u_out = u_in - tau (g - lambda).  u_out must not alias u_in.
 * scalars_dev (device, may be NULL) receives 5 doubles:
 *   E(u_in), mean(u_in), lambda, max|g|, mean|g|.
 * Nothing is synchronised: the call only enqueues work. */
pfc_status pfc_step(pfc_ctx* ctx, const void* u_in, void* u_out, double tau,
                    double* scalars_dev, pfc_stream stream);

/* nsteps descent steps in place on u, keeping mean(u) at its entry value.
 * The step loop is captured once into a CUDA graph and replayed.  trace_host
 * (may be NULL) receives nsteps rows of the 5 scalars of pfc_step, row n
 * describing the field the n-th step evaluated.  Synchronises the stream.
 * Returns PFC_ENONFINITE if any step produced a non-finite scalar. */
pfc_status pfc_run(pfc_ctx* ctx, void* u, int32_t nsteps, double tau, double* trace_host,
                   pfc_stream stream);

/* Spatialised coefficients a(x) of Sec. 5.2: a_field (device, the context's
 * element type) holds 6 planes of N values, a_field[k*N + i] = a_k at voxel i,
 * k in the order of pfc_problem.a.  From the next call on, every evaluation
 * (energy, gradient, step, run) uses a(x) instead of the constant a.  The
 * library converts a(x) into its own copy on `stream`: a_field may be freed
 * or reused once the stream has passed this call.  a_field = NULL returns
 * to the constant a.  The first call allocates 6 fields of scratch.  Fused
 * path only (PFC_EUNSUPPORTED on the plain path); runs the extended sweep. */
pfc_status pfc_set_coefficient_field(pfc_ctx* ctx, const void* a_field, pfc_stream stream);

/* Viability diagnostics of Sec. 4.5 with the central-difference gradient
 * (no xi):  out_host[0] = h^3 sum |eps/2 |grad u|^2 - W(u)/eps| (discrepancy),
 * out_host[1] = h^3 sum (eps/2 |grad u|^2 + W(u)/eps) (Cahn-Hilliard energy,
 * the diffuse area), out_host[2] = out[0]/out[1] (in [0, 1]; 0 when out[1]
 * is 0), out_host[3] = max u, out_host[4] = min u.  The paper deems a shape
 * viable when the ratio is below 0.75 and max u > 0.1 > -0.1 > min u (wells
 * -1 and 1).  Synchronises the stream. */
pfc_status pfc_diagnostics(pfc_ctx* ctx, const void* u, double out_host[5], pfc_stream stream);
/* The same five values written to out_dev (device memory, 5 doubles):
 * enqueue only, one launch (for pipelines and CUDA graphs).  Calls of
 * pfc_diagnostics and pfc_diagnostics_dev on one context share its scratch:
 * issue them on one stream. */
pfc_status pfc_diagnostics_dev(pfc_ctx* ctx, const void* u, double* out_dev, pfc_stream stream);

/* Cells of the curvature diagram (Sec. 4.1, eq. curva_diagram): the surface
 * {u = level} (0 for the paper's wells -1/1, 0.5 for wells 0/1) triangulated
 * by marching tetrahedra on the Freudenthal split of every voxel cube
 * (periodic), one record (area, kappa1, kappa2) per triangle: its area in
 * h^2 units and the diffuse curvatures of pfc_curvatures interpolated
 * trilinearly at its barycenter.  cells (device, the context's type, 3 x cap
 * values) receives the first min(total, cap) records in cube order (z, y,
 * x), then tetrahedron, then triangle order (deterministic); *count_host
 * receives the total, so a call with cap = 0 sizes the buffer.  The first
 * call allocates 2 fields of scratch.  Synchronises the stream. */
pfc_status pfc_surface_cells(pfc_ctx* ctx, const void* u, double level, void* cells, int64_t cap,
                             int64_t* count_host, pfc_stream stream);
/* Area-weighted 2-D histogram of n cells (as written by pfc_surface_cells):
 * hist_dev (device, FP64, nbins x nbins, zeroed by the call) [b1 * nbins + b2]
 * sums the areas of the cells whose kappa1 falls in bin b1 and kappa2 in bin
 * b2 of [lo, hi) split in nbins; values outside are clamped into the edge bins
 * (the paper truncates its diagrams to [-100, 100]).  FP64 atomics: the sums
 * are exact up to rounding order.  Enqueue only. */
pfc_status pfc_curvature_histogram(pfc_ctx* ctx, const void* cells, int64_t n, int32_t nbins, double lo,
                                   double hi, double* hist_dev, pfc_stream stream);

/* Diffuse principal curvatures kappa1 >= kappa2 at every voxel (Sec. 3.1,
 * eqs. kepsa/kepsb, exact positive part, regularised |grad u|).  k1 and k2
 * have the type and layout of u. */
pfc_status pfc_curvatures(pfc_ctx* ctx, const void* u, void* k1, void* k2, pfc_stream stream);

/* ---- One periodic grid split in z across processes (one per GPU).  The
 * stencils of the sweep reach two planes (a voxel's cotangents need its
 * neighbours, whose stencils need theirs: Sec. 4.1 periodic finite
 * differences), so a slab of planes [z0, z0 + nz_local) is evaluated
 * exactly from its own planes plus the two planes below and the two above
 * it, with the periodic wrap of the whole grid.  Per step:
 *   1. fill the slab's halo from its neighbours (the caller's transport:
 *      NCCL send/recv, cudaMemcpyPeerAsync, a local copy for one slab);
 *   2. pfc_slab_sweep: the fused sweep over the slab, writing g or the
 *      stored step v = (u + c) - tau g and the slab's FP64 sums;
 *   3. gather every slab's sums (all-gather, rank order) and pfc_slab_finish:
 *      every slab combines them in the same order into the same scalars,
 *      including the offset c = m - mean(v) of the mass projection in its
 *      fused form (as pfc_run applies it), which the next STEP sweep adds to
 *      u as it loads.
 * pfc_slab_apply_offset adds the pending c to u and closes the chain. */
typedef struct pfc_slab pfc_slab;
enum { PFC_SLAB_ENERGY = 0, PFC_SLAB_GRAD = 1, PFC_SLAB_STEP = 2 };
#define PFC_SLAB_NSUMS 8     /* doubles per slab in a row of sums (6 used, 2 spare) */
/* prob: the WHOLE grid (nx, ny, nz global), fused path, FP32 or FP64 (mu and
 * proj allowed; no coefficient field).  This slab holds planes
 * [z0, z0 + nz_local), nz_local >= 2, inside [0, nz).  Allocates the slab's
 * FP64 partials and scalars (not its fields). */
pfc_status pfc_slab_create(const pfc_problem* prob, int32_t z0, int32_t nz_local, pfc_slab** out);
void pfc_slab_destroy(pfc_slab* slab);
/* One sweep over the slab.  u: the slab's nz_local planes (device, layout of
 * pfc_energy_and_grad with nz = nz_local).  halo: 4 planes of nx*ny values
 * (device, caller-owned): global planes z0-2, z0-1, z0+nz_local,
 * z0+nz_local+1 (mod nz) of the field u belongs to, e.g. the neighbouring
 * slabs' stored fields after a STEP; read, never written.  mode:
 *   PFC_SLAB_ENERGY  out unused (may be NULL);
 *   PFC_SLAB_GRAD    out = g = dE/du on the slab's planes;
 *   PFC_SLAB_STEP    out = (u + c) - tau g, c the pending offset (0 after
 *                    create and after pfc_slab_apply_offset).
 * ENERGY and GRAD evaluate u as given (apply a pending offset first).
 * sums_dev (device, PFC_SLAB_NSUMS doubles) receives this slab's FP64 sums
 * (energy, sum of u + c, sum of g, sum of |g|, max |g|, sum of out).  out
 * must not alias u or halo.  Enqueue only. */
pfc_status pfc_slab_sweep(pfc_slab* slab, const void* u, const void* halo, void* out, int32_t mode, double tau,
                          double* sums_dev, pfc_stream stream);
/* Combines nslabs rows of sums (device, nslabs x PFC_SLAB_NSUMS doubles, in
 * rank order: row r from slab r) of the last sweep, one thread in a fixed
 * order, into the slab's scalars; scalars_dev (device, may be NULL) receives
 * E, mean(u + c) (STEP only), lambda = mean g, max|g|, mean|g| of the whole
 * grid, as pfc_step's.  After a STEP the new offset c is left for the next
 * STEP sweep; the mass kept is that of the first STEP's input after create
 * or apply_offset.  Enqueue only. */
pfc_status pfc_slab_finish(pfc_slab* slab, const double* sums_all_dev, int32_t nslabs, double* scalars_dev,
                           pfc_stream stream);
/* u += c (the pending offset; u: the slab's last stored field), and the
 * chain is closed.  Enqueue only. */
pfc_status pfc_slab_apply_offset(pfc_slab* slab, void* u, pfc_stream stream);

/* Many independent problems (any sizes, each with its own coefficients and
 * step size), advanced together: every step is ONE kernel launch over the
 * tiles of all instances, and the step loop is captured in a CUDA graph.
 * FP32 and the fused path only. */
typedef struct pfc_batch pfc_batch;
pfc_status pfc_batch_create(const pfc_problem* probs, int32_t n_inst, pfc_batch** out);
void pfc_batch_destroy(pfc_batch* batch);
/* u[k]: device field of instance k, advanced in place by nsteps steps of
 * size tau[k] (host array).  trace_host (may be NULL): n_inst x nsteps x 5
 * doubles, instance-major.  Synchronises.  PFC_ENONFINITE if any instance
 * produced a non-finite scalar; the others are still advanced, while such an
 * instance is retired for the rest of the call (it is not evaluated again:
 * its field is filled with NaN and its later trace rows are NaN).  The steps
 * run in chunks of 16 launches; after each chunk the host reads the
 * instances' flags and the retired ones leave the launches, so that the
 * others' work is spread over all SMs again.  Retirement also holds within a
 * chain of pfc_batch_step_lazy calls (without leaving the launches). */
pfc_status pfc_batch_run(pfc_batch* batch, void* const* u, int32_t nsteps, const double* tau,
                         double* trace_host, pfc_stream stream);

/* One exact mass-projected step of every instance (u_out[k] = u_in[k] -
 * tau[k] (g_k - mean g_k)): one fused launch over all instances plus one
 * launch applying the projection.  Only enqueues work (no synchronisation).
 * u_out[k] must not alias u_in[k].  scalars_dev (device, may be NULL)
 * receives n_inst rows of the 5 scalars of pfc_step. */
pfc_status pfc_batch_step(pfc_batch* batch, const void* const* u_in, void* const* u_out, const double* tau,
                          double* scalars_dev, pfc_stream stream);
/* Chained steps in the fused form of the mass projection (the update of the
 * descent step with u <- u - tau (g - mean g) written, as for pfc_run, as
 * v = (u + c) - tau g with the offset c = m - mean(v) applied one step
 * later).  Each call is one fused launch over all instances: it reads
 * u_in[k], adds the offset c_k left by the previous call of the chain as it
 * loads (none when first != 0, which opens the chain and takes the mean of
 * u_in[k] as the mass m_k to keep), stores v in u_out[k] and leaves the new
 * c_k on the device.  After any number of calls the projected field of
 * instance k is u_out[k] + c_k; pfc_batch_lazy_finish(u_out) adds c_k in
 * place (one launch) and closes the chain.  Results equal a sequence of
 * pfc_batch_step calls up to FP32 rounding (the offset enters the loads, not
 * the stencil differences).  u_out[k] must not alias u_in[k]; enqueue only;
 * PFC_EINVAL for first == 0 without an open chain, and for first != 0 while
 * a chain is open (its pending offsets would be lost).  pfc_batch_step,
 * pfc_batch_run and pfc_batch_step_host close an open chain (they reset the
 * offsets). */
pfc_status pfc_batch_step_lazy(pfc_batch* batch, const void* const* u_in, void* const* u_out, const double* tau,
                               int32_t first, pfc_stream stream);
pfc_status pfc_batch_lazy_finish(pfc_batch* batch, void* const* u, pfc_stream stream);
/* pfc_batch_step from and to HOST memory: u_in_host[k] is copied to the
 * device, stepped, and the result copied to u_out_host[k] (host arrays of
 * the instances' sizes, float; page-locked memory lets the copies overlap,
 * pageable memory works but serialises them).  Enqueue only: the instances
 * are pipelined over two internal copy streams beside `stream` (which runs
 * the steps, one fused launch plus its projection per instance), and
 * consecutive calls overlap (the copies out of one step with the copies in
 * of the next).  u_out_host[k] holds the result once pfc_batch_host_wait
 * returns; the caller must not change u_in_host / u_out_host before then.
 * The first call allocates one device field per instance. */
pfc_status pfc_batch_step_host(pfc_batch* batch, const void* const* u_in_host, void* const* u_out_host,
                               const double* tau, pfc_stream stream);
/* Waits for every step enqueued by pfc_batch_step_host (on `stream` and on
 * the copy streams). */
pfc_status pfc_batch_host_wait(pfc_batch* batch, pfc_stream stream);
/* Optional device timing of pfc_batch_step: when enabled, the library records
 * CUDA events on the stream around the whole step and around its fused
 * sweep kernel; pfc_batch_last_timing waits for them and returns the two
 * durations of the most recent step in milliseconds. */
pfc_status pfc_batch_timing(pfc_batch* batch, int enable);
pfc_status pfc_batch_last_timing(pfc_batch* batch, float* step_ms, float* sweep_ms);

/* ---- The paper's generator (Alg. 1, Sec. 4.1): the H^-1 flow of F_eps run as
 * an L2 flow on a periodic vector field A through u = div A + m0 (eq.
 * change_var), with a small Gaussian blur of u before the energy and Adam on
 * A.  A, and the Adam moments m, v, are caller-owned device arrays of 3 x N
 * values (component-major: A_x, A_y, A_z, each laid out like u) of the
 * problem's type.  The mass of u = k * (div A + m0) is m0 exactly. */
typedef struct {
    double m0;              /* mean of u (Alg. 1: the mass)                             */
    double lr, beta1, beta2, adam_eps;   /* Adam; Sec. 4.1: 1e-3, 0.9, 0.999, no decay  */
    double blur_sigma;      /* Gaussian std in voxels (Sec. 4.1: 2); 0 = no blur        */
    int32_t blur_radius;    /* taps per side; 0 = ceil(3 sigma); at most 32             */
    int32_t reserved;
} pfc_hflow_params;
typedef struct pfc_hflow pfc_hflow;
/* prob: grid, coefficients and precision (fused path); allocates 4 fields of
 * scratch plus reduction slots. */
pfc_status pfc_hflow_create(const pfc_problem* prob, const pfc_hflow_params* params, pfc_hflow** out);
void pfc_hflow_destroy(pfc_hflow* flow);
/* ut = k * (div A + m0): the phase field the flow evaluates (enqueue only). */
pfc_status pfc_hflow_field(pfc_hflow* flow, const void* A, void* ut, pfc_stream stream);
/* G(A) = F_eps(k * (div A + m0)) and gA = dG/dA (3 x N).  G_host may be NULL
 * (then nothing is synchronised). */
pfc_status pfc_hflow_grad(pfc_hflow* flow, const void* A, void* gA, double* G_host, pfc_stream stream);
/* nsteps Adam steps of Alg. 1 in place on A, m, v; *t is Adam's step count
 * (0 for fresh moments), advanced by nsteps.  trace_host (may be NULL):
 * nsteps rows {G, max|dG/dA|, mean|dG/dA|, mean(u), t}.  The loop runs as
 * CUDA-graph replays of 32 steps.  Synchronises the stream. */
pfc_status pfc_hflow_run(pfc_hflow* flow, void* A, void* m, void* v, int32_t nsteps, int32_t* t,
                         double* trace_host, pfc_stream stream);

/* Batches of the generator: up to 64 flows on grids of one size advanced
 * together, every kernel of an iteration one launch over all of them (the
 * paper generates many shapes, e.g. its atlas of Sec. 4.5; one 100^3 flow
 * alone cannot fill the GPU).  probs: n_inst problems with equal nx, ny, nz,
 * FP32, fused path, mu = 0, proj = 0 (otherwise PFC_EUNSUPPORTED or
 * PFC_EINVAL); their coefficients, eps, h, xi and double wells may differ.
 * m0: n_inst masses (params->m0 is ignored); the blur and Adam's settings of
 * params are shared.  A[k], m[k], v[k]: instance k's fields as for
 * pfc_hflow_run; *t is the common Adam step count.  trace_host (may be
 * NULL): n_inst x nsteps rows of pfc_hflow_run's trace, instance-major.
 * Allocates 4 fields of scratch per instance. */
typedef struct pfc_hflow_batch pfc_hflow_batch;
pfc_status pfc_hflow_batch_create(const pfc_problem* probs, const double* m0, int32_t n_inst,
                                  const pfc_hflow_params* params, pfc_hflow_batch** out);
void pfc_hflow_batch_destroy(pfc_hflow_batch* batch);
/* ut[k] = k * (div A[k] + m0[k]) for every instance (enqueue only). */
pfc_status pfc_hflow_batch_field(pfc_hflow_batch* batch, const void* const* A, void* const* ut, pfc_stream stream);
/* nsteps Adam steps of every instance, in place; CUDA-graph replays of 32
 * steps; synchronises the stream. */
pfc_status pfc_hflow_batch_run(pfc_hflow_batch* batch, void* const* A, void* const* m, void* const* v,
                               int32_t nsteps, int32_t* t, double* trace_host, pfc_stream stream);

/* Spatialised generation parameters (Sec. 5.2) for the flow: a(x) as for
 * pfc_set_coefficient_field, and m(x) (device, N values of the problem's
 * type): u = k * (div A + m(x)), whose mean is mean(m).  Both are copied on
 * `stream` (the caller's buffers may be freed once the stream has passed the
 * call); NULL returns to the constant a / m0. */
pfc_status pfc_hflow_set_coefficient_field(pfc_hflow* flow, const void* a_field, pfc_stream stream);
pfc_status pfc_hflow_set_mass_field(pfc_hflow* flow, const void* m_field, pfc_stream stream);

/* pfc_energy_and_grad without any device allocation, for callers that may not
 * call cudaMalloc/cudaFree (graph-capture regions, host callbacks, plugins in
 * a process that owns the device's memory budget, loops that must not take
 * the allocator's implicit device-wide synchronisation).  The paper has no
 * counterpart: this is an interface convenience.
 *  - prob: the problem (impl must be PFC_IMPL_FUSED); u, g: caller-owned
 *    fields of the current device as for pfc_energy_and_grad (PFC_EINVAL for
 *    host memory, another device's memory, or g == u); E_host may be NULL:
 *    then the call only enqueues work, and the scratch stays in use until the
 *    stream has run it.  PFC_ENONFINITE if E_host receives a non-finite energy.
 *  - Scratch: a static device array in the library (49,232 bytes, held by
 *    every GPU that loads the library until the process exits) with room for
 *    1024 CTAs of FP64 partial sums; a problem that would need more CTAs
 *    (only possible with a small tile_z) returns PFC_EINVAL.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 *  - All calls share the one array: calls that overlap on the GPU (two
 *    streams, or two host threads) race and give wrong results.  Serialise
 *    them, e.g. on one stream. */
pfc_status pfc_energy_and_grad_noalloc(const pfc_problem* prob, const void* u, void* g, double* E_host,
                                       pfc_stream stream);

/* FP32 FMA throughput of the current device in TFLOP/s (2 flops per FMA):
 * independent FMA chains on every SM, the best of three launches timed with
 * CUDA events on `stream` after one warm-up (about 20 ms each at the GB300's
 * maximum clock).  The denominator of the fused sweep's arithmetic roofline;
 * the paper has no counterpart.  Allocates nothing (two events); changes no
 * device setting; synchronises the stream. */
pfc_status pfc_measure_fp32_peak(double* tflops_host, pfc_stream stream);

/* eq. redundant: b = (h2, H0, k1, alpha, kappa1_0, beta, kappa2_0) expanded
 * into a = (a20, a11, a02, a10, a01, a00).  Host only. */
pfc_status pfc_b_to_a(const double b[7], double a_out[6]);

const char* pfc_status_string(pfc_status s);
const char* pfc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
