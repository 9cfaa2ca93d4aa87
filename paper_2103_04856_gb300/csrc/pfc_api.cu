// pfc_api.cu -- the C ABI declared in include/pfc.h: argument checks, device
// scratch, launch geometry, the CUDA-graph step loop and the batch runner.
#include <cuda_runtime.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pfc.h"
#include "pfc_internal.h"

using namespace pfc;

static thread_local char g_err[512] = "";

// NVTX range around an entry point (visible in profilers; no cost otherwise)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

static pfc_status fail(pfc_status s, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}

namespace pfc {
// lets other translation units of the library report through pfc_last_error
void set_last_error(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }
}  // namespace pfc

#define PFC_CU(call)                                                                                 \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) {                                                                     \
            (void)cudaGetLastError();                                                                \
            return fail(PFC_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                                   \
        }                                                                                            \
    } while (0)

// ------------------------------------------------------------ context

struct pfc_ctx {
    pfc_problem P;
    int device = 0;
    int esz = 4;
    long N = 0;
    int tile_y = 16, zc = 0, tiles_x = 0, tiles_y = 0, chunks_z = 0, nblocks = 0;
    int plain_nblocks = 0;
    void* ping = nullptr;            // second field of the step loop
    double* partials = nullptr;
    unsigned* ints = nullptr;
    double* scal = nullptr;
    double* trace = nullptr;
    int trace_cap = 0;
    void* plain_mem = nullptr;       // 21 fields for the plain path
    void* cfield = nullptr;          // c(x) from pfc_set_coefficient_field (NCF fields)
    bool cf_on = false;
    double* dpart = nullptr;         // diagnostics: block partials, ticket, 5 results
    unsigned* dticket = nullptr;
    double* dout = nullptr;
    void* skap = nullptr;            // surface cells: kappa1, kappa2 fields, block counts, offsets
    unsigned* sblk = nullptr;
    long long* soff = nullptr;
    // cached step-loop graph
    cudaGraphExec_t gexec = nullptr;
    const void* g_u = nullptr;
    double g_tau = 0.0;
    int g_len = 0;
    double* g_trace = nullptr;
    bool g_cf = false;
    cudaStream_t cap = nullptr;
};


// 1 unless the problem turns the FP32 discriminant refinement off
static int refine_of(const pfc_problem& p) { return (p.flags & PFC_FLAG_NO_DISCRIMINANT_REFINEMENT) ? 0 : 1; }

static pfc_status check_problem(const pfc_problem* p)
{
    if (!p) return fail(PFC_EINVAL, "problem is NULL");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(PFC_EINVAL, "grid %dx%dx%d: every size must be >= 1", p->nx, p->ny, p->nz);
    if ((double)p->nx * p->ny * p->nz > 2.0e9) return fail(PFC_EINVAL, "grid too large (more than 2e9 voxels)");
    if (!(p->h > 0) || !isfinite(p->h)) return fail(PFC_EINVAL, "h must be finite and > 0");
    if (!(p->eps > 0) || !isfinite(p->eps)) return fail(PFC_EINVAL, "eps must be finite and > 0");
    if (!(p->xi > 0) || !isfinite(p->xi)) return fail(PFC_EINVAL, "xi must be finite and > 0");
    for (int i = 0; i < 6; ++i)
        if (!isfinite(p->a[i])) return fail(PFC_EINVAL, "coefficient a[%d] is not finite", i);
    if (p->well != PFC_WELL_01 && p->well != PFC_WELL_PM1) return fail(PFC_EINVAL, "unknown double well %d", p->well);
    if (p->prec != PFC_FP32 && p->prec != PFC_FP64) return fail(PFC_EINVAL, "unknown precision %d", p->prec);
    if (p->impl != PFC_IMPL_FUSED && p->impl != PFC_IMPL_PLAIN) return fail(PFC_EINVAL, "unknown implementation %d", p->impl);
    if (p->tile_y != 0 && p->tile_y != 8 && p->tile_y != 13 && p->tile_y != 16) return fail(PFC_EINVAL, "tile_y must be 0, 8, 13 or 16");
    if (p->tile_z < 0) return fail(PFC_EINVAL, "tile_z must be >= 0");
    if (!isfinite(p->mu) || !isfinite(p->theta[0]) || !isfinite(p->theta[1]) || !isfinite(p->theta[2]))
        return fail(PFC_EINVAL, "mu and theta must be finite");
    if (p->mu != 0.0 && p->impl != PFC_IMPL_FUSED)
        return fail(PFC_EUNSUPPORTED, "the orientation term (mu != 0) runs on the fused path only");
    if (p->proj != 0 && p->proj != 1) return fail(PFC_EINVAL, "proj must be 0 or 1");
    if (p->flags & ~PFC_FLAG_NO_DISCRIMINANT_REFINEMENT) return fail(PFC_EINVAL, "unknown flags 0x%x", p->flags);
    if (p->proj && p->impl != PFC_IMPL_FUSED)
        return fail(PFC_EUNSUPPORTED, "the projected M runs on the fused path only");
    return PFC_OK;
}

// Automatic tile height of a batch (its launches run the batched
// instantiations, MAXI = 64): the one of 16 and 13 rows with the smaller
// cost, the rows padded to whole tiles (summed over the problems' x-z planes)
// times the measured cost of a row.  In the symmetric sweep a 13-row tile's
// row costs 4.3 % more (four 128^3 problems: 87.5 us at 16 rows, 92.7 us at
// 13, padded to 130 rows).  In the general sweep the 16-row instantiation (20
// warps at 96 registers) keeps more values in local memory than the 13-row
// one (16 warps at 128 registers), the more so when the problems' coefficients
// differ (they are then loaded per use from the descriptor table): its row
// costs 3.5 % more with one coefficient set (a 512^3 problem: 1.795 ms at 16
// rows, 1.761 ms at 13, padded to 520 rows) and 10 % more with many (the
// 64-instance mixed batch of 64^3, 96^3 and 128^3 problems: 1.03 against 0.97
// ms per step, 4.1 % more rows at 13).  Single problems (MAXI = 1) take
// default_tile_y.
static int auto_tile_y(const pfc_problem* p, int n)
{
    if (p[0].prec == PFC_FP64) return 8;
    bool general = false, one_set = true;
    double rows16 = 0.0, rows13 = 0.0;
    for (int k = 0; k < n; ++k) {
        const double plane = (double)p[k].nx * p[k].nz;
        rows16 += plane * ((p[k].ny + 15) / 16 * 16);
        rows13 += plane * ((p[k].ny + 12) / 13 * 13);
        general = general || !make_coef<float>(p[k].a, p[k].h, p[k].eps, p[k].xi, p[k].well).sym;
        one_set = one_set && memcmp(p[k].a, p[0].a, sizeof(p[0].a)) == 0 && p[k].h == p[0].h &&
                  p[k].eps == p[0].eps && p[k].xi == p[0].xi && p[k].well == p[0].well;
    }
    const double c16 = general ? (one_set ? 1.035 : 1.10) : 1.0, c13 = general ? 1.0 : 1.043;
    return rows13 * c13 < rows16 * c16 ? 13 : 16;
}

// Launch geometry of one problem: 32 x tile_y columns per CTA, z chunks chosen
// so that the grid fills the GPU about twice unless the user fixed tile_z.
static void geometry(const pfc_problem* p, int sms, int* tile_y, int* zc, int* tx, int* ty, int* cz)
{
    const bool general = !make_coef<float>(p->a, p->h, p->eps, p->xi, p->well).sym;
    int tyv = p->tile_y ? p->tile_y : default_tile_y(p->ny, p->prec == PFC_FP64, general);
    *tile_y = tyv;
    *tx = (p->nx + 31) / 32;
    *ty = (p->ny + tyv - 1) / tyv;
    int z = p->tile_z ? p->tile_z : p->nz;
    if (!p->tile_z) {
        const long cols = (long)(*tx) * (*ty);
        while (z > 16 && cols * ((p->nz + z - 1) / z) < 2L * sms) z = (z + 1) / 2;
    }
    if (z > p->nz) z = p->nz;
    *zc = z;
    *cz = (p->nz + z - 1) / z;
}

// ptr is device (or managed) memory of `device`, and `device` is current:
// the kernels run on the current device and must not touch another GPU's
// memory
static bool on_device(const void* ptr, int device)
{
    cudaPointerAttributes at;
    int cur = -1;
    if (!ptr || cudaGetDevice(&cur) != cudaSuccess || cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == device &&
           cur == device;
}

static pfc_status check_dev_ptr(const pfc_ctx* c, const void* ptr, const char* name)
{
    if (!ptr) return fail(PFC_EINVAL, "%s is NULL", name);
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(PFC_EINVAL, "%s: not a CUDA pointer (%s)", name, cudaGetErrorString(e));
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(PFC_EINVAL, "%s is not device memory", name);
    if (at.device != c->device) return fail(PFC_EINVAL, "%s is on device %d, context on %d", name, at.device, c->device);
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != c->device) {
        (void)cudaGetLastError();
        return fail(PFC_EINVAL, "the context's device %d is not the current device", c->device);
    }
    return PFC_OK;
}

static void free_ctx_mem(pfc_ctx* c)
{
    cudaFree(c->ping);
    cudaFree(c->partials);
    cudaFree(c->ints);
    cudaFree(c->scal);
    cudaFree(c->trace);
    cudaFree(c->plain_mem);
    cudaFree(c->cfield);
    cudaFree(c->dpart);
    cudaFree(c->dticket);
    cudaFree(c->dout);
    cudaFree(c->skap);
    cudaFree(c->sblk);
    cudaFree(c->soff);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->cap) cudaStreamDestroy(c->cap);
}

extern "C" pfc_status pfc_create(const pfc_problem* prob, pfc_ctx** out)
{
    if (!out) return fail(PFC_EINVAL, "out is NULL");
    *out = nullptr;
    pfc_status st = check_problem(prob);
    if (st) return st;
    pfc_ctx* c = new (std::nothrow) pfc_ctx();
    if (!c) return fail(PFC_ENOMEM, "host allocation failed");
    c->P = *prob;
    c->esz = prob->prec == PFC_FP64 ? 8 : 4;
    c->N = (long)prob->nx * prob->ny * prob->nz;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        delete c;
        (void)cudaGetLastError();
        return fail(PFC_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    }
    geometry(prob, device_sms(), &c->tile_y, &c->zc, &c->tiles_x, &c->tiles_y, &c->chunks_z);
    c->nblocks = (int)fused_slots(prob->nx, prob->ny, prob->nz, c->tile_y, prob->tile_z);
    c->plain_nblocks = plain_blocks(c->N);
    const int nparts = c->nblocks > c->plain_nblocks ? c->nblocks : c->plain_nblocks;
    bool ok = cudaMalloc(&c->ping, (size_t)c->esz * c->N) == cudaSuccess &&
              cudaMalloc((void**)&c->partials, sizeof(double) * NPART * (size_t)nparts) == cudaSuccess &&
              cudaMalloc((void**)&c->ints, sizeof(unsigned) * NINTS) == cudaSuccess &&
              cudaMalloc((void**)&c->scal, sizeof(double) * NSCAL) == cudaSuccess &&
              cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) == cudaSuccess;
    if (ok && prob->impl == PFC_IMPL_PLAIN)
        ok = cudaMalloc(&c->plain_mem, (size_t)c->esz * c->N * 21) == cudaSuccess;
    // cleared on the context's own stream (no device-wide wait, see ensure_trace)
    if (ok) ok = cudaMemsetAsync(c->ints, 0, sizeof(unsigned) * NINTS, c->cap) == cudaSuccess &&
                 cudaMemsetAsync(c->scal, 0, sizeof(double) * NSCAL, c->cap) == cudaSuccess &&
                 cudaStreamSynchronize(c->cap) == cudaSuccess;
    if (!ok) {
        cudaError_t le = cudaGetLastError();
        free_ctx_mem(c);
        delete c;
        return fail(PFC_ENOMEM, "device allocation failed: %s", cudaGetErrorString(le));
    }
    *out = c;
    return PFC_OK;
}

extern "C" void pfc_destroy(pfc_ctx* c)
{
    if (!c) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    free_ctx_mem(c);
    cudaSetDevice(prev);
    delete c;
}

template <typename T>
static Inst<T> make_inst(const pfc_ctx* c, const void* u, void* out, double tau)
{
    Inst<T> in{};
    const pfc_problem& P = c->P;
    in.u = (const T*)u;
    in.out = (T*)out;
    in.nx = P.nx; in.ny = P.ny; in.nz = P.nz;
    in.zc = c->zc;
    in.tiles_x = c->tiles_x; in.tiles_y = c->tiles_y; in.chunks_z = c->chunks_z;
    const int vecw = 16 / (int)sizeof(T);
    in.vec = (P.nx % vecw == 0) && (((uintptr_t)u) % 16 == 0);
    in.first_block = 0;
    in.nblocks = c->nblocks;
    in.C = make_coef<T>(P.a, P.h, P.eps, P.xi, P.well, P.mu, P.theta, P.proj, refine_of(P));
    in.cf = c->cf_on ? (const T*)c->cfield : nullptr;
    in.tau = (T)tau;
    in.inv_N = 1.0 / (double)c->N;
    in.partials = c->partials;
    in.ints = c->ints;
    in.scal = c->scal;
    in.trace = c->trace;
    in.trace_cap = c->trace_cap;
    return in;
}

template <typename T>
static PlainBufs<T> plain_bufs(const pfc_ctx* c)
{
    PlainBufs<T> b;
    T* base = (T*)c->plain_mem;
    for (int i = 0; i < 9; ++i) b.d[i] = base + (size_t)i * c->N;
    for (int i = 0; i < 10; ++i) b.ct[i] = base + (size_t)(9 + i) * c->N;
    b.e = base + (size_t)19 * c->N;
    b.g = base + (size_t)20 * c->N;
    return b;
}

// Enqueue one evaluation (MODE_ENERGY / MODE_GRAD) or one step (MODE_STEP;
// fused: lazy offset, plain: explicit projection).
static cudaError_t enqueue(pfc_ctx* c, int mode, const void* u, void* out, double tau, cudaStream_t s)
{
    if (c->P.impl == PFC_IMPL_PLAIN) {
        if (c->P.prec == PFC_FP64)
            return launch_plain<double>((const double*)u, (double*)out, plain_bufs<double>(c), c->P.nx, c->P.ny,
                                        c->P.nz, make_coef<double>(c->P.a, c->P.h, c->P.eps, c->P.xi, c->P.well, c->P.mu, c->P.theta, c->P.proj, refine_of(c->P)),
                                        mode, tau, 1.0 / (double)c->N, c->partials, c->plain_nblocks, c->ints,
                                        c->scal, c->trace, c->trace_cap, s);
        return launch_plain<float>((const float*)u, (float*)out, plain_bufs<float>(c), c->P.nx, c->P.ny, c->P.nz,
                                   make_coef<float>(c->P.a, c->P.h, c->P.eps, c->P.xi, c->P.well, c->P.mu, c->P.theta, c->P.proj, refine_of(c->P)), mode,
                                   (float)tau, 1.0 / (double)c->N, c->partials, c->plain_nblocks, c->ints, c->scal,
                                   c->trace, c->trace_cap, s);
    }
    if (c->P.prec == PFC_FP64)
        return launch_fused<double>(make_inst<double>(c, u, out, tau), mode, c->tile_y, c->P.tile_z, s);
    return launch_fused<float>(make_inst<float>(c, u, out, tau), mode, c->tile_y, c->P.tile_z, s);
}

static pfc_status read_scalar(pfc_ctx* c, int slot, double* host, cudaStream_t s)
{
    PFC_CU(cudaMemcpyAsync(host, c->scal + slot, sizeof(double), cudaMemcpyDeviceToHost, s));
    PFC_CU(cudaStreamSynchronize(s));
    return PFC_OK;
}

extern "C" pfc_status pfc_energy(pfc_ctx* c, const void* u, double* E_host, pfc_stream stream)
{
    if (!c) return fail(PFC_EINVAL, "context is NULL");
    if (!E_host) return fail(PFC_EINVAL, "E_host is NULL");
    pfc_status st = check_dev_ptr(c, u, "u");
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    PFC_CU(enqueue(c, MODE_ENERGY, u, nullptr, 0.0, s));
    st = read_scalar(c, S_E, E_host, s);
    if (st) return st;
    if (!isfinite(*E_host)) return fail(PFC_ENONFINITE, "energy is not finite");
    return PFC_OK;
}

extern "C" pfc_status pfc_energy_and_grad(pfc_ctx* c, const void* u, void* g, double* E_host, pfc_stream stream)
{
    NvtxRange nvtx_("pfc_energy_and_grad");
    if (!c) return fail(PFC_EINVAL, "context is NULL");
    pfc_status st = check_dev_ptr(c, u, "u");
    if (st) return st;
    if ((st = check_dev_ptr(c, g, "g"))) return st;
    if (u == g) return fail(PFC_EINVAL, "g must not alias u");
    cudaStream_t s = (cudaStream_t)stream;
    PFC_CU(enqueue(c, MODE_GRAD, u, g, 0.0, s));
    if (E_host) {
        st = read_scalar(c, S_E, E_host, s);
        if (st) return st;
        if (!isfinite(*E_host)) return fail(PFC_ENONFINITE, "energy is not finite");
    }
    return PFC_OK;
}

// One step without the graph: u_out = u_in - tau (g - mean g).
static pfc_status step_now(pfc_ctx* c, const void* u_in, void* u_out, double tau, cudaStream_t s)
{
    PFC_CU(cudaMemsetAsync(c->ints + I_COUNTER, 0, sizeof(unsigned), s));
    PFC_CU(cudaMemsetAsync(c->scal + S_C, 0, sizeof(double), s));
    PFC_CU(enqueue(c, MODE_STEP, u_in, u_out, tau, s));
    if (c->P.impl == PFC_IMPL_FUSED) {
        if (c->P.prec == PFC_FP64)
            PFC_CU(launch_add_offset<double>((double*)u_out, (const double*)u_out, c->N, c->scal + S_C, s));
        else
            PFC_CU(launch_add_offset<float>((float*)u_out, (const float*)u_out, c->N, c->scal + S_C, s));
    }
    return PFC_OK;
}

extern "C" pfc_status pfc_step(pfc_ctx* c, const void* u_in, void* u_out, double tau, double* scalars_dev,
                               pfc_stream stream)
{
    if (!c) return fail(PFC_EINVAL, "context is NULL");
    pfc_status st = check_dev_ptr(c, u_in, "u_in");
    if (st) return st;
    if ((st = check_dev_ptr(c, u_out, "u_out"))) return st;
    if (u_in == u_out) return fail(PFC_EINVAL, "u_out must not alias u_in");
    if (!isfinite(tau)) return fail(PFC_EINVAL, "tau is not finite");
    if (scalars_dev && (st = check_dev_ptr(c, scalars_dev, "scalars_dev"))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = step_now(c, u_in, u_out, tau, s))) return st;
    if (scalars_dev)
        PFC_CU(cudaMemcpyAsync(scalars_dev, c->scal, 5 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return PFC_OK;
}

// Grows the trace buffer.  Only this call's stream is waited for (earlier
// runs of the context ended with a synchronisation of theirs): a device-wide
// wait would break a graph capture that another thread has in progress.
static pfc_status ensure_trace(pfc_ctx* c, int n, cudaStream_t s)
{
    if (n <= c->trace_cap) return PFC_OK;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    PFC_CU(cudaStreamSynchronize(s));
    cudaFree(c->trace);
    c->trace = nullptr;
    c->trace_cap = 0;
    PFC_CU(cudaMalloc((void**)&c->trace, sizeof(double) * 5 * (size_t)n));
    c->trace_cap = n;
    return PFC_OK;
}

// Steps i0 .. i0+n-1 of a run: even steps read `a` and write `b`, odd steps the
// reverse (n even keeps the parity).
static cudaError_t enqueue_steps(pfc_ctx* c, void* a, void* b, int i0, int n, double tau, cudaStream_t s)
{
    for (int i = i0; i < i0 + n; ++i) {
        const bool even = (i % 2) == 0;
        cudaError_t e = enqueue(c, MODE_STEP, even ? a : b, even ? b : a, tau, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

extern "C" pfc_status pfc_run(pfc_ctx* c, void* u, int32_t nsteps, double tau, double* trace_host, pfc_stream stream)
{
    NvtxRange nvtx_("pfc_run");
    if (!c) return fail(PFC_EINVAL, "context is NULL");
    pfc_status st = check_dev_ptr(c, u, "u");
    if (st) return st;
    if (nsteps < 0) return fail(PFC_EINVAL, "nsteps must be >= 0");
    if (!isfinite(tau)) return fail(PFC_EINVAL, "tau is not finite");
    if (nsteps == 0) return PFC_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_trace(c, nsteps, s))) return st;
    PFC_CU(cudaMemsetAsync(c->ints, 0, sizeof(unsigned) * NINTS, s));
    PFC_CU(cudaMemsetAsync(c->scal, 0, sizeof(double) * NSCAL, s));
    // a CUDA graph of G steps (G even) replayed; the remainder is launched directly
    const int G = nsteps >= 64 ? 64 : (nsteps & ~1);
    if (G >= 2) {
        if (!(c->gexec && c->g_u == u && c->g_tau == tau && c->g_len == G && c->g_trace == c->trace &&
              c->g_cf == c->cf_on)) {
            if (c->gexec) {
                cudaGraphExecDestroy(c->gexec);
                c->gexec = nullptr;
            }
            cudaGraph_t graph = nullptr;
            PFC_CU(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = enqueue_steps(c, u, c->ping, 0, G, tau, c->cap);
            cudaError_t e2 = cudaStreamEndCapture(c->cap, &graph);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                (void)cudaGetLastError();
                return fail(PFC_ECUDA, "graph capture failed: %s",
                            cudaGetErrorString(e != cudaSuccess ? e : e2));
            }
            e = cudaGraphInstantiate(&c->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                c->gexec = nullptr;
                (void)cudaGetLastError();
                return fail(PFC_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
            }
            c->g_u = u;
            c->g_tau = tau;
            c->g_len = G;
            c->g_trace = c->trace;
            c->g_cf = c->cf_on;
        }
        for (int k = 0; k + G <= nsteps; k += G) PFC_CU(cudaGraphLaunch(c->gexec, s));
    }
    const int done = G >= 2 ? (nsteps / G) * G : 0;
    PFC_CU(enqueue_steps(c, u, c->ping, done, nsteps - done, tau, s));
    // the result is in u (even nsteps) or in the ping buffer; apply the offset
    const bool in_ping = (nsteps % 2) == 1;
    if (c->P.impl == PFC_IMPL_FUSED) {
        if (c->P.prec == PFC_FP64)
            PFC_CU(launch_add_offset<double>((double*)u, (const double*)(in_ping ? c->ping : u), c->N, c->scal + S_C, s));
        else
            PFC_CU(launch_add_offset<float>((float*)u, (const float*)(in_ping ? c->ping : u), c->N, c->scal + S_C, s));
    } else if (in_ping) {
        PFC_CU(cudaMemcpyAsync(u, c->ping, (size_t)c->esz * c->N, cudaMemcpyDeviceToDevice, s));
    }
    unsigned ints[NINTS];
    PFC_CU(cudaMemcpyAsync(ints, c->ints, sizeof ints, cudaMemcpyDeviceToHost, s));
    if (trace_host)
        PFC_CU(cudaMemcpyAsync(trace_host, c->trace, sizeof(double) * 5 * (size_t)nsteps, cudaMemcpyDeviceToHost, s));
    PFC_CU(cudaStreamSynchronize(s));
    if (ints[I_COUNTER] != (unsigned)nsteps)
        return fail(PFC_ECUDA, "step counter %u != %d", ints[I_COUNTER], nsteps);
    if (ints[I_NONFINITE]) return fail(PFC_ENONFINITE, "a step produced a non-finite energy, mass or multiplier");
    return PFC_OK;
}

extern "C" pfc_status pfc_curvatures(pfc_ctx* c, const void* u, void* k1, void* k2, pfc_stream stream)
{
    if (!c) return fail(PFC_EINVAL, "context is NULL");
    pfc_status st = check_dev_ptr(c, u, "u");
    if (st) return st;
    if ((st = check_dev_ptr(c, k1, "k1")) || (st = check_dev_ptr(c, k2, "k2"))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const pfc_problem& P = c->P;
    if (P.prec == PFC_FP64)
        PFC_CU(launch_curvatures<double>((const double*)u, (double*)k1, (double*)k2, P.nx, P.ny, P.nz,
                                         make_coef<double>(P.a, P.h, P.eps, P.xi, P.well, 0.0, nullptr, P.proj), P.eps, s));
    else
        PFC_CU(launch_curvatures<float>((const float*)u, (float*)k1, (float*)k2, P.nx, P.ny, P.nz,
                                        make_coef<float>(P.a, P.h, P.eps, P.xi, P.well, 0.0, nullptr, P.proj), P.eps, s));
    return PFC_OK;
}

extern "C" pfc_status pfc_set_coefficient_field(pfc_ctx* c, const void* a_field, pfc_stream stream)
{
    if (!c) return fail(PFC_EINVAL, "context is NULL");
    if (c->P.impl != PFC_IMPL_FUSED) return fail(PFC_EUNSUPPORTED, "a(x) runs on the fused path only");
    if (!a_field) {
        c->cf_on = false;
        return PFC_OK;
    }
    pfc_status st = check_dev_ptr(c, a_field, "a_field");
    if (st) return st;
    if (!c->cfield) PFC_CU(cudaMalloc(&c->cfield, (size_t)c->esz * NCF * c->N));
    cudaStream_t s = (cudaStream_t)stream;
    if (c->P.prec == PFC_FP64)
        PFC_CU(launch_coef_field<double>((const double*)a_field, (double*)c->cfield, c->N, c->P.h, c->P.eps, s));
    else
        PFC_CU(launch_coef_field<float>((const float*)a_field, (float*)c->cfield, c->N, c->P.h, c->P.eps, s));
    c->cf_on = true;
    return PFC_OK;
}

// One diagnostics launch writing its five values to out (device; null: the
// context's own five doubles).
static pfc_status diagnostics_launch(pfc_ctx* c, const void* u, double* out, cudaStream_t s)
{
    if (!c->dpart) {
        PFC_CU(cudaMalloc((void**)&c->dpart, sizeof(double) * 4 * (size_t)diag_blocks(c->P.nx, c->P.ny, c->P.nz)));
        PFC_CU(cudaMalloc((void**)&c->dticket, sizeof(unsigned)));
        PFC_CU(cudaMalloc((void**)&c->dout, sizeof(double) * 5));
        PFC_CU(cudaMemset(c->dticket, 0, sizeof(unsigned)));
    }
    const pfc_problem& P = c->P;
    if (!out) out = c->dout;
    if (P.prec == PFC_FP64)
        PFC_CU(launch_diagnostics<double>((const double*)u, P.nx, P.ny, P.nz, P.h, P.eps, P.well, c->dpart,
                                          c->dticket, out, s));
    else
        PFC_CU(launch_diagnostics<float>((const float*)u, P.nx, P.ny, P.nz, P.h, P.eps, P.well, c->dpart,
                                         c->dticket, out, s));
    return PFC_OK;
}

extern "C" pfc_status pfc_diagnostics(pfc_ctx* c, const void* u, double out_host[5], pfc_stream stream)
{
    NvtxRange nvtx_("pfc_diagnostics");
    if (!c) return fail(PFC_EINVAL, "context is NULL");
    if (!out_host) return fail(PFC_EINVAL, "out_host is NULL");
    pfc_status st = check_dev_ptr(c, u, "u");
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = diagnostics_launch(c, u, nullptr, s))) return st;
    PFC_CU(cudaMemcpyAsync(out_host, c->dout, sizeof(double) * 5, cudaMemcpyDeviceToHost, s));
    PFC_CU(cudaStreamSynchronize(s));
    return PFC_OK;
}

extern "C" pfc_status pfc_diagnostics_dev(pfc_ctx* c, const void* u, double* out_dev, pfc_stream stream)
{
    NvtxRange nvtx_("pfc_diagnostics_dev");
    if (!c) return fail(PFC_EINVAL, "context is NULL");
    pfc_status st = check_dev_ptr(c, u, "u");
    if (st) return st;
    if (!out_dev || !on_device(out_dev, c->device))
        return fail(PFC_EINVAL, "out_dev is not device memory of the context's device");
    return diagnostics_launch(c, u, out_dev, (cudaStream_t)stream);
}

extern "C" pfc_status pfc_surface_cells(pfc_ctx* c, const void* u, double level, void* cells, int64_t cap,
                                        int64_t* count_host, pfc_stream stream)
{
    NvtxRange nvtx_("pfc_surface_cells");
    if (!c) return fail(PFC_EINVAL, "context is NULL");
    if (!count_host) return fail(PFC_EINVAL, "count_host is NULL");
    if (!isfinite(level)) return fail(PFC_EINVAL, "level is not finite");
    if (cap < 0) return fail(PFC_EINVAL, "cap must be >= 0");
    pfc_status st = check_dev_ptr(c, u, "u");
    if (st) return st;
    if (cap > 0 && (st = check_dev_ptr(c, cells, "cells"))) return st;
    const long nb = surface_blocks(c->N);
    if (!c->skap) {
        PFC_CU(cudaMalloc(&c->skap, (size_t)c->esz * 2 * c->N));
        PFC_CU(cudaMalloc((void**)&c->sblk, sizeof(unsigned) * (size_t)nb));
        PFC_CU(cudaMalloc((void**)&c->soff, sizeof(long long) * (size_t)(nb + 1)));
    }
    cudaStream_t s = (cudaStream_t)stream;
    const pfc_problem& P = c->P;
    if (P.prec == PFC_FP64) {
        double* k1 = (double*)c->skap;
        double* k2 = k1 + c->N;
        PFC_CU(launch_curvatures<double>((const double*)u, k1, k2, P.nx, P.ny, P.nz,
                                         make_coef<double>(P.a, P.h, P.eps, P.xi, P.well, 0.0, nullptr, P.proj), P.eps, s));
        PFC_CU(launch_surface_cells<double>((const double*)u, k1, k2, P.nx, P.ny, P.nz, P.h, level, c->sblk, c->soff,
                                            (double*)cells, cap, s));
    } else {
        float* k1 = (float*)c->skap;
        float* k2 = k1 + c->N;
        PFC_CU(launch_curvatures<float>((const float*)u, k1, k2, P.nx, P.ny, P.nz,
                                        make_coef<float>(P.a, P.h, P.eps, P.xi, P.well, 0.0, nullptr, P.proj), P.eps, s));
        PFC_CU(launch_surface_cells<float>((const float*)u, k1, k2, P.nx, P.ny, P.nz, P.h, level, c->sblk, c->soff,
                                           (float*)cells, cap, s));
    }
    long long total = 0;
    PFC_CU(cudaMemcpyAsync(&total, c->soff + nb, sizeof total, cudaMemcpyDeviceToHost, s));
    PFC_CU(cudaStreamSynchronize(s));
    *count_host = (int64_t)total;
    return PFC_OK;
}

extern "C" pfc_status pfc_curvature_histogram(pfc_ctx* c, const void* cells, int64_t n, int32_t nbins, double lo,
                                              double hi, double* hist_dev, pfc_stream stream)
{
    if (!c) return fail(PFC_EINVAL, "context is NULL");
    if (n < 0 || nbins < 1 || !(hi > lo) || !isfinite(lo) || !isfinite(hi))
        return fail(PFC_EINVAL, "need n >= 0, nbins >= 1 and finite lo < hi");
    pfc_status st = check_dev_ptr(c, hist_dev, "hist_dev");
    if (st) return st;
    if (n > 0 && (st = check_dev_ptr(c, cells, "cells"))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (c->P.prec == PFC_FP64)
        PFC_CU(launch_curvature_histogram<double>((const double*)cells, n, nbins, lo, hi, hist_dev, s));
    else
        PFC_CU(launch_curvature_histogram<float>((const float*)cells, n, nbins, lo, hi, hist_dev, s));
    return PFC_OK;
}

// ------------------------------------------------------------ z-slab

// One z-slab of a periodic grid split across processes (one per GPU): the
// slab's planes, a caller-owned halo of the two planes beyond each end
// (filled from the neighbouring slabs before every sweep), and the scalars
// combined from every slab's FP64 sums.
struct pfc_slab {
    pfc_problem P;          // the whole grid
    int z0 = 0, nzl = 0;    // global index of the first plane, planes held
    int device = 0;
    int tile_y = 16;
    long long N = 0;        // voxels of the whole grid
    int nblocks = 0;        // partial slots of one sweep
    double* mem = nullptr;  // partials, then scalars, then counters
    double* partials = nullptr;
    double* scal = nullptr;
    unsigned* ints = nullptr;
    int last_mode = -1;     // mode of the last sweep: what pfc_slab_finish combines
};

extern "C" pfc_status pfc_slab_create(const pfc_problem* prob, int32_t z0, int32_t nz_local, pfc_slab** out)
{
    if (!out) return fail(PFC_EINVAL, "out is NULL");
    *out = nullptr;
    pfc_status st = check_problem(prob);
    if (st) return st;
    if (prob->impl != PFC_IMPL_FUSED) return fail(PFC_EUNSUPPORTED, "z-slabs run on the fused path only");
    if (nz_local < 2 || z0 < 0 || (long long)z0 + nz_local > prob->nz)
        return fail(PFC_EINVAL, "slab [%d, %d + %d) must hold >= 2 planes inside 0..nz = %d", z0, z0, nz_local, prob->nz);
    pfc_slab* sl = new (std::nothrow) pfc_slab();
    if (!sl) return fail(PFC_ENOMEM, "host allocation failed");
    sl->P = *prob;
    sl->z0 = z0;
    sl->nzl = nz_local;
    sl->N = (long long)prob->nx * prob->ny * prob->nz;
    if (cudaGetDevice(&sl->device) != cudaSuccess) {
        (void)cudaGetLastError();
        delete sl;
        return fail(PFC_ECUDA, "cudaGetDevice failed");
    }
    pfc_problem local = *prob;
    local.nz = nz_local;
    int zc, tx, ty, cz;
    geometry(&local, device_sms(), &sl->tile_y, &zc, &tx, &ty, &cz);
    sl->nblocks = (int)fused_slots(prob->nx, prob->ny, nz_local, sl->tile_y, prob->tile_z);
    const size_t bytes = sizeof(double) * ((size_t)NPART * sl->nblocks + NSCAL) + sizeof(unsigned) * NINTS;
    if (cudaMalloc((void**)&sl->mem, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        delete sl;
        return fail(PFC_ENOMEM, "device allocation of %zu bytes failed", bytes);
    }
    sl->partials = sl->mem;
    sl->scal = sl->mem + (size_t)NPART * sl->nblocks;
    sl->ints = reinterpret_cast<unsigned*>(sl->scal + NSCAL);
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMemsetAsync(sl->scal, 0, sizeof(double) * NSCAL + sizeof(unsigned) * NINTS, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        if (s) cudaStreamDestroy(s);
        cudaFree(sl->mem);
        delete sl;
        return fail(PFC_ECUDA, "clearing the slab's scalars failed: %s", cudaGetErrorString(e));
    }
    cudaStreamDestroy(s);
    *out = sl;
    return PFC_OK;
}

extern "C" void pfc_slab_destroy(pfc_slab* sl)
{
    if (!sl) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(sl->device);
    cudaDeviceSynchronize();
    cudaFree(sl->mem);
    cudaSetDevice(prev);
    delete sl;
}

template <typename T>
static Inst<T> slab_inst(const pfc_slab* sl, const void* u, const void* halo, void* out, double tau, double* sums)
{
    Inst<T> in{};
    const pfc_problem& P = sl->P;
    in.u = (const T*)u;
    in.out = (T*)out;
    in.nx = P.nx; in.ny = P.ny; in.nz = sl->nzl;
    in.vec = (P.nx % (16 / (int)sizeof(T)) == 0) && ((uintptr_t)u) % 16 == 0 && ((uintptr_t)halo) % 16 == 0;
    in.nblocks = sl->nblocks;
    in.C = make_coef<T>(P.a, P.h, P.eps, P.xi, P.well, P.mu, P.theta, P.proj, refine_of(P));
    in.tau = (T)tau;
    in.inv_N = 1.0 / (double)sl->N;
    in.partials = sl->partials;
    in.ints = sl->ints;
    in.scal = sl->scal;
    in.halo = (const T*)halo;
    in.sums_out = sums;
    return in;
}

extern "C" pfc_status pfc_slab_sweep(pfc_slab* sl, const void* u, const void* halo, void* out, int32_t mode,
                                     double tau, double* sums_dev, pfc_stream stream)
{
    NvtxRange nvtx_("pfc_slab_sweep");
    if (!sl) return fail(PFC_EINVAL, "slab is NULL");
    if (mode != MODE_ENERGY && mode != MODE_GRAD && mode != MODE_STEP) return fail(PFC_EINVAL, "unknown mode %d", mode);
    if (!on_device(u, sl->device) || !on_device(halo, sl->device) || !on_device(sums_dev, sl->device))
        return fail(PFC_EINVAL, "u, halo and sums_dev must be device memory of the slab's (current) device");
    if (mode != MODE_ENERGY) {
        if (!on_device(out, sl->device)) return fail(PFC_EINVAL, "out must be device memory of the slab's device");
        if (out == u || out == halo) return fail(PFC_EINVAL, "out must not alias u or halo");
    }
    if (!isfinite(tau)) return fail(PFC_EINVAL, "tau is not finite");
    cudaStream_t s = (cudaStream_t)stream;
    if (sl->P.prec == PFC_FP64)
        PFC_CU(launch_fused<double>(slab_inst<double>(sl, u, halo, out, tau, sums_dev), mode, sl->tile_y,
                                    sl->P.tile_z, s));
    else
        PFC_CU(launch_fused<float>(slab_inst<float>(sl, u, halo, out, tau, sums_dev), mode, sl->tile_y,
                                   sl->P.tile_z, s));
    sl->last_mode = mode;
    return PFC_OK;
}

extern "C" pfc_status pfc_slab_finish(pfc_slab* sl, const double* sums_all_dev, int32_t nslabs, double* scalars_dev,
                                      pfc_stream stream)
{
    NvtxRange nvtx_("pfc_slab_finish");
    if (!sl) return fail(PFC_EINVAL, "slab is NULL");
    if (sl->last_mode < 0) return fail(PFC_EINVAL, "no sweep to finish");
    if (nslabs < 1) return fail(PFC_EINVAL, "nslabs must be >= 1");
    if (!on_device(sums_all_dev, sl->device)) return fail(PFC_EINVAL, "sums_all_dev must be device memory of the slab's device");
    if (scalars_dev && !on_device(scalars_dev, sl->device))
        return fail(PFC_EINVAL, "scalars_dev must be device memory of the slab's device");
    PFC_CU(launch_slab_finish(sums_all_dev, nslabs, 1.0 / (double)sl->N, sl->last_mode, sl->scal, sl->ints,
                              scalars_dev, (cudaStream_t)stream));
    return PFC_OK;
}

extern "C" pfc_status pfc_slab_apply_offset(pfc_slab* sl, void* u, pfc_stream stream)
{
    if (!sl) return fail(PFC_EINVAL, "slab is NULL");
    if (!on_device(u, sl->device)) return fail(PFC_EINVAL, "u must be device memory of the slab's (current) device");
    cudaStream_t s = (cudaStream_t)stream;
    const long n = (long)sl->P.nx * sl->P.ny * sl->nzl;
    if (sl->P.prec == PFC_FP64)
        PFC_CU(launch_add_offset<double>((double*)u, (const double*)u, n, sl->scal + S_C, s));
    else
        PFC_CU(launch_add_offset<float>((float*)u, (const float*)u, n, sl->scal + S_C, s));
    // the chain is closed: no pending offset, and the next step takes its input's mass as the target
    PFC_CU(cudaMemsetAsync(sl->scal + S_C, 0, sizeof(double), s));
    PFC_CU(cudaMemsetAsync(sl->ints + I_COUNTER, 0, sizeof(unsigned), s));
    return PFC_OK;
}

// ------------------------------------------------------------ batch

struct pfc_batch {
    int n = 0;
    int device = 0;
    int tile_y = 16;
    int max_run = 0;
    int total_blocks = 0;
    std::vector<pfc_problem> P;
    std::vector<Inst<float>> host;   // geometry + scratch pointers, u/out filled per run
    std::vector<void*> ping;
    double* partials = nullptr;
    unsigned* ints = nullptr;
    double* scal = nullptr;
    double* trace = nullptr;
    int trace_cap = 0;
    cudaGraphExec_t gexec = nullptr;   // cached step loop, keyed by fields, steps and G
    std::vector<void*> g_u;
    std::vector<double> g_tau;
    int g_len = 0;
    double* g_trace = nullptr;
    cudaStream_t cap = nullptr;
    cudaEvent_t ev[4] = { nullptr, nullptr, nullptr, nullptr };
    bool timing = false;
    int lazy = 0;   // a chain of pfc_batch_step_lazy is open (offsets pending in scal)
    // pfc_batch_step_host: device staging and the copy pipeline
    std::vector<void*> hin;
    cudaStream_t hs[2] = { nullptr, nullptr };    // host-to-device, device-to-host
    // per instance: copied in, stepped (staging input free), result ready, copied out (result buffer free)
    std::vector<cudaEvent_t> evin, evstep, evres, evdone;
};

static void free_batch_mem(pfc_batch* b)
{
    for (void* p : b->ping) cudaFree(p);
    cudaFree(b->partials);
    cudaFree(b->scal);       // also holds the counters (b->ints)
    cudaFree(b->trace);
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    for (void* p : b->hin) cudaFree(p);
    for (cudaStream_t s : b->hs)
        if (s) cudaStreamDestroy(s);
    for (auto* v : { &b->evin, &b->evstep, &b->evres, &b->evdone })
        for (cudaEvent_t e : *v)
            if (e) cudaEventDestroy(e);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->cap) cudaStreamDestroy(b->cap);
}

extern "C" pfc_status pfc_batch_create(const pfc_problem* probs, int32_t n, pfc_batch** out)
{
    if (!out) return fail(PFC_EINVAL, "out is NULL");
    *out = nullptr;
    if (!probs || n < 1) return fail(PFC_EINVAL, "need at least one problem");
    for (int k = 0; k < n; ++k) {
        pfc_status st = check_problem(&probs[k]);
        if (st) return fail(st, "problem %d: %s", k, g_err);
        if (probs[k].prec != PFC_FP32 || probs[k].impl != PFC_IMPL_FUSED)
            return fail(PFC_EUNSUPPORTED, "problem %d: batches run FP32 on the fused path only", k);
        if (probs[k].mu != 0.0 || probs[k].proj)
            return fail(PFC_EUNSUPPORTED, "problem %d: the orientation term and the projected M are not available "
                        "in batches", k);
    }
    pfc_batch* b = new (std::nothrow) pfc_batch();
    if (!b) return fail(PFC_ENOMEM, "host allocation failed");
    b->n = n;
    b->P.assign(probs, probs + n);
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        (void)cudaGetLastError();
        return fail(PFC_ECUDA, "cudaGetDevice failed");
    }
    const int sms = device_sms();
    b->host.resize(n);
    b->ping.assign(n, nullptr);
    bool ok = true;
    b->tile_y = probs[0].tile_y ? probs[0].tile_y : auto_tile_y(probs, n);   // one height for all instances
    b->max_run = probs[0].tile_z;
    long long units = 0;
    for (int k = 0; k < n && ok; ++k) {
        pfc_problem p = probs[k];
        p.tile_y = b->tile_y;
        int ty, zc, tx, tyn, cz;
        geometry(&p, sms, &ty, &zc, &tx, &tyn, &cz);
        Inst<float>& in = b->host[k];
        in = Inst<float>{};
        in.nx = p.nx; in.ny = p.ny; in.nz = p.nz;
        in.zc = zc;
        in.tiles_x = tx; in.tiles_y = tyn; in.chunks_z = cz;
        units += (long long)tx * tyn * p.nz;
        in.C = make_coef<float>(p.a, p.h, p.eps, p.xi, p.well, 0.0, nullptr, 0, refine_of(p));
        in.inv_N = 1.0 / ((double)p.nx * p.ny * p.nz);
        ok = cudaMalloc(&b->ping[k], sizeof(float) * (size_t)p.nx * p.ny * p.nz) == cudaSuccess;
    }
    // every problem may get a partial from every CTA of its launch
    const long long slots = fused_grid(units, b->max_run);
    b->total_blocks = (int)slots;
    // the problems' scalars and counters in one block, cleared by one memset per step
    ok = ok && cudaMalloc((void**)&b->partials, sizeof(double) * NPART * (size_t)slots * n) == cudaSuccess &&
         cudaMalloc((void**)&b->scal, sizeof(double) * NSCAL * (size_t)n + sizeof(unsigned) * NINTS * (size_t)n) ==
             cudaSuccess &&
         cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) b->ints = reinterpret_cast<unsigned*>(b->scal + (size_t)NSCAL * n);
    if (!ok) {
        cudaError_t le = cudaGetLastError();
        free_batch_mem(b);
        delete b;
        return fail(PFC_ENOMEM, "device allocation failed: %s", cudaGetErrorString(le));
    }
    for (int k = 0; k < n; ++k) {
        Inst<float>& in = b->host[k];
        in.partials = b->partials + (size_t)k * slots * NPART;
        in.ints = b->ints + (size_t)k * NINTS;
        in.scal = b->scal + (size_t)k * NSCAL;
    }
    *out = b;
    return PFC_OK;
}

extern "C" void pfc_batch_destroy(pfc_batch* b)
{
    if (!b) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    free_batch_mem(b);
    cudaSetDevice(prev);
    delete b;
}

extern "C" pfc_status pfc_batch_run(pfc_batch* b, void* const* u, int32_t nsteps, const double* tau,
                                    double* trace_host, pfc_stream stream)
{
    NvtxRange nvtx_("pfc_batch_run");
    if (!b) return fail(PFC_EINVAL, "batch is NULL");
    if (!u || !tau) return fail(PFC_EINVAL, "u and tau arrays are required");
    if (nsteps < 0) return fail(PFC_EINVAL, "nsteps must be >= 0");
    for (int k = 0; k < b->n; ++k) {
        if (!u[k]) return fail(PFC_EINVAL, "u[%d] is NULL", k);
        if (!on_device(u[k], b->device)) return fail(PFC_EINVAL, "u[%d] is not device memory of the batch's device", k);
        if (!isfinite(tau[k])) return fail(PFC_EINVAL, "tau[%d] is not finite", k);
    }
    if (nsteps == 0) return PFC_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (nsteps > b->trace_cap) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        PFC_CU(cudaStreamSynchronize(s));   // not device-wide: see ensure_trace
        cudaFree(b->trace);
        b->trace = nullptr;
        b->trace_cap = 0;
        PFC_CU(cudaMalloc((void**)&b->trace, sizeof(double) * 5 * (size_t)nsteps * b->n));
        b->trace_cap = nsteps;
    }
    // per-instance descriptors for the two step parities
    std::vector<Inst<float>> ev(b->host), od(b->host);
    for (int k = 0; k < b->n; ++k) {
        ev[k].u = (const float*)u[k];
        ev[k].out = (float*)b->ping[k];
        od[k].u = (const float*)b->ping[k];
        od[k].out = (float*)u[k];
        const bool aligned = ((uintptr_t)u[k]) % 16 == 0;
        ev[k].vec = (b->P[k].nx % 4 == 0) && aligned;
        od[k].vec = (b->P[k].nx % 4 == 0);
        ev[k].tau = od[k].tau = (float)tau[k];
        ev[k].trace = od[k].trace = b->trace + (size_t)k * 5 * b->trace_cap;
        ev[k].trace_cap = od[k].trace_cap = b->trace_cap;
    }
    b->lazy = 0;
    PFC_CU(cudaMemsetAsync(b->scal, 0, (sizeof(double) * NSCAL + sizeof(unsigned) * NINTS) * b->n, s));
    // The loop runs in chunks of G steps.  After each chunk the host reads
    // the instances' flags, and the instances whose scalars became non-finite
    // leave the launches: the persistent schedule splits a launch's units
    // evenly over the CTAs, so a retired instance left in it (its runs only
    // store NaN) would leave its CTAs idle while the others work.  A dropped
    // instance's two field buffers are filled with NaN, its later trace rows
    // too.  A chunk runs from a CUDA graph of G launches when one was
    // captured for the same instances; otherwise it is launched directly and
    // the graph is captured while the GPU runs it, for the chunks after.
    std::vector<int> live;
    for (int k = 0; k < b->n; ++k) live.push_back(k);
    std::vector<int> dropped_at(b->n, -1);
    std::vector<Inst<float>> evl(ev), odl(od);
    auto steps = [&](int i0, int cnt, cudaStream_t st) -> cudaError_t {
        if (live.empty()) return cudaSuccess;
        for (int i = i0; i < i0 + cnt; ++i) {
            cudaError_t e = launch_fused_batch((i % 2) == 0 ? evl.data() : odl.data(), (int)live.size(), b->tile_y,
                                               b->max_run, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    constexpr int kChunk = 16;
    const int G = nsteps >= kChunk ? kChunk : (nsteps & ~1);
    std::vector<unsigned> ints((size_t)NINTS * b->n);
    int done = 0;
    if (G >= 2) {
        const std::vector<double> tkey(tau, tau + b->n);
        while (!live.empty() && done + G <= nsteps) {
            // the descriptors are kernel parameters: a graph holds the
            // fields, the step sizes and the instances still advanced
            std::vector<void*> key(u, u + b->n);
            for (int k = 0; k < b->n; ++k)
                if (dropped_at[k] >= 0) key[k] = nullptr;
            if (b->gexec && b->g_len == G && b->g_trace == b->trace && b->g_u == key && b->g_tau == tkey) {
                PFC_CU(cudaGraphLaunch(b->gexec, s));
            } else {
                PFC_CU(steps(done, G, s));
                if (b->gexec) {
                    cudaGraphExecDestroy(b->gexec);
                    b->gexec = nullptr;
                }
                cudaGraph_t graph = nullptr;
                PFC_CU(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
                cudaError_t e = steps(0, G, b->cap);
                cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
                if (e != cudaSuccess || e2 != cudaSuccess) {
                    if (graph) cudaGraphDestroy(graph);
                    (void)cudaGetLastError();
                    return fail(PFC_ECUDA, "graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
                }
                e = cudaGraphInstantiate(&b->gexec, graph, 0);
                cudaGraphDestroy(graph);
                if (e != cudaSuccess) {
                    b->gexec = nullptr;
                    (void)cudaGetLastError();
                    return fail(PFC_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
                }
                b->g_len = G;
                b->g_trace = b->trace;
                b->g_u = key;
                b->g_tau = tkey;
            }
            done += G;
            if (done >= nsteps) break;
            PFC_CU(cudaMemcpyAsync(ints.data(), b->ints, sizeof(unsigned) * ints.size(), cudaMemcpyDeviceToHost, s));
            PFC_CU(cudaStreamSynchronize(s));
            std::vector<int> keep;
            for (int k : live) {
                if (ints[(size_t)k * NINTS + I_NONFINITE] == 0) {
                    keep.push_back(k);
                    continue;
                }
                dropped_at[k] = done;
                const size_t bytes = sizeof(float) * (size_t)b->P[k].nx * b->P[k].ny * b->P[k].nz;
                PFC_CU(cudaMemsetAsync(u[k], 0xff, bytes, s));   // all-ones words: NaN
                PFC_CU(cudaMemsetAsync(b->ping[k], 0xff, bytes, s));
            }
            if (keep.size() != live.size()) {
                live.swap(keep);
                evl.clear();
                odl.clear();
                for (int k : live) {
                    evl.push_back(ev[k]);
                    odl.push_back(od[k]);
                }
            }
        }
    }
    PFC_CU(steps(done, nsteps - done, s));
    const bool in_ping = (nsteps % 2) == 1;
    for (int k = 0; k < b->n; ++k) {
        const long N = (long)b->P[k].nx * b->P[k].ny * b->P[k].nz;
        PFC_CU(launch_add_offset<float>((float*)u[k], (const float*)(in_ping ? b->ping[k] : u[k]), N,
                                        b->scal + (size_t)k * NSCAL + S_C, s));
    }
    PFC_CU(cudaMemcpyAsync(ints.data(), b->ints, sizeof(unsigned) * ints.size(), cudaMemcpyDeviceToHost, s));
    if (trace_host)
        for (int k = 0; k < b->n; ++k)
            PFC_CU(cudaMemcpyAsync(trace_host + (size_t)k * 5 * nsteps, b->trace + (size_t)k * 5 * b->trace_cap,
                                   sizeof(double) * 5 * (size_t)nsteps, cudaMemcpyDeviceToHost, s));
    PFC_CU(cudaStreamSynchronize(s));
    if (trace_host)
        for (int k = 0; k < b->n; ++k)
            if (dropped_at[k] >= 0)
                for (size_t i = (size_t)dropped_at[k] * 5; i < (size_t)nsteps * 5; ++i)
                    trace_host[(size_t)k * 5 * nsteps + i] = NAN;
    int bad = 0;
    for (int k = 0; k < b->n; ++k) {
        const unsigned want = dropped_at[k] >= 0 ? (unsigned)dropped_at[k] : (unsigned)nsteps;
        if (ints[(size_t)k * NINTS + I_COUNTER] != want)
            return fail(PFC_ECUDA, "instance %d: step counter %u != %u", k, ints[(size_t)k * NINTS + I_COUNTER], want);
        bad += ints[(size_t)k * NINTS + I_NONFINITE] != 0;
    }
    if (bad) return fail(PFC_ENONFINITE, "%d instance(s) produced non-finite scalars", bad);
    return PFC_OK;
}

// The launch descriptors of one step of every instance from u_in to u_out
// (device fields, not aliased, finite step sizes).
static pfc_status step_descriptors(const pfc_batch* b, const void* const* u_in, void* const* u_out,
                                   const double* tau, std::vector<Inst<float>>& d)
{
    d = b->host;
    for (int k = 0; k < b->n; ++k) {
        for (int w = 0; w < 2; ++w) {
            const void* p = w ? (const void*)u_out[k] : u_in[k];
            if (!on_device(p, b->device))
                return fail(PFC_EINVAL, "%s[%d] is not device memory of the batch's device", w ? "u_out" : "u_in", k);
        }
        if (u_in[k] == u_out[k]) return fail(PFC_EINVAL, "u_out[%d] aliases u_in[%d]", k, k);
        if (!isfinite(tau[k])) return fail(PFC_EINVAL, "tau[%d] is not finite", k);
        d[k].u = (const float*)u_in[k];
        d[k].out = (float*)u_out[k];
        d[k].vec = (b->P[k].nx % 4 == 0) && ((uintptr_t)u_in[k]) % 16 == 0;
        d[k].tau = (float)tau[k];
        d[k].trace = nullptr;
        d[k].trace_cap = 0;
    }
    return PFC_OK;
}

extern "C" pfc_status pfc_batch_step(pfc_batch* b, const void* const* u_in, void* const* u_out, const double* tau,
                                     double* scalars_dev, pfc_stream stream)
{
    NvtxRange nvtx_("pfc_batch_step");
    if (!b) return fail(PFC_EINVAL, "batch is NULL");
    if (!u_in || !u_out || !tau) return fail(PFC_EINVAL, "u_in, u_out and tau arrays are required");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<Inst<float>> d;
    if (pfc_status st = step_descriptors(b, u_in, u_out, tau, d); st != PFC_OK) return st;
    b->lazy = 0;   // the scalars are reset: an open chain of lazy steps ends here
    if (b->timing) PFC_CU(cudaEventRecord(b->ev[0], s));
    PFC_CU(cudaMemsetAsync(b->scal, 0, (sizeof(double) * NSCAL + sizeof(unsigned) * NINTS) * b->n, s));
    if (b->timing) PFC_CU(cudaEventRecord(b->ev[1], s));
    PFC_CU(launch_fused_batch(d.data(), b->n, b->tile_y, b->max_run, s));
    if (b->timing) PFC_CU(cudaEventRecord(b->ev[2], s));
    PFC_CU(launch_add_offset_batch(d.data(), b->n, s));
    if (scalars_dev)
        PFC_CU(cudaMemcpy2DAsync(scalars_dev, 5 * sizeof(double), b->scal, NSCAL * sizeof(double), 5 * sizeof(double),
                                 b->n, cudaMemcpyDeviceToDevice, s));
    if (b->timing) PFC_CU(cudaEventRecord(b->ev[3], s));
    return PFC_OK;
}

// Chained steps in the fused form of the mass projection: the step stores
// v = (u_in + c) - tau g with the pending offset c of the previous chained
// step added as the sweep loads u_in, and leaves the new offset
// c' = target - mean(v) (FP64, from the CTAs' partials) in the instance's
// scalar slot for the next step; pfc_batch_lazy_finish adds it.  The target
// mass is the mean of the first step's input.
extern "C" pfc_status pfc_batch_step_lazy(pfc_batch* b, const void* const* u_in, void* const* u_out,
                                          const double* tau, int32_t first, pfc_stream stream)
{
    NvtxRange nvtx_("pfc_batch_step_lazy");
    if (!b) return fail(PFC_EINVAL, "batch is NULL");
    if (!u_in || !u_out || !tau) return fail(PFC_EINVAL, "u_in, u_out and tau arrays are required");
    if (!first && !b->lazy) return fail(PFC_EINVAL, "no chain of lazy steps is open: start one with first = 1");
    // opening a chain resets the offsets: the open chain's last output would lose its projection
    if (first && b->lazy) return fail(PFC_EINVAL, "a chain of lazy steps is open: close it with pfc_batch_lazy_finish");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<Inst<float>> d;
    if (pfc_status st = step_descriptors(b, u_in, u_out, tau, d); st != PFC_OK) return st;
    if (b->timing) PFC_CU(cudaEventRecord(b->ev[0], s));
    if (first) PFC_CU(cudaMemsetAsync(b->scal, 0, (sizeof(double) * NSCAL + sizeof(unsigned) * NINTS) * b->n, s));
    if (b->timing) PFC_CU(cudaEventRecord(b->ev[1], s));
    PFC_CU(launch_fused_batch(d.data(), b->n, b->tile_y, b->max_run, s));
    if (b->timing) {
        PFC_CU(cudaEventRecord(b->ev[2], s));
        PFC_CU(cudaEventRecord(b->ev[3], s));
    }
    b->lazy = 1;
    return PFC_OK;
}

extern "C" pfc_status pfc_batch_lazy_finish(pfc_batch* b, void* const* u, pfc_stream stream)
{
    NvtxRange nvtx_("pfc_batch_lazy_finish");
    if (!b) return fail(PFC_EINVAL, "batch is NULL");
    if (!u) return fail(PFC_EINVAL, "u array is required");
    if (!b->lazy) return fail(PFC_EINVAL, "no chain of lazy steps is open");
    std::vector<Inst<float>> d(b->host);
    for (int k = 0; k < b->n; ++k) {
        if (!on_device(u[k], b->device)) return fail(PFC_EINVAL, "u[%d] is not device memory of the batch's device", k);
        d[k].out = (float*)u[k];
    }
    PFC_CU(launch_add_offset_batch(d.data(), b->n, (cudaStream_t)stream));
    b->lazy = 0;
    return PFC_OK;
}

// One step of every instance from and to host memory, pipelined per
// instance over three streams: copies in on hs[0], the steps on `stream`,
// copies out on hs[1].  Nothing waits for the host: the copy of instance k
// into its staging buffer waits only until the previous step of k has read
// it, and the step of k only until the previous copy out of k has left its
// result buffer, so consecutive calls overlap (the copies out of one step
// with the copies in of the next).
extern "C" pfc_status pfc_batch_step_host(pfc_batch* b, const void* const* u_in_host, void* const* u_out_host,
                                          const double* tau, pfc_stream stream)
{
    NvtxRange nvtx_("pfc_batch_step_host");
    if (!b) return fail(PFC_EINVAL, "batch is NULL");
    if (!u_in_host || !u_out_host || !tau) return fail(PFC_EINVAL, "u_in_host, u_out_host and tau arrays are required");
    for (int k = 0; k < b->n; ++k) {
        if (!u_in_host[k] || !u_out_host[k]) return fail(PFC_EINVAL, "host buffer %d is NULL", k);
        if (u_in_host[k] == u_out_host[k]) return fail(PFC_EINVAL, "u_out_host[%d] aliases u_in_host[%d]", k, k);
        if (!isfinite(tau[k])) return fail(PFC_EINVAL, "tau[%d] is not finite", k);
        for (int w = 0; w < 2; ++w) {
            cudaPointerAttributes at;
            const void* p = w ? (const void*)u_out_host[k] : u_in_host[k];
            if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
                (void)cudaGetLastError();
                continue;                        // plain pageable memory: allowed, the copies then block
            }
            if (at.type == cudaMemoryTypeDevice) return fail(PFC_EINVAL, "buffer %d is device memory", k);
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (b->hin.empty()) {
        b->hin.assign(b->n, nullptr);
        for (auto* v : { &b->evin, &b->evstep, &b->evres, &b->evdone }) v->assign(b->n, nullptr);
        for (int k = 0; k < b->n; ++k) {
            const size_t bytes = sizeof(float) * (size_t)b->P[k].nx * b->P[k].ny * b->P[k].nz;
            PFC_CU(cudaMalloc(&b->hin[k], bytes));
            for (auto* v : { &b->evin, &b->evstep, &b->evres, &b->evdone })
                PFC_CU(cudaEventCreateWithFlags(&(*v)[k], cudaEventDisableTiming));
        }
        for (cudaStream_t& hs : b->hs) PFC_CU(cudaStreamCreateWithFlags(&hs, cudaStreamNonBlocking));
        // first use: the copy streams start after everything already on `stream`
        for (int k = 0; k < b->n; ++k) {
            PFC_CU(cudaEventRecord(b->evstep[k], s));
            PFC_CU(cudaEventRecord(b->evdone[k], s));
        }
    }
    b->lazy = 0;
    PFC_CU(cudaMemsetAsync(b->scal, 0, (sizeof(double) * NSCAL + sizeof(unsigned) * NINTS) * b->n, s));
    for (int k = 0; k < b->n; ++k) {
        const long N = (long)b->P[k].nx * b->P[k].ny * b->P[k].nz;
        PFC_CU(cudaStreamWaitEvent(b->hs[0], b->evstep[k], 0));
        PFC_CU(cudaMemcpyAsync(b->hin[k], u_in_host[k], sizeof(float) * N, cudaMemcpyHostToDevice, b->hs[0]));
        PFC_CU(cudaEventRecord(b->evin[k], b->hs[0]));
        PFC_CU(cudaStreamWaitEvent(s, b->evin[k], 0));
        PFC_CU(cudaStreamWaitEvent(s, b->evdone[k], 0));
        Inst<float> in = b->host[k];
        in.u = (const float*)b->hin[k];
        in.out = (float*)b->ping[k];
        in.vec = b->P[k].nx % 4 == 0;
        in.tau = (float)tau[k];
        in.trace = nullptr;
        in.trace_cap = 0;
        PFC_CU(launch_fused<float>(in, MODE_STEP, b->tile_y, b->max_run, s));
        PFC_CU(cudaEventRecord(b->evstep[k], s));
        PFC_CU(launch_add_offset<float>((float*)b->ping[k], (const float*)b->ping[k], N, in.scal + S_C, s));
        PFC_CU(cudaEventRecord(b->evres[k], s));
        PFC_CU(cudaStreamWaitEvent(b->hs[1], b->evres[k], 0));
        PFC_CU(cudaMemcpyAsync(u_out_host[k], b->ping[k], sizeof(float) * N, cudaMemcpyDeviceToHost, b->hs[1]));
        PFC_CU(cudaEventRecord(b->evdone[k], b->hs[1]));
    }
    return PFC_OK;
}

extern "C" pfc_status pfc_batch_host_wait(pfc_batch* b, pfc_stream stream)
{
    if (!b) return fail(PFC_EINVAL, "batch is NULL");
    PFC_CU(cudaStreamSynchronize((cudaStream_t)stream));
    for (cudaStream_t hs : b->hs)
        if (hs) PFC_CU(cudaStreamSynchronize(hs));
    return PFC_OK;
}

extern "C" pfc_status pfc_batch_timing(pfc_batch* b, int enable)
{
    if (!b) return fail(PFC_EINVAL, "batch is NULL");
    if (enable && !b->ev[0])
        for (cudaEvent_t& e : b->ev) PFC_CU(cudaEventCreate(&e));
    b->timing = enable != 0;
    return PFC_OK;
}

extern "C" pfc_status pfc_batch_last_timing(pfc_batch* b, float* step_ms, float* sweep_ms)
{
    if (!b) return fail(PFC_EINVAL, "batch is NULL");
    if (!b->timing || !b->ev[0]) return fail(PFC_EINVAL, "timing is not enabled");
    PFC_CU(cudaEventSynchronize(b->ev[3]));
    float a = 0.f, c = 0.f;
    PFC_CU(cudaEventElapsedTime(&a, b->ev[0], b->ev[3]));
    PFC_CU(cudaEventElapsedTime(&c, b->ev[1], b->ev[2]));
    if (step_ms) *step_ms = a;
    if (sweep_ms) *sweep_ms = c;
    return PFC_OK;
}

// ------------------------------------------------------------ host helpers

extern "C" pfc_status pfc_b_to_a(const double b[7], double a[6])
{
    if (!b || !a) return fail(PFC_EINVAL, "b and a_out are required");
    // h2 (H - H0)^2 + k1 K + alpha (kappa1 - kappa1_0)^2 + beta (kappa2 - kappa2_0)^2
    const double h2 = b[0], H0 = b[1], kK = b[2], al = b[3], k10 = b[4], be = b[5], k20 = b[6];
    a[0] = h2 + al;
    a[1] = 2.0 * h2 + kK;
    a[2] = h2 + be;
    a[3] = -2.0 * (h2 * H0 + al * k10);
    a[4] = -2.0 * (h2 * H0 + be * k20);
    a[5] = h2 * H0 * H0 + al * k10 * k10 + be * k20 * k20;
    return PFC_OK;
}

extern "C" const char* pfc_status_string(pfc_status s)
{
    switch (s) {
    case PFC_OK: return "ok";
    case PFC_EINVAL: return "invalid argument";
    case PFC_ENOMEM: return "out of memory";
    case PFC_ECUDA: return "CUDA error";
    case PFC_ENONFINITE: return "non-finite result";
    case PFC_ETIMEOUT: return "device wait timed out";
    case PFC_EUNSUPPORTED: return "unsupported";
    default: return "unknown status";
    }
}

extern "C" const char* pfc_last_error(void) { return g_err; }
