// pfc_noalloc.cu -- pfc_energy_and_grad_noalloc: the fused energy + gradient
// sweep for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc / cudaFree are off limits --
// inside a host callback or a region being captured into a CUDA graph (both
// implicitly synchronise or are not capturable), plugins hosted by a process
// whose memory manager owns the whole device budget, and real-time loops that
// must not take the driver's allocation lock or its implicit device-wide
// synchronisation.  Such callers pass their own input and output buffers;
// the only other device memory the sweep needs -- its per-CTA FP64 partial
// sums, the problem's scalars and the completion counters -- lives in the
// file-scope array below, which every GPU that loads this library holds
// until the process exits.
#include <cuda_runtime.h>

#include <math.h>
#include <mutex>

#include "../../include/pfc.h"
#include "pfc_internal.h"

using namespace pfc;

namespace {

// Partial sums for at most this many CTAs (the sweep uses one CTA per SM).
constexpr int kMaxCtas = 1024;
constexpr size_t kPartBytes = sizeof(double) * NPART * (size_t)kMaxCtas;
constexpr size_t kScalBytes = sizeof(double) * NSCAL;
constexpr size_t kIntsBytes = sizeof(unsigned) * NINTS;
constexpr size_t kScratchBytes = kPartBytes + kScalBytes + kIntsBytes;
static_assert(kScratchBytes == 49232, "the scratch size stated in include/pfc.h");

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};   // device address of the array, per device
std::mutex g_scratch_lock;

}  // namespace

// The scratch.  In host code this name is only a stand-in for the symbol:
// its device address comes from cudaGetSymbolAddress, per device.
static __device__ __align__(256) unsigned char g_pfc_noalloc_scratch[kScratchBytes];

namespace pfc {
void set_last_error(const char* msg);
}

static pfc_status na_fail(pfc_status s, const char* msg)
{
    pfc::set_last_error(msg);
    return s;
}

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does it, so that call must not be made
// while a stream is being captured).
static void* scratch_on_current_device(pfc_status* st)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        *st = na_fail(PFC_ECUDA, "noalloc: cudaGetDevice failed");
        return nullptr;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        *st = na_fail(PFC_EUNSUPPORTED, "noalloc: device ordinal beyond 63");
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_scratch_lock);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_pfc_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            *st = na_fail(PFC_ECUDA, "noalloc: cudaGetSymbolAddress of the scratch array failed");
            return nullptr;
        }
        g_scratch_addr[dev] = p;
    }
    *st = PFC_OK;
    return g_scratch_addr[dev];
}

// p is device (or managed) memory of the current device: the kernels run on
// the current device and must not touch another GPU's memory
static bool is_current_device_ptr(const void* p)
{
    cudaPointerAttributes at;
    int dev = -1;
    if (!p || cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

template <typename T>
static pfc_status run_noalloc(const pfc_problem* p, const void* u, void* g, double* E_host, cudaStream_t s,
                              unsigned char* base)
{
    Inst<T> in{};
    in.u = (const T*)u;
    in.out = (T*)g;
    in.nx = p->nx; in.ny = p->ny; in.nz = p->nz;
    const int tile_y = p->tile_y ? p->tile_y : default_tile_y(p->ny, sizeof(T) == 8);
    in.tiles_x = (p->nx + 31) / 32;
    in.tiles_y = (p->ny + tile_y - 1) / tile_y;
    in.zc = p->nz;
    in.chunks_z = 1;
    in.vec = (p->nx % (16 / (int)sizeof(T)) == 0) && ((uintptr_t)u) % 16 == 0;
    in.C = make_coef<T>(p->a, p->h, p->eps, p->xi, p->well, p->mu, p->theta, p->proj,
                      (p->flags & PFC_FLAG_NO_DISCRIMINANT_REFINEMENT) ? 0 : 1);
    in.cf = nullptr;
    in.tau = T(0);
    in.inv_N = 1.0 / ((double)p->nx * p->ny * p->nz);
    in.partials = (double*)base;
    in.scal = (double*)(base + kPartBytes);
    in.ints = (unsigned*)(base + kPartBytes + kScalBytes);
    in.trace = nullptr;
    in.trace_cap = 0;
    if (fused_slots(p->nx, p->ny, p->nz, tile_y, p->tile_z) > kMaxCtas)
        return na_fail(PFC_EINVAL, "noalloc: the launch would need more than 1024 CTAs of scratch "
                                   "(lower tile_z or use pfc_energy_and_grad)");
    // the counters must start at zero; everything else is written before it is read
    cudaError_t e = cudaMemsetAsync(in.ints, 0, kIntsBytes, s);
    if (e == cudaSuccess) e = launch_fused<T>(in, MODE_GRAD, tile_y, p->tile_z, s);
    if (e == cudaSuccess && E_host) {
        e = cudaMemcpyAsync(E_host, in.scal + S_E, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return na_fail(PFC_ECUDA, cudaGetErrorString(e));
    }
    if (E_host && !isfinite(*E_host)) return na_fail(PFC_ENONFINITE, "noalloc: energy is not finite");
    return PFC_OK;
}

extern "C" pfc_status pfc_energy_and_grad_noalloc(const pfc_problem* prob, const void* u, void* g, double* E_host,
                                                  pfc_stream stream)
{
    if (!prob) return na_fail(PFC_EINVAL, "noalloc: problem is NULL");
    const pfc_problem& p = *prob;
    if (p.nx < 1 || p.ny < 1 || p.nz < 1 || (double)p.nx * p.ny * p.nz > 2.0e9)
        return na_fail(PFC_EINVAL, "noalloc: grid sizes must be >= 1 and hold at most 2e9 voxels");
    if (!(p.h > 0) || !(p.eps > 0) || !(p.xi > 0) || !isfinite(p.h) || !isfinite(p.eps) || !isfinite(p.xi))
        return na_fail(PFC_EINVAL, "noalloc: h, eps and xi must be finite and > 0");
    for (int i = 0; i < 6; ++i)
        if (!isfinite(p.a[i])) return na_fail(PFC_EINVAL, "noalloc: a coefficient is not finite");
    if (!isfinite(p.mu) || !isfinite(p.theta[0]) || !isfinite(p.theta[1]) || !isfinite(p.theta[2]))
        return na_fail(PFC_EINVAL, "noalloc: mu and theta must be finite");
    if ((p.proj != 0 && p.proj != 1) || (p.flags & ~PFC_FLAG_NO_DISCRIMINANT_REFINEMENT))
        return na_fail(PFC_EINVAL, "noalloc: proj 0 or 1, unknown flags");
    if (p.well != PFC_WELL_01 && p.well != PFC_WELL_PM1) return na_fail(PFC_EINVAL, "noalloc: unknown double well");
    if (p.prec != PFC_FP32 && p.prec != PFC_FP64) return na_fail(PFC_EINVAL, "noalloc: unknown precision");
    if (p.impl != PFC_IMPL_FUSED) return na_fail(PFC_EUNSUPPORTED, "noalloc: only the fused path needs no allocation");
    if (p.tile_y != 0 && p.tile_y != 8 && p.tile_y != 13 && p.tile_y != 16) return na_fail(PFC_EINVAL, "noalloc: tile_y must be 0, 8, 13 or 16");
    if (p.tile_z < 0) return na_fail(PFC_EINVAL, "noalloc: tile_z must be >= 0");
    if (!is_current_device_ptr(u) || !is_current_device_ptr(g))
        return na_fail(PFC_EINVAL, "noalloc: u and g must be device memory of the current device");
    if (u == g) return na_fail(PFC_EINVAL, "noalloc: g must not alias u");
    pfc_status st;
    unsigned char* base = (unsigned char*)scratch_on_current_device(&st);
    if (!base) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (p.prec == PFC_FP64) return run_noalloc<double>(&p, u, g, E_host, s, base);
    return run_noalloc<float>(&p, u, g, E_host, s, base);
}
