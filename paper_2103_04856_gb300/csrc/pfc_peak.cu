// pfc_peak.cu -- pfc_measure_fp32_peak: the FP32 FMA throughput of the
// current device, measured with independent FMA chains and CUDA events.  It
// is the denominator of the fused sweep's arithmetic roofline (the sweep is
// bound by FP32 instruction issue, not by HBM).  Nothing is allocated: the
// kernel's one possible store goes to a file-scope device word.
#include <cuda_runtime.h>

#include "../../include/pfc.h"
#include "pfc_internal.h"

namespace pfc {
void set_last_error(const char* msg);
}

namespace {

constexpr int kChains = 8;        // independent FMA chains per thread
constexpr int kUnroll = 16;       // FMAs per chain per loop trip
constexpr int kThreads = 512;
constexpr int kBlocksPerSm = 4;   // 64 warps per SM: enough to hide FMA latency

__device__ float g_peak_sink;

// kChains x kUnroll dependent FMAs per trip; the sum is stored only if it
// equals an impossible value, so the chains stay live without a memory write.
__global__ void __launch_bounds__(kThreads) k_ffma_chains(int trips, float b, float c)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1234.5f) g_peak_sink = s;
}

}  // namespace

extern "C" pfc_status pfc_measure_fp32_peak(double* tflops_host, pfc_stream stream)
{
    if (!tflops_host) {
        pfc::set_last_error("tflops_host is NULL");
        return PFC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = kBlocksPerSm * pfc::device_sms();
    const int trips = 20000;
    const double flops = 2.0 * kChains * kUnroll * (double)trips * kThreads * blocks;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double best = 0.0;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // one warm-up launch, then the best of three timed ones
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) {
            k_ffma_chains<<<blocks, kThreads, 0, s>>>(trips, 0.9999f, 1e-7f);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms > 0.0f) {
            const double tf = flops / (ms * 1e-3) / 1e12;
            best = tf > best ? tf : best;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        pfc::set_last_error(cudaGetErrorString(e));
        return PFC_ECUDA;
    }
    *tflops_host = best;
    return PFC_OK;
}
