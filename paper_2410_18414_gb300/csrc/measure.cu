// pic_measure_fp64_fma: the FP64 fused multiply-add rate of the current device, measured
// (a measurement aid; the paper has no counterpart).  The FP64 path's particle kernels are
// bound by the FP64 pipe, so their roofline needs this rate; it is timed here rather than
// taken from a data sheet.
#include <cuda_runtime.h>

#include "pic.h"

namespace {

constexpr int kChains = 8;      // independent FMA chains per thread (hides the latency)
constexpr int kIters = 4096;    // FMAs per chain
constexpr int kThreads = 256;

// Every thread runs kChains chains of kIters FMAs a <- a b + c, with b just below one so
// that each chain stays finite (it tends to c/(1 - b)); the result is written only in a
// case that does not happen, so the chains are not removed.
__global__ void __launch_bounds__(kThreads) k_fma_chains(double b, double c, double* out) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k);
#pragma unroll 4
    for (int i = 0; i < kIters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __fma_rn(a[k], b, c);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.0) out[0] = s;
}

}  // namespace

extern "C" pic_status pic_measure_fp64_fma(void* stream, double* gflops) {
    if (!gflops) return PIC_ERR_INVALID_ARG;
    *gflops = 0.0;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PIC_ERR_CUDA;
    double* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = sms * 8;
    float best = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first run warms up
        cudaEventRecord(e0, s);
        k_fma_chains<<<blocks, kThreads, 0, s>>>(0.999999, 1e-6, out);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (e != cudaSuccess || best <= 0.f) return PIC_ERR_CUDA;
    const double flops = 2.0 * kChains * kIters * (double)blocks * kThreads;
    *gflops = flops / (best * 1e-3) / 1e9;
    return PIC_OK;
}
