// Throughput of the FP64 fused multiply-add pipe, the ceiling of the
// all-double storage path (declaration: kbc_fp64_fma_rate in include/kbc.h).
//
// Every thread runs kChains independent chains a <- a * b + c (one DFMA
// each per iteration), so the pipe is never waiting on a dependency; the
// grid fills every SM.  The chains' sum is compared with a value it never
// takes (the host passes it), which keeps the compiler from removing the
// loop without adding a store per iteration.
#include <cuda_runtime.h>

#include "../../include/kbc.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kIters = 2048;

__device__ double g_fma_sink;

__global__ void __launch_bounds__(kThreads) dfma_chains(double b, double c, double never)
{
    double acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = __fma_rn(acc[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += acc[k];
    if (s == never) g_fma_sink = s;
}

}  // namespace

extern "C" int kbc_fp64_fma_rate(void* stream, double* dfma_per_s)
{
    if (!dfma_per_s) return KBC_ERR_ARG;
    *dfma_per_s = 0.0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return KBC_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = sms * 8;
    const double ops = (double)blocks * kThreads * kChains * kIters;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return KBC_ERR_CUDA;
    }
    double best = 0.0;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {  // the first launch warms up
        err = cudaEventRecord(e0, s);
        dfma_chains<<<blocks, kThreads, 0, s>>>(0.9999999, 1e-7, -1.0);
        if (err == cudaSuccess) err = cudaGetLastError();
        if (err == cudaSuccess) err = cudaEventRecord(e1, s);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && rep > 0 && ms > 0.0f) {
            const double r = ops / (ms * 1e-3);
            if (r > best) best = r;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return KBC_ERR_CUDA;
    }
    *dfma_per_s = best;
    return KBC_OK;
}
