// Diagnostics of a caller-owned FP64 population field with no device
// allocation (declaration and contract: kbc_diagnostics_noalloc in
// include/kbc.h).
//
// The per-block partial sums and the final result live in one file-scope
// device array.  Host code must not hand the array's name to a kernel: on
// the host that name is only a stand-in, and on a GPU that can reach host
// memory the kernel would silently work on the wrong memory.  The device
// address is fetched with cudaGetSymbolAddress once per device and context
// (the context's unique id tells a context created after cudaDeviceReset
// from the one the cached address belongs to) and cached.
#include <chrono>
#include <mutex>
#include <thread>

#include <cudaTypedefs.h>

#include "../../include/kbc.h"
#include "kbc_launch.cuh"

namespace kbc {
namespace {

// caller populations are the plain f_i; the kernels work on d_i = f_i - W_i
struct CodecF64Plain {
    using S = double;
    using T = double;
    __device__ __forceinline__ static double to_f64(S s, int i, const CodecScale&)
    {
        return s - wgt(i);
    }
};

constexpr long long kNodesPerBlock = 64LL * kDiagBlock;  // 64 nodes per thread
constexpr int kMaxBlocks = 16384;                        // => at most 2^28 nodes
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_scratch[kMaxBlocks * kDiagParts + 32];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// Unique id of the current context (0 when it cannot be had: the address is
// then looked up on every call instead of cached).
unsigned long long current_context_id()
{
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(fn);
        cudaGetLastError();
        looked_up = true;
    }
    unsigned long long id = 0;
    if (!get_id || get_id(nullptr, &id) != CUDA_SUCCESS) return 0;
    return id;
}

}  // namespace
}  // namespace kbc

using namespace kbc;

extern "C" int kbc_diagnostics_noalloc(int nx, int ny, int variant, double beta, const double* f,
                                       double* out, void* stream)
{
    if (nx < 1 || ny < 1) return handle_free_error(KBC_ERR_ARG, "noalloc diagnostics: nx, ny >= 1");
    const long long total = (long long)nx * ny;
    if (total > kNodesPerBlock * kMaxBlocks)
        return handle_free_error(KBC_ERR_ARG,
                                 "noalloc diagnostics: more than 2^28 nodes, the size its static "
                                 "scratch holds (use kbc_diagnostics)");
    if (variant < KBC_LBGK || variant > KBC_D || !(beta > 0.0 && beta <= 1.0) || !f || !out)
        return handle_free_error(KBC_ERR_ARG, "noalloc diagnostics: bad variant, beta or pointer");
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, f) != cudaSuccess) {
        cudaGetLastError();
        return handle_free_error(KBC_ERR_ARG, "noalloc diagnostics: f is not a known pointer");
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return handle_free_error(KBC_ERR_ARG,
                                 "noalloc diagnostics: f must be device memory (staging a host "
                                 "field would allocate)");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return handle_free_error(KBC_ERR_CUDA, "noalloc diagnostics: no usable current device");
    // the kernels read f directly: it must live on the current device
    if (at.type == cudaMemoryTypeDevice && at.device != dev)
        return handle_free_error(KBC_ERR_ARG, "noalloc diagnostics: f is on another device");
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        const unsigned long long ctx = current_context_id();
        if (!g_scratch_addr[dev] || ctx == 0 || g_scratch_ctx[dev] != ctx) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return handle_free_error(KBC_ERR_CUDA, "noalloc diagnostics: cudaGetSymbolAddress failed");
            }
            g_scratch_addr[dev] = static_cast<double*>(p);
            g_scratch_ctx[dev] = ctx;
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StepArgs a{};
    a.nx = nx;
    a.ny = ny;
    a.plane = total;
    a.cs = make_scale(1.0);
    a.pd = make_params<double>(beta, 0, 2.0, 0.0);
    a.pf = make_params<float>(beta, 0, 2.0, 0.0);
    a.beta = beta;
    a.ywrap = 1;
    const int nblocks = (int)((total + kNodesPerBlock - 1) / kNodesPerBlock);
    double* result = scratch + (long long)kMaxBlocks * kDiagParts;
    switch (variant) {
    case kLBGK: diag_partial<kLBGK, CodecF64Plain><<<nblocks, kDiagBlock, 0, s>>>(f, scratch, a); break;
    case kA: diag_partial<kA, CodecF64Plain><<<nblocks, kDiagBlock, 0, s>>>(f, scratch, a); break;
    case kB: diag_partial<kB, CodecF64Plain><<<nblocks, kDiagBlock, 0, s>>>(f, scratch, a); break;
    case kC: diag_partial<kC, CodecF64Plain><<<nblocks, kDiagBlock, 0, s>>>(f, scratch, a); break;
    default: diag_partial<kD, CodecF64Plain><<<nblocks, kDiagBlock, 0, s>>>(f, scratch, a); break;
    }
    diag_final<<<1, kDiagBlock, 0, s>>>(scratch, nblocks, result, total, 0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, result, KBC_DIAG_N * sizeof(double), cudaMemcpyDefault, s);
    if (e != cudaSuccess) return handle_free_error(KBC_ERR_CUDA, "noalloc diagnostics: launch or copy failed");
    // bounded wait for the result (the shared scratch is free again afterwards)
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        e = cudaStreamQuery(s);
        if (e == cudaSuccess) return KBC_OK;
        if (e != cudaErrorNotReady) return handle_free_error(KBC_ERR_CUDA, "noalloc diagnostics: stream error");
        if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(600))
            return handle_free_error(KBC_ERR_TIMEOUT, "noalloc diagnostics: timed out waiting for the stream");
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}
