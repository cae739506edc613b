// Host-side launchers, one explicit instantiation per storage codec
// (kbc_f64.cu, kbc_f32.cu, kbc_f16.cu).
#pragma once

#include <type_traits>

#include <cuda_runtime.h>

#include "kbc_adjoint.cuh"
#include "kbc_adjoint_async.cuh"
#include "kbc_kernels.cuh"
#include "kbc_tma.cuh"

namespace kbc {

struct Launch {
    const void* src;
    void* dst;
    StepArgs a;
    int variant;
    bool rows;      // vectorised row kernel (nx % (32 * kVec) == 0)
    bool tma;       // persistent bulk-copy kernel (nx % kTmaTile == 0, F32/F16)
    bool all_f64;   // whole collision in double (exact-gamma mode)
    bool fixup;     // FP64 re-evaluation pass after the step
    cudaStream_t stream;
    int num_sms;
};

// Records msg as the message of kbc_last_error(NULL) and returns code (for
// the entry points that take no handle).
int handle_free_error(int code, const char* msg);

constexpr int kRowBlock = 64;
constexpr int kNodeBlock = 256;

inline int grid_for(long long total, int block, int num_sms, int per_sm)
{
    long long b = (total + block - 1) / block;
    long long cap = (long long)num_sms * per_sm;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

template <int VAR, class C>
cudaError_t launch_step_v(const Launch& L)
{
    using S = typename C::S;
    const S* src = static_cast<const S*>(L.src);
    S* dst = static_cast<S*>(L.dst);
    if (L.all_f64) {
        const long long total = (long long)L.a.nx * L.a.ny;
        step_nodes_f64<VAR, C><<<grid_for(total, kNodeBlock, L.num_sms, 16), kNodeBlock, 0,
                                 L.stream>>>(src, dst, L.a);
        return cudaGetLastError();
    }
    if constexpr (!std::is_same<C, CodecF64>::value) {
        if (L.tma) {
            constexpr size_t smem = tma_smem_bytes<S, kTmaTile>();
            constexpr int threads = kTmaTile / C::kVec + 32;
            static int per_sm = 0;  // resident CTAs per SM, from the occupancy calculator
            if (per_sm == 0) {
                cudaError_t e = cudaFuncSetAttribute(step_tma<VAR, C, kTmaTile>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)smem);
                if (e != cudaSuccess) return e;
                int n = 0;
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_tma<VAR, C, kTmaTile>,
                                                                  threads, smem);
                if (e != cudaSuccess) return e;
                per_sm = n > 0 ? n : 1;
            }
            const long long tiles = (long long)(L.a.nx / kTmaTile) * L.a.ny;
            long long grid = (long long)L.num_sms * per_sm;
            if (grid > tiles) grid = tiles;
            step_tma<VAR, C, kTmaTile><<<(unsigned)grid, threads, smem, L.stream>>>(src, dst, L.a);
            if constexpr (VAR != kLBGK) {
                if (L.fixup)
                    step_fixup<VAR, C><<<L.num_sms * 2, kNodeBlock, 0, L.stream>>>(src, dst, L.a);
            }
            return cudaGetLastError();
        }
    }
    if (L.rows) {
        constexpr int NV = C::kVec;
        const int nbx = (L.a.nx + kRowBlock * NV - 1) / (kRowBlock * NV);
        step_rows<VAR, C, NV, kRowBlock>
            <<<(unsigned)((long long)nbx * L.a.ny), kRowBlock, 0, L.stream>>>(src, dst, L.a, nbx);
    } else {
        const long long total = (long long)L.a.nx * L.a.ny;
        step_nodes<VAR, C><<<grid_for(total, kNodeBlock, L.num_sms, 16), kNodeBlock, 0, L.stream>>>(
            src, dst, L.a);
    }
    if constexpr (VAR != kLBGK) {
        if (L.fixup)
            step_fixup<VAR, C><<<L.num_sms * 2, kNodeBlock, 0, L.stream>>>(src, dst, L.a);
    }
    return cudaGetLastError();
}

template <class C>
cudaError_t launch_step(const Launch& L)
{
    switch (L.variant) {
    case kLBGK: return launch_step_v<kLBGK, C>(L);
    case kA: return launch_step_v<kA, C>(L);
    case kB: return launch_step_v<kB, C>(L);
    case kC: return launch_step_v<kC, C>(L);
    case kD: return launch_step_v<kD, C>(L);
    default: return cudaErrorInvalidValue;
    }
}

template <class C>
cudaError_t launch_init(const double* rho, const double* ux, const double* uy, void* dst,
                        const StepArgs& a, bool grad, cudaStream_t s, int num_sms)
{
    const long long total = (long long)a.nx * a.ny;
    const int g = grid_for(total, kNodeBlock, num_sms, 16);
    if (grad)
        init_grad<C><<<g, kNodeBlock, 0, s>>>(rho, ux, uy, static_cast<typename C::S*>(dst), a);
    else
        init_feq<C><<<g, kNodeBlock, 0, s>>>(rho, ux, uy, static_cast<typename C::S*>(dst), a);
    return cudaGetLastError();
}

template <class C>
cudaError_t launch_set(const double* f, void* dst, const StepArgs& a, cudaStream_t s, int num_sms)
{
    const long long total = (long long)a.nx * a.ny;
    set_populations<C><<<grid_for(total, kNodeBlock, num_sms, 16), kNodeBlock, 0, s>>>(
        f, static_cast<typename C::S*>(dst), a);
    return cudaGetLastError();
}

template <class C>
cudaError_t launch_get(const void* src, double* f, const StepArgs& a, cudaStream_t s, int num_sms)
{
    const long long total = (long long)a.nx * a.ny;
    get_populations<C><<<grid_for(total, kNodeBlock, num_sms, 16), kNodeBlock, 0, s>>>(
        static_cast<const typename C::S*>(src), f, a);
    return cudaGetLastError();
}

template <class C>
cudaError_t launch_moments(const void* src, double* rho, double* ux, double* uy,
                           const StepArgs& a, cudaStream_t s, int num_sms)
{
    const long long total = (long long)a.nx * a.ny;
    moments<C><<<grid_for(total, kNodeBlock, num_sms, 16), kNodeBlock, 0, s>>>(
        static_cast<const typename C::S*>(src), rho, ux, uy, a);
    return cudaGetLastError();
}

template <class C>
cudaError_t launch_probe(const void* src, const long long* nodes, int count, double* f, int* bad,
                         const StepArgs& a, cudaStream_t s, int num_sms)
{
    probe_nodes<C><<<grid_for(count, kNodeBlock, num_sms, 4), kNodeBlock, 0, s>>>(
        static_cast<const typename C::S*>(src), nodes, count, f, bad, a);
    return cudaGetLastError();
}

// number of partial-sum blocks the diagnostics use for this grid
inline int diag_blocks(long long total, int num_sms)
{
    return grid_for(total, kDiagBlock, num_sms, 4);
}

template <class C>
cudaError_t launch_diag(const void* src, double* part, int nblocks, double* out, int variant,
                        const StepArgs& a, cudaStream_t s, int raw)
{
    const typename C::S* p = static_cast<const typename C::S*>(src);
    switch (variant) {
    case kLBGK: diag_partial<kLBGK, C><<<nblocks, kDiagBlock, 0, s>>>(p, part, a); break;
    case kA: diag_partial<kA, C><<<nblocks, kDiagBlock, 0, s>>>(p, part, a); break;
    case kB: diag_partial<kB, C><<<nblocks, kDiagBlock, 0, s>>>(p, part, a); break;
    case kC: diag_partial<kC, C><<<nblocks, kDiagBlock, 0, s>>>(p, part, a); break;
    case kD: diag_partial<kD, C><<<nblocks, kDiagBlock, 0, s>>>(p, part, a); break;
    default: return cudaErrorInvalidValue;
    }
    diag_final<<<1, kDiagBlock, 0, s>>>(part, nblocks, out, (long long)a.nx * a.ny, raw);
    return cudaGetLastError();
}

template <class C>
cudaError_t launch_diag_ext(const void* src, double* part, int nblocks, double* out,
                            const StepArgs& a, cudaStream_t s)
{
    diag_ext_partial<C><<<nblocks, kDiagBlock, 0, s>>>(static_cast<const typename C::S*>(src), part, a);
    diag_ext_final<<<1, kDiagBlock, 0, s>>>(part, nblocks, out, (long long)a.nx * a.ny);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- adjoint

inline int adj_blocks(long long total, int num_sms) { return grid_for(total, 256, num_sms, 8); }

// One reverse step: FP32 storage prefetches each thread's operands by
// asynchronous copies (adj_step_async); the other storages load them node
// by node (adj_step).
template <int VAR, class C>
void launch_adj_step_v(const typename C::S* g, const typename C::T* li, typename C::T* lo,
                       double* part, unsigned* fixmask, int nblocks, const StepArgs& a, cudaStream_t s)
{
    if constexpr (std::is_same<C, CodecF32>::value)
        adj_step_async<VAR><<<nblocks, kAdjBlock, 0, s>>>(g, li, lo, part, fixmask, a);
    else
        adj_step<VAR, C><<<nblocks, kAdjBlock, 0, s>>>(g, li, lo, part, fixmask, a);
}

template <class C>
cudaError_t launch_adj_step(int variant, const void* g, const void* lam_in, void* lam_out,
                            double* part, unsigned* fixmask, int nblocks, const StepArgs& a,
                            cudaStream_t s)
{
    using S = typename C::S;
    using T = typename C::T;
    const S* gp = static_cast<const S*>(g);
    const T* li = static_cast<const T*>(lam_in);
    T* lo = static_cast<T*>(lam_out);
    constexpr bool fix = !std::is_same<T, double>::value;
    // the double redo scans one mask word per thread: a grid sized to the
    // mask (at most the step's), so small grids do not pay for idle blocks;
    // its beta partial sums land in part[0 .. fblocks) in a fixed order
    const long long words = ((long long)a.nx * a.ny + 31) / 32;
    const int fblocks = (int)((words + 255) / 256 < nblocks ? (words + 255) / 256 : nblocks);
    switch (variant) {
    case kLBGK: launch_adj_step_v<kLBGK, C>(gp, li, lo, part, fixmask, nblocks, a, s); break;
#define KBC_ADJ_CASE(V)                                                                  \
    case V:                                                                              \
        launch_adj_step_v<V, C>(gp, li, lo, part, fixmask, nblocks, a, s);               \
        if (fix) adj_fixup<V, C><<<fblocks, 256, 0, s>>>(gp, li, lo, part, fixmask, a); \
        break;
    KBC_ADJ_CASE(kA)
    KBC_ADJ_CASE(kB)
    KBC_ADJ_CASE(kC)
    KBC_ADJ_CASE(kD)
#undef KBC_ADJ_CASE
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class C>
cudaError_t launch_adj_objective(const void* g, const double* tx, const double* ty, int objective,
                                 void* lam, double* part, int nblocks, const StepArgs& a,
                                 cudaStream_t s)
{
    adj_objective<C><<<nblocks, 256, 0, s>>>(static_cast<const typename C::S*>(g), tx, ty, objective,
                                             static_cast<typename C::T*>(lam), part, a);
    return cudaGetLastError();
}

template <class C>
cudaError_t launch_adj_grad_u0(const double* rho0, const double* ux0, const double* uy0,
                               const void* lam, double* gx, double* gy, const StepArgs& a,
                               cudaStream_t s, int num_sms)
{
    const long long total = (long long)a.nx * a.ny;
    adj_grad_u0<C><<<grid_for(total, 256, num_sms, 16), 256, 0, s>>>(
        rho0, ux0, uy0, static_cast<const typename C::T*>(lam), gx, gy, a);
    return cudaGetLastError();
}

// explicit instantiations live in the per-codec translation units
#define KBC_DECLARE_CODEC(C)                                                                   \
    extern template cudaError_t launch_step<C>(const Launch&);                                \
    extern template cudaError_t launch_init<C>(const double*, const double*, const double*,   \
                                               void*, const StepArgs&, bool, cudaStream_t,    \
                                               int);                                          \
    extern template cudaError_t launch_set<C>(const double*, void*, const StepArgs&,          \
                                              cudaStream_t, int);                             \
    extern template cudaError_t launch_get<C>(const void*, double*, const StepArgs&,          \
                                              cudaStream_t, int);                             \
    extern template cudaError_t launch_moments<C>(const void*, double*, double*, double*,     \
                                                  const StepArgs&, cudaStream_t, int);        \
    extern template cudaError_t launch_diag<C>(const void*, double*, int, double*, int,       \
                                               const StepArgs&, cudaStream_t, int);           \
    extern template cudaError_t launch_probe<C>(const void*, const long long*, int, double*,  \
                                                int*, const StepArgs&, cudaStream_t, int);    \
    extern template cudaError_t launch_diag_ext<C>(const void*, double*, int, double*,        \
                                                   const StepArgs&, cudaStream_t);            \
    extern template cudaError_t launch_adj_step<C>(int, const void*, const void*, void*,      \
                                                   double*, unsigned*, int, const StepArgs&,  \
                                                   cudaStream_t);                             \
    extern template cudaError_t launch_adj_objective<C>(const void*, const double*,           \
                                                        const double*, int, void*, double*,   \
                                                        int, const StepArgs&, cudaStream_t);  \
    extern template cudaError_t launch_adj_grad_u0<C>(const double*, const double*,           \
                                                      const double*, const void*, double*,    \
                                                      double*, const StepArgs&, cudaStream_t, \
                                                      int);

#define KBC_DEFINE_CODEC(C)                                                                    \
    template cudaError_t launch_step<C>(const Launch&);                                       \
    template cudaError_t launch_init<C>(const double*, const double*, const double*, void*,   \
                                        const StepArgs&, bool, cudaStream_t, int);            \
    template cudaError_t launch_set<C>(const double*, void*, const StepArgs&, cudaStream_t,   \
                                       int);                                                  \
    template cudaError_t launch_get<C>(const void*, double*, const StepArgs&, cudaStream_t,   \
                                       int);                                                  \
    template cudaError_t launch_moments<C>(const void*, double*, double*, double*,            \
                                           const StepArgs&, cudaStream_t, int);               \
    template cudaError_t launch_diag<C>(const void*, double*, int, double*, int,              \
                                        const StepArgs&, cudaStream_t, int);                  \
    template cudaError_t launch_probe<C>(const void*, const long long*, int, double*, int*,   \
                                         const StepArgs&, cudaStream_t, int);                 \
    template cudaError_t launch_diag_ext<C>(const void*, double*, int, double*,               \
                                            const StepArgs&, cudaStream_t);                   \
    template cudaError_t launch_adj_step<C>(int, const void*, const void*, void*, double*,    \
                                            unsigned*, int, const StepArgs&, cudaStream_t);   \
    template cudaError_t launch_adj_objective<C>(const void*, const double*, const double*,   \
                                                 int, void*, double*, int, const StepArgs&,   \
                                                 cudaStream_t);                               \
    template cudaError_t launch_adj_grad_u0<C>(const double*, const double*, const double*,   \
                                               const void*, double*, double*,                 \
                                               const StepArgs&, cudaStream_t, int);

#ifndef KBC_CODEC_TU
KBC_DECLARE_CODEC(CodecF64)
KBC_DECLARE_CODEC(CodecF32)
KBC_DECLARE_CODEC(CodecF16)
#endif

}  // namespace kbc
