// Persistent step kernel with bulk asynchronous copies (sm_100 family).
//
// Each CTA walks over row tiles of TX nodes (tile t covers row y, columns
// [x0, x0 + TX)).  A producer warp issues, per tile and population plane,
// the bulk copy (cp.async.bulk, completion counted in bytes on the stage's
// "full" mbarrier) of the source row segment the pull needs -- shifted by
// one column for a = +-1, so the segment is widened by a 16-byte halo on the
// side it reads from, with the periodic wrap at the row ends split into a
// second copy.  Consumer warps wait on "full", take their operands into
// registers, release the stage on its "empty" mbarrier (one arrival per
// warp) and compute; the producer refills a stage once every consumer warp
// has released it.  No CTA-wide barrier sits in the loop, so loads stay in
// flight while the consumers compute.  The collision is the same
// register-only collide() as the other step kernels, and results go straight
// to global memory with 16- or 8-byte vector stores.
//
// Shared memory per stage: [9][TX + 2H] elements, H = 16 / sizeof(S); the
// element for column x of the tile is at index x - x0 + H.
//
// Every wait on an mbarrier has an iteration limit; when it runs out the
// kernel raises bit 1 of the status flag and the CTA drains its own copies
// (again with a limit) before returning, so a fault in the copy path ends
// the launch with an error status instead of hanging the GPU.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "kbc_kernels.cuh"

namespace kbc {

constexpr int kTmaStages = 4;
constexpr int kTmaTile = 512;           // nodes per tile
constexpr unsigned kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// true when the phase with the given parity has completed
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return done != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity)
{
    for (unsigned it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, unsigned bytes,
                                         uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst_smem)), "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bytes one stage receives: three unshifted planes of TX elements and six
// shifted planes of TX + H elements.
template <class S, int TX>
__host__ __device__ constexpr unsigned tma_stage_tx_bytes()
{
    return (unsigned)((3 * TX + 6 * (TX + 16 / (int)sizeof(S))) * (int)sizeof(S));
}

template <class S, int TX>
__host__ __device__ constexpr size_t tma_smem_bytes()
{
    return (size_t)kTmaStages * 9 * (TX + 2 * (16 / sizeof(S))) * sizeof(S) + 2 * kTmaStages * 8 + 64;
}

// issue the copies of tile `t` into stage buffer `buf` (one thread)
template <class S, int TX>
__device__ __forceinline__ void tma_issue(const S* __restrict__ src, S* buf, uint64_t* bar, int t,
                                          int tiles_per_row, const StepArgs& a)
{
    constexpr int H = 16 / (int)sizeof(S);
    constexpr int ROW = TX + 2 * H;
    const int y = t / tiles_per_row;
    const int x0 = (t - y * tiles_per_row) * TX;
    const int ym = pull_row(y - 1, a);
    const int yp = pull_row(y + 1, a);
    mbar_expect_tx(bar, tma_stage_tx_bytes<S, TX>());
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ai = i % 3 - 1, bi = i / 3 - 1;
        const int sy = (bi == 1) ? ym : (bi == -1 ? yp : y);
        const S* row = src + (long long)i * a.plane + (long long)sy * a.nx;
        S* dst = buf + i * ROW;
        if (ai == 0) {
            bulk_g2s(dst + H, row + x0, TX * sizeof(S), bar);
        } else if (ai == 1) {  // reads columns x0 - 1 ... : load [x0 - H, x0 + TX)
            if (x0 == 0) {
                bulk_g2s(dst, row + (a.nx - H), H * sizeof(S), bar);
                bulk_g2s(dst + H, row, TX * sizeof(S), bar);
            } else {
                bulk_g2s(dst, row + (x0 - H), (TX + H) * sizeof(S), bar);
            }
        } else {               // reads columns ... x0 + TX: load [x0, x0 + TX + H)
            if (x0 + TX == a.nx) {
                bulk_g2s(dst + H, row + x0, TX * sizeof(S), bar);
                bulk_g2s(dst + H + TX, row, H * sizeof(S), bar);
            } else {
                bulk_g2s(dst + H, row + x0, (TX + H) * sizeof(S), bar);
            }
        }
    }
}

template <class S, int NV>
__device__ __forceinline__ void lds_vec(const S* p, S (&v)[NV])
{
    using Raw = typename RawT<int(sizeof(S)) * NV>::type;
    union {
        Raw r;
        S s[NV];
    } u;
    u.r = *reinterpret_cast<const Raw*>(p);
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = u.s[k];
}

// Requires nx % TX == 0.  Grid: persistent, at most (tiles) CTAs of
// TX/NV + 32 threads (TX/NV consumers, one producer warp), dynamic shared
// memory tma_smem_bytes<S, TX>().
template <int VAR, class C, int TX>
__global__ void __launch_bounds__(TX / C::kVec + 32)
step_tma(const typename C::S* __restrict__ src, typename C::S* __restrict__ dst, StepArgs a)
{
    using S = typename C::S;
    using T = typename C::T;
    constexpr int NV = C::kVec;
    constexpr int H = 16 / (int)sizeof(S);
    constexpr int ROW = TX + 2 * H;
    constexpr int NCW = TX / NV / 32;  // consumer warps
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S* stage_buf = reinterpret_cast<S*>(smem_raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + (size_t)kTmaStages * 9 * ROW * sizeof(S));
    uint64_t* empty = full + kTmaStages;
    __shared__ volatile int abort_flag;

    const int tiles_per_row = a.nx / TX;
    const int tiles = tiles_per_row * a.ny;
    const int first = blockIdx.x, stride = gridDim.x;
    const int my_tiles = first < tiles ? (tiles - 1 - first) / stride + 1 : 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (blockIdx.x == 0 && threadIdx.x == 0 && a.fix_count) a.fix_count[a.fix_slot ^ 1] = 0;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < kTmaStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == NCW) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            for (int k = 0; k < my_tiles; ++k) {
                const int s = k % kTmaStages;
                if (k >= kTmaStages) {
                    const unsigned par = (unsigned)(((k / kTmaStages) - 1) & 1);
                    if (!mbar_wait_bounded(&empty[s], par)) {
                        abort_flag = 1;
                        break;
                    }
                    fence_proxy_async();
                }
                if (abort_flag) break;
                tma_issue<S, TX>(src, stage_buf + (size_t)s * 9 * ROW, &full[s],
                                 first + k * stride, tiles_per_row, a);
            }
        }
        return;
    }

    // -------------------------------------------------------------- consumers
    const CollideParams<T>& p = params_of<T>(a);
    const int lx = (warp * 32 + lane) * NV;
    bool bad = false;
    int k = 0;
    for (; k < my_tiles; ++k) {
        const int s = k % kTmaStages;
        const unsigned parity = (unsigned)((k / kTmaStages) & 1);
        if (!mbar_wait_bounded(&full[s], parity)) {
            abort_flag = 1;
            break;
        }
        const int t = first + k * stride;
        const int y = t / tiles_per_row;
        const int x0 = (t - y * tiles_per_row) * TX;
        const S* buf = stage_buf + (size_t)s * 9 * ROW;
        T f[NV][9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ai = i % 3 - 1;
            const S* pl = buf + i * ROW;
            if (ai == 0) {
                S v[NV];
                lds_vec<S, NV>(pl + H + lx, v);
#pragma unroll
                for (int q = 0; q < NV; ++q) f[q][i] = C::load(v[q], i, a.cs);
            } else if (ai == 1) {  // column x - 1
                S lo[NV], hi[NV];
                lds_vec<S, NV>(pl + H - NV + lx, lo);
                lds_vec<S, NV>(pl + H + lx, hi);
                f[0][i] = C::load(lo[NV - 1], i, a.cs);
#pragma unroll
                for (int q = 1; q < NV; ++q) f[q][i] = C::load(hi[q - 1], i, a.cs);
            } else {               // column x + 1
                S lo[NV], hi[NV];
                lds_vec<S, NV>(pl + H + lx, lo);
                lds_vec<S, NV>(pl + H + NV + lx, hi);
#pragma unroll
                for (int q = 0; q < NV - 1; ++q) f[q][i] = C::load(lo[q + 1], i, a.cs);
                f[NV - 1][i] = C::load(hi[0], i, a.cs);
            }
        }
        // this warp's operands are in registers: release the stage
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        // storage units (FP16): node pairs in packed FP32x2 arithmetic
        const unsigned hits = collide_vec<VAR, C::kUnits, C::kUnits>(f, p, bad);
        if constexpr (VAR != kLBGK) {
            if (a.fix_list) record_fix_mask<NV>(hits, y * a.nx + x0 + lx, a);
        }
        const long long o = (long long)y * a.nx + x0 + lx;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if constexpr (std::is_same<C, CodecF16>::value && NV % 2 == 0) {
                unsigned pk[NV / 2];
#pragma unroll
                for (int q = 0; q < NV; q += 2) pk[q / 2] = C::store2(f[q][i], f[q + 1][i], i, a.cs);
                Vec<unsigned, NV / 2>::store(reinterpret_cast<unsigned*>(dst + (long long)i * a.plane + o), pk);
            } else {
                S out[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) out[q] = C::store(f[q][i], i, a.cs);
                Vec<S, NV>::store(dst + (long long)i * a.plane + o, out);
            }
        }
    }
    if (bad) atomicOr(a.flag, 1);
    if (k < my_tiles && lane == 0) {
        // aborted: report, then wait (bounded) for the copies that may still be
        // in flight into this CTA's shared memory before it is released
        atomicOr(a.flag, 2);
        if (warp == 0)
            for (int kk = k; kk < my_tiles && kk < k + kTmaStages; ++kk)
                mbar_wait_bounded(&full[kk % kTmaStages], (unsigned)((kk / kTmaStages) & 1));
    }
}

}  // namespace kbc
