// Reverse step of the adjoint for FP32 storage with its operands prefetched
// by per-thread asynchronous copies.
//
// Same arithmetic and outputs as adj_step (one node per thread over row
// segments, collide_adjoint, the scatter of lambda^n to the pull sources,
// the guard mask, the per-block beta sums).  While a thread computes its
// node of one segment, the eighteen operands of its node in the next
// segment (nine pulled forward-state values, nine of lambda^{n+1}) are
// already on their way into its own shared-memory slots by cp.async (4-byte
// copies, one commit group per segment, two stages); the thread then waits
// only for its own group.  No slot is shared between threads, so no block
// barrier orders the stages, and no register holds a prefetched value.
#pragma once

#include <cuda_runtime.h>

#include "kbc_adjoint.cuh"

namespace kbc {

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                     static_cast<unsigned>(__cvta_generic_to_shared(smem))),
                 "l"(gmem)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int VAR>
__global__ void __launch_bounds__(kAdjBlock, adj_min_blocks<VAR, float>())
adj_step_async(const float* __restrict__ g, const float* __restrict__ lam_in,
               float* __restrict__ lam_out, double* __restrict__ part,
               unsigned* __restrict__ fixmask, StepArgs a)
{
    // [stage][operand][thread]: consecutive threads use consecutive banks
    __shared__ float slot[2][18][kAdjBlock];
    const CollideParams<float>& p = a.pf;
    const int nbx = (a.nx + kAdjBlock - 1) / kAdjBlock;
    const int segs = nbx * a.ny;  // nx * ny < 2^31
    const int t = threadIdx.x;
    // each block takes a contiguous run of segments (fixed, so the beta sums
    // keep their order), stepping row and column without a division
    const int per = (segs + (int)gridDim.x - 1) / (int)gridDim.x;
    const int sg0 = (int)blockIdx.x * per;
    const int sg1 = sg0 + per < segs ? sg0 + per : segs;
    // Offset of population i's pull source from node n: plane, source row
    // (y - b, periodic: dn / up for b = +1 / -1) and source column (x - a:
    // -a except at the row ends, where cl / cr wrap).  In a segment away from
    // the row ends the column offsets are the constants -1, +1 for the whole
    // block.
    auto src_off = [&](int i, long long dn, long long up, int cl, int cr) {
        const int ai = i % 3 - 1, bi = i / 3 - 1;
        return (long long)i * a.plane + (bi == 1 ? dn : (bi == -1 ? up : 0)) +
               (ai == 1 ? cl : (ai == -1 ? cr : 0));
    };
    auto row_offs = [&](int y, long long& dn, long long& up) {
        dn = (y == 0) ? (long long)(a.ny - 1) * a.nx : -(long long)a.nx;
        up = (y == a.ny - 1) ? -(long long)(a.ny - 1) * a.nx : (long long)a.nx;
    };
    auto prefetch = [&](int y, int bx, bool live, int s) {
        const int x0 = bx * kAdjBlock, x = x0 + t;
        if (live && x < a.nx) {
            long long dn, up;
            row_offs(y, dn, up);
            const long long n = (long long)y * a.nx + x;
            const float* gn = g + n;
            const float* ln = lam_in + n;
            if (x0 > 0 && x0 + kAdjBlock < a.nx) {
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    cp_async4(&slot[s][i][t], gn + src_off(i, dn, up, -1, 1));
                    cp_async4(&slot[s][9 + i][t], ln + (long long)i * a.plane);
                }
            } else {
                const int cl = (x == 0) ? a.nx - 1 : -1;
                const int cr = (x == a.nx - 1) ? 1 - a.nx : 1;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    cp_async4(&slot[s][i][t], gn + src_off(i, dn, up, cl, cr));
                    cp_async4(&slot[s][9 + i][t], ln + (long long)i * a.plane);
                }
            }
        }
        cp_async_commit();  // one group per segment, empty or not
    };
    double bsum = 0.0;
    int y = sg0 < segs ? sg0 / nbx : 0;
    int bx = sg0 - y * nbx;
    prefetch(y, bx, sg0 < sg1, 0);
    for (int k = 0, sg = sg0; sg < sg1; ++k, ++sg) {
        int yn = y, bn = bx + 1;
        if (bn == nbx) {
            bn = 0;
            ++yn;
        }
        prefetch(yn, bn, sg + 1 < sg1, (k + 1) & 1);
        cp_async_wait<1>();  // this thread's copies of segment sg have landed
        const int x0 = bx * kAdjBlock, x = x0 + t;
        const int yc = y;
        y = yn;
        bx = bn;
        if (x >= a.nx) continue;
        const int s = k & 1;
        float d[9], lam[9], mu[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            d[i] = slot[s][i][t];
            lam[i] = slot[s][9 + i][t];
        }
        float bbar;
        const long long n = (long long)yc * a.nx + x;
        const bool guarded = collide_adjoint<VAR>(d, lam, p, mu, bbar);
        if constexpr (VAR != kLBGK) {
            if (guarded) {
                atomicOr(fixmask + (n >> 5), 1u << (n & 31));
                bbar = 0.0f;  // summed by adj_fixup
            }
        }
        bsum += (double)bbar;
        long long dn, up;
        row_offs(yc, dn, up);
        float* lo = lam_out + n;
        if (x0 > 0 && x0 + kAdjBlock < a.nx) {
#pragma unroll
            for (int i = 0; i < 9; ++i) lo[src_off(i, dn, up, -1, 1)] = mu[i];
        } else {
            const int cl = (x == 0) ? a.nx - 1 : -1;
            const int cr = (x == a.nx - 1) ? 1 - a.nx : 1;
#pragma unroll
            for (int i = 0; i < 9; ++i) lo[src_off(i, dn, up, cl, cr)] = mu[i];
        }
    }
    cp_async_wait<0>();  // nothing left in flight into this block's slots
    block_add(bsum, part + blockIdx.x);
}

}  // namespace kbc
