// Kernels of the fused pull-stream + collide step and its helpers.
//
// Data layout in device memory (one population field):
//   S f[9][plane], plane >= nx * ny, row-major [ny][nx] inside a plane, x
//   fastest; plane is padded so every plane starts on a 256-byte boundary.
// Two fields (A, B) alternate: a step reads A and writes B (pull pattern:
// f_i(x) = f'_i(x - v_i) with periodic wrap, Eq. Egeneral).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <type_traits>

#include "kbc_collide.cuh"

namespace kbc {

struct StepArgs {
    int nx, ny;
    long long plane;     // elements between population planes
    CodecScale cs;
    CollideParams<float> pf;   // collision constants, computed on the host
    CollideParams<double> pd;
    double beta;               // relaxation parameter (Grad initialisation)
    int* fix_count;      // two counters, used alternately by successive steps
    int* fix_list;       // node indices recorded for the FP64 re-evaluation
    int fix_slot;        // counter used by this step
    int* flag;           // set to 1 when a node's density is not finite
    int ywrap;           // 1: periodic in y; 0: a y-slab whose rows -1 and ny are
                         // ghost rows holding the neighbouring slabs' populations
};

// Source row of a pull that lands on row sy (y - b, so -1 <= sy <= ny):
// periodic wrap, or on a y-slab the ghost row itself.
__device__ __forceinline__ int pull_row(int sy, const StepArgs& a)
{
    if (!a.ywrap) return sy;
    return sy < 0 ? sy + a.ny : (sy >= a.ny ? sy - a.ny : sy);
}

// ---------------------------------------------------------------- vectors

template <int BYTES> struct RawT;
template <> struct RawT<16> { using type = uint4; };
template <> struct RawT<8> { using type = uint2; };
template <> struct RawT<4> { using type = unsigned int; };

template <class S, int NV>
struct Vec {
    static constexpr int kBytes = int(sizeof(S)) * NV;
    using Raw = typename RawT<kBytes>::type;
    union U {
        Raw r;
        S s[NV];
    };
    __device__ __forceinline__ static void load(const S* p, S (&v)[NV])
    {
        U u;
        u.r = __ldg(reinterpret_cast<const Raw*>(p));
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = u.s[k];
    }
    __device__ __forceinline__ static void store(S* p, const S (&v)[NV])
    {
        U u;
#pragma unroll
        for (int k = 0; k < NV; ++k) u.s[k] = v[k];
        *reinterpret_cast<Raw*>(p) = u.r;
    }
};

template <class S> __device__ __forceinline__ S shfl_up1(S v)
{
    if constexpr (sizeof(S) == 2) {
        return (S)__shfl_up_sync(0xffffffffu, (unsigned)v, 1);
    } else {
        return __shfl_up_sync(0xffffffffu, v, 1);
    }
}
template <class S> __device__ __forceinline__ S shfl_down1(S v)
{
    if constexpr (sizeof(S) == 2) {
        return (S)__shfl_down_sync(0xffffffffu, (unsigned)v, 1);
    } else {
        return __shfl_down_sync(0xffffffffu, v, 1);
    }
}

// warp-aggregated append of node n to the re-evaluation list
__device__ __forceinline__ void record_fix(bool hit, int n, const StepArgs& a)
{
    const unsigned active = __activemask();
    const unsigned m = __ballot_sync(active, hit);
    if (m == 0u) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(a.fix_count + a.fix_slot, __popc(m));
    base = __shfl_sync(active, base, leader);
    const int idx = base + __popc(m & ((1u << lane) - 1u));
    if (hit && idx < a.nx * a.ny) a.fix_list[idx] = n;  // the list holds one entry per node
}

template <typename T> __device__ __forceinline__ const CollideParams<T>& params_of(const StepArgs& a);
template <> __device__ __forceinline__ const CollideParams<float>& params_of<float>(const StepArgs& a)
{
    return a.pf;
}
template <> __device__ __forceinline__ const CollideParams<double>& params_of<double>(const StepArgs& a)
{
    return a.pd;
}

// warp-aggregated append of up to NV node indices per lane (bit k of `hits`
// marks node n0 + k); one vote when no lane has a hit
template <int NV>
__device__ __forceinline__ void record_fix_mask(unsigned hits, int n0, const StepArgs& a)
{
    if (!__any_sync(0xffffffffu, hits != 0u)) return;
    if (hits) {
        int base = atomicAdd(a.fix_count + a.fix_slot, __popc(hits));
        const int cap = a.nx * a.ny;  // the list holds one entry per node
#pragma unroll
        for (int k = 0; k < NV; ++k)
            if (hits & (1u << k)) {
                if (base < cap) a.fix_list[base] = n0 + k;
                ++base;
            }
    }
}

// ---------------------------------------------------------------- step, rows

// Collides the NV nodes one thread holds.  Sets `bad` when a density is not
// finite; bit k of the result marks a guard hit of node k.  PAIRS: collide
// nodes 2j, 2j + 1 in one packed lane pair (float, NV even; the same bits as
// one node at a time, about half the arithmetic instructions, twice the
// registers of the collision).
template <int VAR, bool U, bool PAIRS = false, typename T, int NV>
__device__ __forceinline__ unsigned collide_vec(T (&f)[NV][9], const CollideParams<T>& p, bool& bad)
{
    unsigned hits = 0u;
    if constexpr (PAIRS && std::is_same<T, float>::value && NV % 2 == 0) {
#pragma unroll
        for (int k = 0; k < NV; k += 2) {
            T r0, r1;
            unsigned h;
            collide_pair<VAR, U>(f[k], f[k + 1], p, r0, r1, h);
            bad |= !isfinite(r0) || !isfinite(r1);
            hits |= h << k;
        }
    } else {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            T rho;
            bool hit;
            collide_node<VAR, U>(f[k], p, rho, hit);
            bad |= !isfinite(rho);
            hits |= (hit ? 1u : 0u) << k;
        }
    }
    return hits;
}

//
// One thread updates NV consecutive nodes of one row with 16-byte loads and
// stores per population plane.  Populations moving along x (a = +-1) need
// the neighbour one element to the left/right: it comes from the adjacent
// lane by a warp shuffle, and lanes 0 / 31 fetch it from memory (periodic
// wrap at the row ends).  Requires nx % (32 NV) == 0; a 1-D grid of
// nbx * ny blocks, nbx = ceil(nx / (BLOCK NV)) blocks per row; warps past
// the row end exit as a whole.
template <int VAR, class C, int NV, int BLOCK>
__global__ void __launch_bounds__(BLOCK, C::kRowMinBlocks)
step_rows(const typename C::S* __restrict__ src, typename C::S* __restrict__ dst, StepArgs a,
          int nbx)
{
    using S = typename C::S;
    using T = typename C::T;
    const int y = blockIdx.x / nbx;
    const int bx = blockIdx.x - y * nbx;
    const int x0 = (bx * BLOCK + threadIdx.x) * NV;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.fix_count)
        a.fix_count[a.fix_slot ^ 1] = 0;  // free the other counter for the next step
    if (x0 >= a.nx) return;               // whole warps only (nx % (32 NV) == 0)
    const int lane = threadIdx.x & 31;
    const int ym = pull_row(y - 1, a);
    const int yp = pull_row(y + 1, a);
    const int xl = (x0 == 0) ? a.nx - 1 : x0 - 1;
    const int xr = (x0 + NV == a.nx) ? 0 : x0 + NV;

    S raw[9][NV];
    S edge[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ai = i % 3 - 1, bi = i / 3 - 1;
        const int sy = (bi == 1) ? ym : (bi == -1 ? yp : y);   // source row y - b
        const S* row = src + (long long)i * a.plane + (long long)sy * a.nx;
        Vec<S, NV>::load(row + x0, raw[i]);
        if (ai == 1) {
            edge[i] = S(0);
            if (lane == 0) edge[i] = __ldg(row + xl);
        } else if (ai == -1) {
            edge[i] = S(0);
            if (lane == 31) edge[i] = __ldg(row + xr);
        }
    }
    T f[NV][9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ai = i % 3 - 1;
        if (ai == 0) {
#pragma unroll
            for (int k = 0; k < NV; ++k) f[k][i] = C::load(raw[i][k], i, a.cs);
        } else if (ai == 1) {  // source x - 1
            S left = shfl_up1(raw[i][NV - 1]);
            if (lane == 0) left = edge[i];
            f[0][i] = C::load(left, i, a.cs);
#pragma unroll
            for (int k = 1; k < NV; ++k) f[k][i] = C::load(raw[i][k - 1], i, a.cs);
        } else {               // source x + 1
            S right = shfl_down1(raw[i][0]);
            if (lane == 31) right = edge[i];
#pragma unroll
            for (int k = 0; k < NV - 1; ++k) f[k][i] = C::load(raw[i][k + 1], i, a.cs);
            f[NV - 1][i] = C::load(right, i, a.cs);
        }
    }
    bool bad = false;
    const unsigned hits = collide_vec<VAR, C::kUnits>(f, params_of<T>(a), bad);
    if constexpr (VAR != kLBGK) {
        if (a.fix_list) record_fix_mask<NV>(hits, y * a.nx + x0, a);
    }
    if (bad) *a.flag = 1;
    const long long o = (long long)y * a.nx + x0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        if constexpr (std::is_same<C, CodecF16>::value && NV % 2 == 0) {
            unsigned pk[NV / 2];
#pragma unroll
            for (int k = 0; k < NV; k += 2) pk[k / 2] = C::store2(f[k][i], f[k + 1][i], i, a.cs);
            Vec<unsigned, NV / 2>::store(reinterpret_cast<unsigned*>(dst + (long long)i * a.plane + o), pk);
        } else {
            S out[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) out[k] = C::store(f[k][i], i, a.cs);
            Vec<S, NV>::store(dst + (long long)i * a.plane + o, out);
        }
    }
}

// ---------------------------------------------------------------- step, nodes
//
// One node per thread, any nx, ny; same arithmetic as step_rows.
template <int VAR, class C>
__global__ void __launch_bounds__(256)
step_nodes(const typename C::S* __restrict__ src, typename C::S* __restrict__ dst, StepArgs a)
{
    using S = typename C::S;
    using T = typename C::T;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.fix_count) a.fix_count[a.fix_slot ^ 1] = 0;
    const long long total = (long long)a.nx * a.ny;
    const CollideParams<T>& p = params_of<T>(a);
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < total;
         n += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(n / a.nx), x = (int)(n - (long long)y * a.nx);
        T f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ai = i % 3 - 1, bi = i / 3 - 1;
            int sx = x - ai, sy = y - bi;
            sx = sx < 0 ? sx + a.nx : (sx >= a.nx ? sx - a.nx : sx);
            sy = pull_row(sy, a);
            f[i] = C::load(__ldg(src + (long long)i * a.plane + (long long)sy * a.nx + sx), i, a.cs);
        }
        T rho;
        bool hit;
        collide_node<VAR, C::kUnits>(f, p, rho, hit);
        if (!isfinite(rho)) *a.flag = 1;
        if constexpr (VAR != kLBGK) {
            if (a.fix_list) record_fix(hit, (int)n, a);
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) dst[(long long)i * a.plane + n] = C::store(f[i], i, a.cs);
    }
}

// ---------------------------------------------------------------- all-FP64 step
//
// One node per thread with the whole collision in double whatever the
// storage; used for the exact-gamma mode (root of Eq. result1), whose Newton
// iteration runs in double.
template <int VAR, class C>
__global__ void __launch_bounds__(256)
step_nodes_f64(const typename C::S* __restrict__ src, typename C::S* __restrict__ dst, StepArgs a)
{
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.fix_count) a.fix_count[a.fix_slot ^ 1] = 0;
    const long long total = (long long)a.nx * a.ny;
    CollideParams<double> p = a.pd;
    p.guard = 0.0;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < total;
         n += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(n / a.nx), x = (int)(n - (long long)y * a.nx);
        double f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ai = i % 3 - 1, bi = i / 3 - 1;
            int sx = x - ai, sy = y - bi;
            sx = sx < 0 ? sx + a.nx : (sx >= a.nx ? sx - a.nx : sx);
            sy = pull_row(sy, a);
            f[i] = C::to_f64(src[(long long)i * a.plane + (long long)sy * a.nx + sx], i, a.cs);
        }
        double rho;
        bool hit;
        collide_node<VAR>(f, p, rho, hit);
        if (!isfinite(rho)) *a.flag = 1;
#pragma unroll
        for (int i = 0; i < 9; ++i) dst[(long long)i * a.plane + n] = C::from_f64(f[i], i, a.cs);
    }
}

// ---------------------------------------------------------------- FP64 re-evaluation
//
// Recomputes, entirely in double, the nodes the step recorded (entropic
// denominator at or below the guard) from the same source field, and
// overwrites their stored result.
template <int VAR, class C>
__global__ void __launch_bounds__(256)
step_fixup(const typename C::S* __restrict__ src, typename C::S* __restrict__ dst, StepArgs a)
{
    using S = typename C::S;
    const int recorded = a.fix_count[a.fix_slot];
    const int count = recorded < a.nx * a.ny ? recorded : a.nx * a.ny;
    if (count == 0) return;
    // node t goes to block t % gridDim.x: the few recorded nodes spread over
    // every SM's FP64 pipe instead of filling the first blocks
    for (int t = threadIdx.x * gridDim.x + blockIdx.x; t < count; t += gridDim.x * blockDim.x) {
        const int n = a.fix_list[t];
        const int y = n / a.nx, x = n - y * a.nx;
        double f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ai = i % 3 - 1, bi = i / 3 - 1;
            int sx = x - ai, sy = y - bi;
            sx = sx < 0 ? sx + a.nx : (sx >= a.nx ? sx - a.nx : sx);
            sy = pull_row(sy, a);
            f[i] = C::to_f64(src[(long long)i * a.plane + (long long)sy * a.nx + sx], i, a.cs);
        }
        CollideParams<double> q = a.pd;
        q.guard = 0.0;
        double rho;
        bool hit;
        collide_node<VAR>(f, q, rho, hit);
#pragma unroll
        for (int i = 0; i < 9; ++i) dst[(long long)i * a.plane + n] = C::from_f64(f[i], i, a.cs);
    }
}

// ---------------------------------------------------------------- init / io

// f = f^eq(rho, u) (Eq. Eq) stored as deviations from W_i; computed in double.
template <class C>
__global__ void init_feq(const double* __restrict__ rho, const double* __restrict__ ux,
                         const double* __restrict__ uy, typename C::S* __restrict__ dst,
                         StepArgs a)
{
    const long long total = (long long)a.nx * a.ny;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < total;
         n += (long long)gridDim.x * blockDim.x) {
        const double r = rho[n], x = ux[n], y = uy[n];
        const double usq15 = 1.5 * (x * x + y * y);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double xi = va(i) * x + vb(i) * y;
            const double P = xi * (3.0 + 4.5 * xi) - usq15;
            const double dev = wgt(i) * ((r - 1.0) + r * P);
            dst[(long long)i * a.plane + n] = C::from_f64(dev, i, a.cs);
        }
    }
}

// Grad's approximation (Eq. Grad) with Pi = Pi^eq + Pi^(1) (Eq. Peq,
// Eq. P1AC), velocity gradients by periodic central differences.
template <class C>
__global__ void init_grad(const double* __restrict__ rho, const double* __restrict__ ux,
                          const double* __restrict__ uy, typename C::S* __restrict__ dst,
                          StepArgs a)
{
    const long long total = (long long)a.nx * a.ny;
    // cs^2 = 1/3: the divisions by cs^2 and 2 cs^4 of Eq. Grad are the
    // multiplications by 3 and 4.5 (double division is many FP64-pipe
    // instructions, and this kernel is bound by that pipe)
    const double cs2 = 1.0 / 3.0;
    const double half_inv_beta = 0.5 / a.beta;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < total;
         n += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(n / a.nx), x = (int)(n - (long long)y * a.nx);
        const long long row = (long long)y * a.nx;
        const long long xp = row + (x + 1 == a.nx ? 0 : x + 1);
        const long long xm = row + (x == 0 ? a.nx - 1 : x - 1);
        const long long yp = (long long)(y + 1 == a.ny ? 0 : y + 1) * a.nx + x;
        const long long ym = (long long)(y == 0 ? a.ny - 1 : y - 1) * a.nx + x;
        // du[a][b] = d u_b / d x_a
        const double dxux = 0.5 * (ux[xp] - ux[xm]), dxuy = 0.5 * (uy[xp] - uy[xm]);
        const double dyux = 0.5 * (ux[yp] - ux[ym]), dyuy = 0.5 * (uy[yp] - uy[ym]);
        const double r = rho[n], u0 = ux[n], u1 = uy[n];
        const double c = r * cs2 * half_inv_beta;
        // non-equilibrium-shifted stress minus the isotropic part rho cs2 delta
        const double sxx = r * u0 * u0 - c * 2.0 * dxux;
        const double syy = r * u1 * u1 - c * 2.0 * dyuy;
        const double sxy = r * u0 * u1 - c * (dxuy + dyux);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double vx = va(i), vy = vb(i);
            const double lin = 3.0 * r * (u0 * vx + u1 * vy);
            const double quad = sxx * (vx * vx - cs2) + syy * (vy * vy - cs2) + 2.0 * sxy * vx * vy;
            const double fi = wgt(i) * (r + lin + 4.5 * quad);
            dst[(long long)i * a.plane + n] = C::from_f64(fi - wgt(i), i, a.cs);
        }
    }
}

template <class C>
__global__ void set_populations(const double* __restrict__ f, typename C::S* __restrict__ dst,
                                StepArgs a)
{
    const long long total = (long long)a.nx * a.ny;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < total;
         n += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < 9; ++i)
            dst[(long long)i * a.plane + n] = C::from_f64(f[(long long)i * total + n] - wgt(i), i, a.cs);
    }
}

template <class C>
__global__ void get_populations(const typename C::S* __restrict__ src, double* __restrict__ f,
                                StepArgs a)
{
    const long long total = (long long)a.nx * a.ny;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < total;
         n += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < 9; ++i)
            f[(long long)i * total + n] = C::to_f64(src[(long long)i * a.plane + n], i, a.cs) + wgt(i);
    }
}

// f[k][9] = populations of node nodes[k]; bad indices set *bad and are skipped
template <class C>
__global__ void probe_nodes(const typename C::S* __restrict__ src, const long long* __restrict__ nodes,
                            int count, double* __restrict__ f, int* bad, StepArgs a)
{
    const long long total = (long long)a.nx * a.ny;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        const long long n = nodes[k];
        if (n < 0 || n >= total) {
            *bad = 1;
            continue;
        }
#pragma unroll
        for (int i = 0; i < 9; ++i)
            f[(long long)k * 9 + i] = C::to_f64(src[(long long)i * a.plane + n], i, a.cs) + wgt(i);
    }
}

// rho and u of every node in double (from the stored deviations)
template <class C>
__device__ __forceinline__ void node_macro(const typename C::S* __restrict__ src, long long n,
                                           const StepArgs& a, double& rho, double& ux, double& uy)
{
    double d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = C::to_f64(src[(long long)i * a.plane + n], i, a.cs);
    const double drho = ((d[0] + d[8]) + (d[2] + d[6])) + ((d[1] + d[7]) + (d[3] + d[5])) + d[4];
    const double jx = ((d[2] - d[0]) + (d[8] - d[6])) + (d[5] - d[3]);
    const double jy = ((d[6] - d[0]) + (d[8] - d[2])) + (d[7] - d[1]);
    rho = 1.0 + drho;
    const double irho = 1.0 / rho;  // one division for both components
    ux = jx * irho;
    uy = jy * irho;
}

template <class C>
__global__ void moments(const typename C::S* __restrict__ src, double* __restrict__ rho,
                        double* __restrict__ ux, double* __restrict__ uy, StepArgs a)
{
    const long long total = (long long)a.nx * a.ny;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < total;
         n += (long long)gridDim.x * blockDim.x) {
        double r, x, y;
        node_macro<C>(src, n, a, r, x, y);
        rho[n] = r;
        ux[n] = x;
        uy[n] = y;
    }
}

// ---------------------------------------------------------------- diagnostics
//
// Per block: FP64 partial sums of mass and momentum, the count, mean and sum
// of squared deviations (M2) of |u|^2/2 and of w^2/2, and gamma (sum, min,
// max) over a grid-stride range of nodes, written to part[block][11].  gamma
// is that of the collision the next step performs, evaluated in double.
// Means and M2 are accumulated per thread by Welford's update and combined
// across threads and blocks by Chan et al.'s pairwise formula, so the
// standard deviations need no E[x^2] - E[x]^2 difference (which cancels).
// Deterministic: fixed grid, fixed reduction order.
constexpr int kDiagParts = 11;
constexpr int kDiagBlock = 256;

// Welford's running update of (count n, mean m, M2 q) with one value x.
__device__ __forceinline__ void welford_add(double& n, double& m, double& q, double x)
{
    n += 1.0;
    const double d = x - m;
    m += d / n;
    q += d * (x - m);
}

// Chan, Golub and LeVeque's combination of two partial (n, m, q) sets: the
// second is folded into the first.  mb and qb belong to the same nb.
__device__ __forceinline__ void chan_merge(double na, double nb, double& ma, double& qa, double mb,
                                           double qb)
{
    const double n = na + nb;
    if (nb == 0.0) return;
    if (na == 0.0) {
        ma = mb;
        qa = qb;
        return;
    }
    const double d = mb - ma;
    ma += d * (nb / n);
    qa += qb + d * d * (na * nb / n);
}

// Tiles of the diagnostics kernels: kTileW x kTileH nodes per block
// iteration (two per thread), with rho and u computed once per position of
// the tile and its halo into shared memory (periodic wrap), so that the
// central-difference stencils read them there instead of recomputing them.
constexpr int kTileW = 64, kTileH = 8;

__device__ __forceinline__ int wrap_mod(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// Folds partial set b into partial set a of the diagnostics; element k of a
// set is at a[k * sa] (b[k * sb]).
__device__ __forceinline__ void diag_fold(double* a, int sa, const double* b, int sb)
{
    a[0] += b[0];
    a[sa] += b[sb];
    a[2 * sa] += b[2 * sb];
    const double na = a[3 * sa], nb = b[3 * sb];
    chan_merge(na, nb, a[4 * sa], a[5 * sa], b[4 * sb], b[5 * sb]);
    chan_merge(na, nb, a[6 * sa], a[7 * sa], b[6 * sb], b[7 * sb]);
    a[3 * sa] = na + nb;
    a[8 * sa] += b[8 * sb];
    a[9 * sa] = fmin(a[9 * sa], b[9 * sb]);
    a[10 * sa] = fmax(a[10 * sa], b[10 * sb]);
}

template <int VAR, class C>
__global__ void __launch_bounds__(kDiagBlock)
diag_partial(const typename C::S* __restrict__ src, double* __restrict__ part, StepArgs a)
{
    constexpr int HW = kTileW + 2, HH = kTileH + 2;  // one-node halo
    __shared__ double sr[HH][HW], sux[HH][HW], suy[HH][HW];
    // mass, px, py, n, mean and M2 of |u|^2/2, of w^2/2, gamma sum, min, max
    double acc[kDiagParts] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 1e300, -1e300};
    CollideParams<double> p = a.pd;
    p.guard = 0.0;
    const int ntx = (a.nx + kTileW - 1) / kTileW, nty = (a.ny + kTileH - 1) / kTileH;
    const long long ntiles = (long long)ntx * nty;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int x0 = (int)(tile % ntx) * kTileW, y0 = (int)(tile / ntx) * kTileH;
        __syncthreads();  // the previous tile's readers are done with the arrays
        for (int q = threadIdx.x; q < HH * HW; q += blockDim.x) {
            const int qy = q / HW, qx = q - qy * HW;
            const int gx = wrap_mod(x0 + qx - 1, a.nx);
            int gy = y0 + qy - 1;
            if (a.ywrap) {
                gy = wrap_mod(gy, a.ny);
            } else if (gy > a.ny) {  // y-slab: rows -1 and ny are ghost rows; beyond, unused
                sr[qy][qx] = sux[qy][qx] = suy[qy][qx] = 0.0;
                continue;
            }
            node_macro<C>(src, (long long)gy * a.nx + gx, a, sr[qy][qx], sux[qy][qx], suy[qy][qx]);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < kTileW * kTileH; k += blockDim.x) {
            const int ly = k / kTileW, lx = k - ly * kTileW;
            const int x = x0 + lx, y = y0 + ly;
            if (x >= a.nx || y >= a.ny) continue;
            const int cx = lx + 1, cy = ly + 1;
            const double r = sr[cy][cx], ux = sux[cy][cx], uy = suy[cy][cx];
            acc[0] += r;
            acc[1] += r * ux;
            acc[2] += r * uy;
            const double ke = 0.5 * (ux * ux + uy * uy);
            const double w = 0.5 * (suy[cy][cx + 1] - suy[cy][cx - 1]) - 0.5 * (sux[cy + 1][cx] - sux[cy - 1][cx]);
            const double zz = 0.5 * w * w;
            double cnt = acc[3];
            welford_add(cnt, acc[4], acc[5], ke);
            welford_add(acc[3], acc[6], acc[7], zz);
            double f[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int ai = i % 3 - 1, bi = i / 3 - 1;
                int sx = x - ai, sy = y - bi;
                sx = sx < 0 ? sx + a.nx : (sx >= a.nx ? sx - a.nx : sx);
                sy = pull_row(sy, a);
                f[i] = C::to_f64(src[(long long)i * a.plane + (long long)sy * a.nx + sx], i, a.cs);
            }
            double rr;
            bool hit;
            const double g = collide_node<VAR>(f, p, rr, hit);
            acc[8] += g;
            acc[9] = fmin(acc[9], g);
            acc[10] = fmax(acc[10], g);
        }
    }
    __shared__ double sm[kDiagParts][kDiagBlock];
#pragma unroll
    for (int k = 0; k < kDiagParts; ++k) sm[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = kDiagBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) diag_fold(&sm[0][threadIdx.x], kDiagBlock, &sm[0][threadIdx.x + s], kDiagBlock);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < kDiagParts; ++k) part[(long long)blockIdx.x * kDiagParts + k] = sm[k][0];
    }
}

// Palinstrophy and entropy density per block: part[block][5] = count, and
// the mean and M2 (Welford / Chan, as in diag_partial) of P = |grad w|^2 / 2
// (w and its gradient by periodic central differences, the same w as
// diag_partial) and of the entropy density of Eq. S,
// s = -sum_i f_i ln(f_i / W_i) = -sum_i f_i log1p(d_i / W_i).
constexpr int kDiagExtParts = 5;

__device__ __forceinline__ void diag_ext_fold(double* a, int sa, const double* b, int sb)
{
    const double na = a[0], nb = b[0];
    chan_merge(na, nb, a[sa], a[2 * sa], b[sb], b[2 * sb]);
    chan_merge(na, nb, a[3 * sa], a[4 * sa], b[3 * sb], b[4 * sb]);
    a[0] = na + nb;
}

template <class C>
__global__ void __launch_bounds__(kDiagBlock)
diag_ext_partial(const typename C::S* __restrict__ src, double* __restrict__ part, StepArgs a)
{
    // u on the tile with a two-node halo, w on the tile with a one-node halo
    constexpr int UW = kTileW + 4, UH = kTileH + 4, WW = kTileW + 2, WH = kTileH + 2;
    __shared__ double sux[UH][UW], suy[UH][UW], sw[WH][WW];
    double acc[kDiagExtParts] = {0, 0, 0, 0, 0};  // n, mean and M2 of P, of s
    const int ntx = (a.nx + kTileW - 1) / kTileW, nty = (a.ny + kTileH - 1) / kTileH;
    const long long ntiles = (long long)ntx * nty;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int x0 = (int)(tile % ntx) * kTileW, y0 = (int)(tile / ntx) * kTileH;
        __syncthreads();
        for (int q = threadIdx.x; q < UH * UW; q += blockDim.x) {
            const int qy = q / UW, qx = q - qy * UW;
            const int gx = wrap_mod(x0 + qx - 2, a.nx), gy = wrap_mod(y0 + qy - 2, a.ny);
            double r;
            node_macro<C>(src, (long long)gy * a.nx + gx, a, r, sux[qy][qx], suy[qy][qx]);
        }
        __syncthreads();
        // w = d uy/dx - d ux/dy by central differences
        for (int q = threadIdx.x; q < WH * WW; q += blockDim.x) {
            const int qy = q / WW, qx = q - qy * WW, cy = qy + 1, cx = qx + 1;
            sw[qy][qx] = 0.5 * (suy[cy][cx + 1] - suy[cy][cx - 1]) - 0.5 * (sux[cy + 1][cx] - sux[cy - 1][cx]);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < kTileW * kTileH; k += blockDim.x) {
            const int ly = k / kTileW, lx = k - ly * kTileW;
            const int x = x0 + lx, y = y0 + ly;
            if (x >= a.nx || y >= a.ny) continue;
            const int cx = lx + 1, cy = ly + 1;
            const double wx = 0.5 * (sw[cy][cx + 1] - sw[cy][cx - 1]);
            const double wy = 0.5 * (sw[cy + 1][cx] - sw[cy - 1][cx]);
            const double pp = 0.5 * (wx * wx + wy * wy);
            const long long n = (long long)y * a.nx + x;
            double se = 0.0;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const double d = C::to_f64(src[(long long)i * a.plane + n], i, a.cs);
                se -= (wgt(i) + d) * log1p(d * inv_wgt(i));
            }
            double cnt = acc[0];
            welford_add(cnt, acc[1], acc[2], pp);
            welford_add(acc[0], acc[3], acc[4], se);
        }
    }
    __shared__ double sm[kDiagExtParts][kDiagBlock];
#pragma unroll
    for (int k = 0; k < kDiagExtParts; ++k) sm[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = kDiagBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            diag_ext_fold(&sm[0][threadIdx.x], kDiagBlock, &sm[0][threadIdx.x + s], kDiagBlock);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < kDiagExtParts; ++k) part[(long long)blockIdx.x * kDiagExtParts + k] = sm[k][0];
    }
}

// Reduces part[nblocks][5] into out[4] = (mean P, std P, mean s, std s).
__global__ void diag_ext_final(const double* __restrict__ part, int nblocks,
                               double* __restrict__ out, long long total);

// Reduces part[nblocks][11] (fixed order) into out[KBC_DIAG_N], or with raw
// into the merged partial set out[11] (the layout of one block's part).
__global__ void diag_final(const double* __restrict__ part, int nblocks, double* __restrict__ out,
                           long long total, int raw);

}  // namespace kbc
