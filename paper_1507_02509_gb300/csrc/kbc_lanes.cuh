// Arithmetic lanes of the collision.
//
// Every lane operation is one explicitly rounded IEEE operation (add, sub,
// mul, fma with round-to-nearest) that the compiler never contracts into a
// fused multiply-add or reorders.  Each kernel that inlines the collision
// therefore evaluates exactly the operation sequence written in it, whatever
// the surrounding code, and all step kernels produce identical bits.
#pragma once

#include <cuda_runtime.h>
#include <type_traits>

namespace kbc {

struct Lf {
    using S = float;
    static constexpr int kLanes = 1;
    float v;
    Lf() = default;
    __device__ __forceinline__ explicit Lf(float x) : v(x) {}
    __device__ __forceinline__ explicit Lf(double c) : v((float)c) {}
    __device__ __forceinline__ explicit Lf(int c) : v((float)c) {}
    __device__ __forceinline__ float get(int) const { return v; }
};

struct Ld {
    using S = double;
    static constexpr int kLanes = 1;
    double v;
    Ld() = default;
    __device__ __forceinline__ explicit Ld(double x) : v(x) {}
    __device__ __forceinline__ explicit Ld(int c) : v((double)c) {}
    __device__ __forceinline__ double get(int) const { return v; }
};

// ---- Lf
__device__ __forceinline__ Lf operator+(Lf a, Lf b) { return Lf(__fadd_rn(a.v, b.v)); }
__device__ __forceinline__ Lf operator-(Lf a, Lf b) { return Lf(__fsub_rn(a.v, b.v)); }
__device__ __forceinline__ Lf operator*(Lf a, Lf b) { return Lf(__fmul_rn(a.v, b.v)); }
__device__ __forceinline__ Lf operator-(Lf a) { return Lf(-a.v); }
__device__ __forceinline__ Lf fmaL(Lf a, Lf b, Lf c) { return Lf(__fmaf_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ Lf rcp_fast(Lf x) { return Lf(__fdividef(1.0f, x.v)); }
__device__ __forceinline__ Lf ratio(Lf a, Lf b) { return Lf(__fdividef(a.v, b.v)); }
__device__ __forceinline__ unsigned gt_mask(Lf a, Lf b) { return a.v > b.v ? 1u : 0u; }
__device__ __forceinline__ unsigned finite_mask(Lf a) { return isfinite(a.v) ? 1u : 0u; }
__device__ __forceinline__ Lf select(unsigned m, Lf a, Lf b) { return (m & 1u) ? a : b; }

// ---- Ld
__device__ __forceinline__ Ld operator+(Ld a, Ld b) { return Ld(__dadd_rn(a.v, b.v)); }
__device__ __forceinline__ Ld operator-(Ld a, Ld b) { return Ld(__dsub_rn(a.v, b.v)); }
__device__ __forceinline__ Ld operator*(Ld a, Ld b) { return Ld(__dmul_rn(a.v, b.v)); }
__device__ __forceinline__ Ld operator-(Ld a) { return Ld(-a.v); }
__device__ __forceinline__ Ld fmaL(Ld a, Ld b, Ld c) { return Ld(__fma_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ Ld rcp_fast(Ld x) { return Ld(__drcp_rn(x.v)); }
// a / b as a times the correctly rounded reciprocal of b (two roundings; in
// the double collision it forms gamma*'s ratio <ds|dh> / <dh|dh>): 1.1% more
// FP64 KBC B throughput than the correctly rounded quotient on GB300, whose
// FP64 pipe bounds that path
__device__ __forceinline__ Ld ratio(Ld a, Ld b) { return Ld(__dmul_rn(a.v, __drcp_rn(b.v))); }
__device__ __forceinline__ unsigned gt_mask(Ld a, Ld b) { return a.v > b.v ? 1u : 0u; }
__device__ __forceinline__ unsigned finite_mask(Ld a) { return isfinite(a.v) ? 1u : 0u; }
__device__ __forceinline__ Ld select(unsigned m, Ld a, Ld b) { return (m & 1u) ? a : b; }

// ---- Lf2: two nodes in one packed pair of floats.  The sm_100-family
// FP32x2 operations (compiler builtins) round each component exactly as the
// one-node operation does -- add, mul and fma; a - b is a + (-b), the same
// IEEE result -- so a kernel that collides node pairs reproduces the
// one-node bits while issuing one instruction per two additions,
// multiplications or fused multiply-adds.  Unlike the one-node
// intrinsics, a packed product whose only use is a packed addition may be
// fused with it into one fma (measured; also when written as PTX with an
// explicit .rn); the collision therefore leaves no product as the sole
// operand of an addition on the packed path.  Reciprocals, quotients and
// comparisons are per component.
struct Lf2 {
    using S = float;
    static constexpr int kLanes = 2;
    float2 v;
    Lf2() = default;
    __device__ __forceinline__ Lf2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit Lf2(float2 x) : v(x) {}
    __device__ __forceinline__ explicit Lf2(float x) : v(make_float2(x, x)) {}
    __device__ __forceinline__ explicit Lf2(double c) : v(make_float2((float)c, (float)c)) {}
    __device__ __forceinline__ explicit Lf2(int c) : v(make_float2((float)c, (float)c)) {}
    __device__ __forceinline__ float lo() const { return v.x; }
    __device__ __forceinline__ float hi() const { return v.y; }
    __device__ __forceinline__ float get(int k) const { return k ? v.y : v.x; }
};

__device__ __forceinline__ Lf2 operator+(Lf2 a, Lf2 b) { return Lf2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ Lf2 operator-(Lf2 a) { return Lf2(-a.v.x, -a.v.y); }
__device__ __forceinline__ Lf2 operator-(Lf2 a, Lf2 b) { return Lf2(__fadd2_rn(a.v, (-b).v)); }
__device__ __forceinline__ Lf2 operator*(Lf2 a, Lf2 b) { return Lf2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ Lf2 fmaL(Lf2 a, Lf2 b, Lf2 c) { return Lf2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ Lf2 rcp_fast(Lf2 x)
{
    return Lf2(__fdividef(1.0f, x.v.x), __fdividef(1.0f, x.v.y));
}
__device__ __forceinline__ Lf2 ratio(Lf2 a, Lf2 b)
{
    return Lf2(__fdividef(a.v.x, b.v.x), __fdividef(a.v.y, b.v.y));
}
__device__ __forceinline__ unsigned gt_mask(Lf2 a, Lf2 b)
{
    return (a.v.x > b.v.x ? 1u : 0u) | (a.v.y > b.v.y ? 2u : 0u);
}
__device__ __forceinline__ unsigned finite_mask(Lf2 a)
{
    return (isfinite(a.v.x) ? 1u : 0u) | (isfinite(a.v.y) ? 2u : 0u);
}
__device__ __forceinline__ Lf2 select(unsigned m, Lf2 a, Lf2 b)
{
    return Lf2((m & 1u) ? a.v.x : b.v.x, (m & 2u) ? a.v.y : b.v.y);
}

// scalar arithmetic type -> one-node lane
template <typename T> struct LaneOf;
template <> struct LaneOf<float> { using type = Lf; };
template <> struct LaneOf<double> { using type = Ld; };

}  // namespace kbc
