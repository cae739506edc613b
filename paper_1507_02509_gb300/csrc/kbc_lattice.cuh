// D2Q9 lattice constants and storage codecs for the sm_103a kernels.
//
// Velocity set (Sec. 2): tensor product of {-1, 0, 1}; population index
// i = 3(b+1) + (a+1) for v_i = (a, b).  The weights W_i and cs^2 are not
// printed in the paper (Eq. S, Eq. Eq); the D2Q9 product weights
// W_(a,b) = w_a w_b with w_0 = 2/3, w_{+-1} = 1/6 and cs^2 = 1/3 are used.
//
// Populations are stored as deviations from the rest weights, d_i = f_i - W_i,
// which keeps O(u) information in the leading bits of low-precision storage.
#pragma once

#include <cuda_fp16.h>
#include <cstdint>

namespace kbc {

__host__ __device__ constexpr int va(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int vb(int i) { return i / 3 - 1; }
__host__ __device__ constexpr double w1(int a) { return a == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
__host__ __device__ constexpr double wgt(int i) { return w1(va(i)) * w1(vb(i)); }
// 1 / W_i: 36 (diagonal), 9 (axis), 9/4 (rest)
__host__ __device__ constexpr double inv_wgt(int i)
{
    return (va(i) != 0 && vb(i) != 0) ? 36.0 : (va(i) == 0 && vb(i) == 0) ? 2.25 : 9.0;
}

template <typename T> __device__ __forceinline__ T fmaT(T a, T b, T c);
template <> __device__ __forceinline__ float fmaT<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ double fmaT<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

// weight class of population i: 0 diagonal (W = 1/36), 1 axis (1/9), 2 rest (4/9)
__host__ __device__ constexpr int wclass(int i)
{
    return (va(i) != 0 && vb(i) != 0) ? 0 : (va(i) == 0 && vb(i) == 0) ? 2 : 1;
}

// Scale of the half-precision encoding (unused by the other codecs): S and,
// per weight class, the decode factor W/S, rounded once on the host so that
// the kernels take it from the parameter bank instead of forming it per
// thread.
struct CodecScale {
    float scale;      // S
    float inv_scale;  // 1 / S
    float dec[3];     // W_c / S
};

__host__ inline CodecScale make_scale(double s)
{
    const double w[3] = {1.0 / 36.0, 1.0 / 9.0, 4.0 / 9.0};
    CodecScale c;
    c.scale = (float)s;
    c.inv_scale = (float)(1.0 / s);
    for (int k = 0; k < 3; ++k) c.dec[k] = (float)(w[k] / s);
    return c;
}

// Storage codecs: S = stored element, T = arithmetic type.
//   decode(s, i, c)     -> d_i = f_i - W_i in T
//   load(s, i, c), store(e, i, c)
//                       -> the step kernels' view: the value the collision
//                          works on, d_i itself, or with kUnits the storage
//                          code in T (the collision's storage units)
//   to_f64(s, i, c)     -> d_i in double (exact for F64/F32 storage)
//   from_f64(d, i, c)   -> stored element from a double deviation
// kVec: nodes per thread of the vector-row kernel (kVec * sizeof(S) bytes
// per load/store; 16 for F64/F32, 8 for F16, which keeps F16 registers low).
// kRowMinBlocks: resident 64-thread blocks per SM the vector-row kernel is
// compiled for.  12 caps it at 80 registers (65536 / (12 * 64) = 85; every
// variant fits without spilling) and keeps 24 warps per SM loading: 3%
// faster than 96 registers for KBC B and 5% for C/D.  Left free,
// the compiler takes up to 190 registers and the bandwidth-bound FP32 step
// loses a third of its rate.  FP64 is bound by its arithmetic pipe, not by
// occupancy.
struct CodecF64 {
    using S = double;
    using T = double;
    static constexpr int kVec = 2;
    static constexpr int kRowMinBlocks = 1;
    static constexpr bool kUnits = false;
    __device__ __forceinline__ static T decode(S s, int, const CodecScale&) { return s; }
    __device__ __forceinline__ static T load(S s, int, const CodecScale&) { return s; }
    __device__ __forceinline__ static S store(T d, int, const CodecScale&) { return d; }
    __device__ __forceinline__ static double to_f64(S s, int, const CodecScale&) { return s; }
    __device__ __forceinline__ static S from_f64(double d, int, const CodecScale&) { return d; }
};

struct CodecF32 {
    using S = float;
    using T = float;
    static constexpr int kVec = 4;
    static constexpr int kRowMinBlocks = 12;
    static constexpr bool kUnits = false;
    __device__ __forceinline__ static T decode(S s, int, const CodecScale&) { return s; }
    __device__ __forceinline__ static T load(S s, int, const CodecScale&) { return s; }
    __device__ __forceinline__ static S store(T d, int, const CodecScale&) { return d; }
    __device__ __forceinline__ static double to_f64(S s, int, const CodecScale&) { return (double)s; }
    __device__ __forceinline__ static S from_f64(double d, int, const CodecScale&) { return __double2float_rn(d); }
};

// (f - W)/W * S in IEEE half (stored as its 16-bit pattern), arithmetic in
// float.  The step kernels collide in storage units: load and store are the
// bare conversions.
struct CodecF16 {
    using S = unsigned short;
    using T = float;
    static constexpr int kVec = 4;
    static constexpr int kRowMinBlocks = 12;
    static constexpr bool kUnits = true;
    __device__ __forceinline__ static T load(S s, int, const CodecScale&)
    {
        return __half2float(__ushort_as_half(s));
    }
    __device__ __forceinline__ static S store(T e, int, const CodecScale&)
    {
        return __half_as_ushort(__float2half_rn(e));
    }
    // two populations of the same plane in one packed conversion
    __device__ __forceinline__ static unsigned store2(T e0, T e1, int, const CodecScale&)
    {
        const __half2 h = __floats2half2_rn(e0, e1);
        return *reinterpret_cast<const unsigned*>(&h);
    }
    __device__ __forceinline__ static T decode(S s, int i, const CodecScale& c)
    {
        return __half2float(__ushort_as_half(s)) * c.dec[wclass(i)];
    }
    __device__ __forceinline__ static double to_f64(S s, int i, const CodecScale& c)
    {
        return (double)__half2float(__ushort_as_half(s)) * (wgt(i) * (double)c.inv_scale);
    }
    __device__ __forceinline__ static S from_f64(double d, int i, const CodecScale& c)
    {
        return __half_as_ushort(__double2half(d * (inv_wgt(i) * (double)c.scale)));
    }
};

}  // namespace kbc
