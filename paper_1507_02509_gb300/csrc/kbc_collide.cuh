// Per-node collision of the D2Q9 KBC / LBGK model, register-only.
//
// Input d[9] holds the pre-collision populations as deviations
// d_i = f_i - W_i; on return it holds the post-collision deviations.
//
// Steps (Bosch, Chikatamarla, Karlin):
//   rho = sum f, rho u = sum v f                                  (Sec. 1)
//   f^eq from Eq. Eq, formed directly as the deviation f^eq - W
//   df = f - f^eq
//   second moments of df; because df carries no mass and no momentum,
//   its central and natural second moments coincide, so only the basis
//   vectors below depend on the variant (Table 1, Eq. cm)
//   ds = the population carrying the variant's shear-moment deviations and
//        no other moment (central basis about u for A/B, natural for C/D;
//        this is Eq. momentsD2Q9 restricted to the s group, written with the
//        dual vectors E_pq(c) = e_p(c_x) x e_q(c_y) of the 1-D moment basis)
//   dh = df - ds                            (k carries no deviation, Sec. 5)
//   gamma* = 1/beta - (2 - 1/beta) <ds|dh>/<dh|dh>               (Eq. result21)
//   f' = f - beta (2 ds + gamma dh)                    (Eq. ksh-mirror in Eq. Egeneral)
// The last line is evaluated in the generalised-equilibrium arrangement of
// Eq. EGE / Eq. GE,
//   f' = f - 2 beta df - beta (gamma - 2) dh,
// so that gamma = 2 removes the h term exactly and reproduces the LBGK
// update f - 2 beta df (Eq. LBGKmirr) bit for bit.
#pragma once

#include <type_traits>

#include "kbc_lattice.cuh"

namespace kbc {

// Table 1
enum : int { kLBGK = 0, kA = 1, kB = 2, kC = 3, kD = 4 };

template <typename T>
struct CollideParams {
    T two_beta;        // 2 beta
    T one_m_2beta;     // 1 - 2 beta
    T inv_beta;        // 1 / beta
    T two_m_inv_beta;  // 2 - 1 / beta
    T ch_fixed;        // beta (gamma_fixed - 2)
    T gamma_fixed;
    T guard;           // threshold on rho <dh|dh>; <= 0 disables
    int fixed;         // 1: gamma = gamma_fixed
    int exact;         // 1: gamma from the root of Eq. result1 (double arithmetic only)
};

template <typename T>
__host__ inline CollideParams<T> make_params(double beta, int fixed, double gamma_fixed, double guard)
{
    CollideParams<T> p;
    p.two_beta = (T)(2.0 * beta);
    p.one_m_2beta = (T)(1.0 - 2.0 * beta);
    p.inv_beta = (T)(1.0 / beta);
    p.two_m_inv_beta = (T)(2.0 - 1.0 / beta);
    p.ch_fixed = (T)(beta * (gamma_fixed - 2.0));
    p.gamma_fixed = (T)gamma_fixed;
    p.guard = (T)guard;
    p.fixed = fixed == 1 ? 1 : 0;
    p.exact = fixed == 2 ? 1 : 0;
    return p;
}

// Fast reciprocal / quotient: float uses the approximate hardware path
// (__fdividef, 2 ulp); double the IEEE operations.
template <typename T> __device__ __forceinline__ T rcp_fast(T x);
template <> __device__ __forceinline__ float rcp_fast<float>(float x) { return __fdividef(1.0f, x); }
template <> __device__ __forceinline__ double rcp_fast<double>(double x) { return 1.0 / x; }

template <typename T> __device__ __forceinline__ T ratio(T a, T b);
template <> __device__ __forceinline__ float ratio<float>(float a, float b) { return __fdividef(a, b); }
template <> __device__ __forceinline__ double ratio<double>(double a, double b) { return a / b; }

// xi_i = v_i . u for a compile-time velocity (a, b)
template <int A, int B, typename T>
__device__ __forceinline__ T vdot(T ux, T uy)
{
    if constexpr (A == 0 && B == 0) return T(0);
    else if constexpr (A == 0) return B > 0 ? uy : -uy;
    else if constexpr (B == 0) return A > 0 ? ux : -ux;
    else return (A > 0 ? ux : -ux) + (B > 0 ? uy : -uy);
}

// P_i = 3 xi + 4.5 xi^2 - 1.5 u^2, so that f^eq_i = W_i rho (1 + P_i) (Eq. Eq)
template <int I, typename T>
__device__ __forceinline__ T eq_poly(T ux, T uy, T usq15)
{
    constexpr int A = I % 3 - 1, B = I / 3 - 1;
    if constexpr (A == 0 && B == 0) {
        return -usq15;
    } else {
        const T xi = vdot<A, B>(ux, uy);
        return fmaT(xi, fmaT(T(4.5), xi, T(3)), -usq15);
    }
}

// df_i = d_i - (f^eq_i - W_i), with f^eq - W = W (rho - 1 + rho P)
template <int I, typename T>
__device__ __forceinline__ T neq(T d, T rho, T drho, T P)
{
    return d - T(wgt(I)) * fmaT(rho, P, drho);
}

// Montgomery's simultaneous inversion: w_i = 1 / x_i for nine x_i with one
// reciprocal and 24 multiplications.
template <typename T>
__device__ __forceinline__ void inv9(const T (&x)[9], T (&w)[9])
{
    T pre[9];
    pre[0] = x[0];
#pragma unroll
    for (int k = 1; k < 9; ++k) pre[k] = pre[k - 1] * x[k];
    T inv = rcp_fast(pre[8]);
#pragma unroll
    for (int k = 8; k >= 1; --k) {
        w[k] = inv * pre[k - 1];
        inv = inv * x[k];
    }
    w[0] = inv;
}

// Root of the exact entropic condition Eq. result1,
//   F(g) = sum_i dh_i ln(1 + ((1 - beta g) dh_i - (2 beta - 1) ds_i) / f^eq_i) = 0,
// by Newton's method from gamma* (F is decreasing wherever every
// post-collision population is positive: F'(g) = -beta sum dh_i^2 / f'_i).
// Stops when the step is below 1e-13 |g|; keeps gamma* when an iterate leaves
// that domain, F' is not negative, or 30 iterations pass.  w_i = rho / f^eq_i.
__device__ __forceinline__ double exact_gamma(const double (&ds)[9], const double (&dh)[9],
                                              const double (&w)[9], double rho, double beta,
                                              double g0)
{
    const double irho = 1.0 / rho;
    double g = g0;
    for (int it = 0; it < 30; ++it) {
        double F = 0.0, dF = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double q = w[i] * irho;  // 1 / f^eq_i
            const double x = ((1.0 - beta * g) * dh[i] - (2.0 * beta - 1.0) * ds[i]) * q;
            if (!(x > -1.0)) return g0;
            F += dh[i] * log1p(x);
            dF -= beta * dh[i] * dh[i] * q / (1.0 + x);
        }
        if (!(dF < 0.0)) return g0;
        const double step = F / dF;
        g -= step;
        if (fabs(step) <= 1e-13 * fabs(g)) return g;
    }
    return g0;
}

// Returns gamma; rho_out receives rho (NaN/Inf flags a blown-up node);
// guard_hit is set when the entropic denominator falls to or below the guard.
//
// Only six non-equilibrium parts are formed from the equilibrium; the other
// three follow from sum df = sum a df = sum b df = 0 (the collision
// conserves rho and rho u).  The rounding of f^eq (about eps |f^eq - W|)
// then never leaks into the conserved moments, where nothing would damp it.
template <int VAR, typename T>
__device__ __forceinline__ T collide(T (&d)[9], const CollideParams<T>& p, T& rho_out,
                                     bool& guard_hit)
{
    const T drho = ((d[0] + d[8]) + (d[2] + d[6])) + ((d[1] + d[7]) + (d[3] + d[5])) + d[4];
    const T jx = ((d[2] - d[0]) + (d[8] - d[6])) + (d[5] - d[3]);
    const T jy = ((d[6] - d[0]) + (d[8] - d[2])) + (d[7] - d[1]);
    const T rho = T(1) + drho;
    rho_out = rho;
    const T irho = rcp_fast(rho);
    const T ux = jx * irho, uy = jy * irho;
    const T usq15 = T(1.5) * fmaT(ux, ux, uy * uy);

    T P[9], df[9];
    P[0] = eq_poly<0>(ux, uy, usq15);
    P[1] = eq_poly<1>(ux, uy, usq15);
    P[2] = eq_poly<2>(ux, uy, usq15);
    P[3] = eq_poly<3>(ux, uy, usq15);
    P[6] = eq_poly<6>(ux, uy, usq15);
    P[8] = eq_poly<8>(ux, uy, usq15);
    df[0] = neq<0>(d[0], rho, drho, P[0]);
    df[1] = neq<1>(d[1], rho, drho, P[1]);
    df[2] = neq<2>(d[2], rho, drho, P[2]);
    df[3] = neq<3>(d[3], rho, drho, P[3]);
    df[6] = neq<6>(d[6], rho, drho, P[6]);
    df[8] = neq<8>(d[8], rho, drho, P[8]);
    df[5] = (df[3] - (df[2] + df[8])) + (df[0] + df[6]);
    df[7] = (df[1] - (df[6] + df[8])) + (df[0] + df[2]);
    df[4] = -(((df[0] + df[8]) + (df[2] + df[6])) + ((df[1] + df[7]) + (df[3] + df[5])));

    if constexpr (VAR == kLBGK) {
        guard_hit = false;
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = fmaT(-p.two_beta, df[i], d[i]);
        return T(2);
    } else {
        // second moments of df (natural = central, see header)
        const T corner = (df[0] + df[2]) + (df[6] + df[8]);
        const T m20 = corner + (df[3] + df[5]);
        const T m02 = corner + (df[1] + df[7]);
        const T m11 = (df[0] + df[8]) - (df[2] + df[6]);
        // coefficients of E20, E02, E11 in ds: A/C carry T, N, Pi (all three
        // second moments); B/D carry N and Pi only, i.e. the traceless part
        // (m20 - m02)/2 (E20 - E02)
        T c20, c02;
        if constexpr (VAR == kA || VAR == kC) {
            c20 = m20;
            c02 = m02;
        } else {
            c20 = T(0.5) * (m20 - m02);
            c02 = -c20;
        }
        T ds[9];
        if constexpr (VAR == kA || VAR == kB) {
            // 1-D dual vectors about c: e0(c) = (c(c-1)/2, 1-c^2, c(c+1)/2),
            // e1(c) = (c-1/2, -2c, c+1/2), e2 = (1/2, -1, 1/2)
            const T hx = T(0.5) * ux, hy = T(0.5) * uy;
            const T e0x[3] = {fmaT(hx, ux, -hx), fmaT(-ux, ux, T(1)), fmaT(hx, ux, hx)};
            const T e0y[3] = {fmaT(hy, uy, -hy), fmaT(-uy, uy, T(1)), fmaT(hy, uy, hy)};
            const T e1x[3] = {ux - T(0.5), T(-2) * ux, ux + T(0.5)};
            const T e1y[3] = {uy - T(0.5), T(-2) * uy, uy + T(0.5)};
            // ds_(a,b) = c20 e2[a] e0y[b] + c02 e0x[a] e2[b] + m11 e1x[a] e1y[b]
            T Ab[3], Ba[3], Ca[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                Ab[k] = c20 * e0y[k];
                Ba[k] = c02 * e0x[k];
                Ca[k] = m11 * e1x[k];
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int a = i % 3, b = i / 3;  // a, b in {0,1,2} <-> {-1,0,1}
                const T ta = (a == 1) ? -Ab[b] : T(0.5) * Ab[b];
                const T tb = (b == 1) ? -Ba[a] : T(0.5) * Ba[a];
                ds[i] = fmaT(Ca[a], e1y[b], ta + tb);
            }
        } else {
            // natural basis (c = 0): e0 = (0,1,0), e1 = (-1/2, 0, 1/2)
            const T q = T(0.25) * m11;
            ds[4] = -(c20 + c02);
            ds[3] = ds[5] = T(0.5) * c20;
            ds[1] = ds[7] = T(0.5) * c02;
            ds[0] = ds[8] = q;
            ds[2] = ds[6] = -q;
        }
        P[4] = eq_poly<4>(ux, uy, usq15);
        P[5] = eq_poly<5>(ux, uy, usq15);
        P[7] = eq_poly<7>(ux, uy, usq15);
        T x[9], w[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) x[i] = fmaT(T(wgt(i)), P[i], T(wgt(i)));  // f^eq_i / rho
        inv9(x, w);  // w_i = rho / f^eq_i
        T dh[9];
        T sh = T(0), hh = T(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            dh[i] = df[i] - ds[i];
            const T t = dh[i] * w[i];
            sh = fmaT(ds[i], t, sh);
            hh = fmaT(dh[i], t, hh);
        }
        T ch, gamma;
        guard_hit = false;
        if (p.fixed) {
            ch = p.ch_fixed;
            gamma = p.gamma_fixed;
        } else {
            guard_hit = (p.guard > T(0)) && !(hh > p.guard);
            if (hh > T(0)) {
                const T R = ratio(sh, hh);
                ch = p.one_m_2beta * (T(1) + R);             // beta (gamma - 2)
                gamma = fmaT(-p.two_m_inv_beta, R, p.inv_beta);
                if constexpr (std::is_same<T, double>::value) {
                    if (p.exact) {
                        const double beta = 0.5 * p.two_beta;
                        gamma = exact_gamma(ds, dh, w, rho, beta, gamma);
                        ch = beta * (gamma - 2.0);
                    }
                }
            } else {
                // <dh|dh> = 0: dh = 0 and gamma multiplies nothing; report 2
                ch = T(0);
                gamma = T(2);
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = fmaT(-ch, dh[i], fmaT(-p.two_beta, df[i], d[i]));
        return gamma;
    }
}

}  // namespace kbc
