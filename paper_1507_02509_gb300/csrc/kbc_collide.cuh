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
//        dual vectors E_pq(c) = e_p(c_x) x e_q(c_y) of the 1-D moment basis;
//        for A/B the central moments are first shifted to natural ones)
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

#include "kbc_lanes.cuh"
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
    T unit_s;          // storage units (FP16): S, with d_i = e_i W_i / S
    T unit_c;          // 1 / (36 S), the unit of the diagonal populations
    T guard_u;         // the guard threshold in those units, guard (36 S)^2
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
    p.unit_s = (T)1;
    p.unit_c = (T)1;
    p.guard_u = (T)guard;
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

// P_i = 3 xi + 4.5 xi^2 - 1.5 u^2 with xi = v_i . u, so that
// f^eq_i = W_i rho (1 + P_i) (Eq. Eq).  Opposite velocities share one xi:
// P(-xi) = xi (4.5 xi - 3) - 1.5 u^2, so no negated operand is formed.
// sxy = ux + uy, dxy = ux - uy, nusq15 = -1.5 |u|^2.
template <int I, class L>
__device__ __forceinline__ L eq_poly(L ux, L uy, L sxy, L dxy, L nusq15)
{
    constexpr int A = I % 3 - 1, B = I / 3 - 1;
    if constexpr (A == 0 && B == 0) {
        return nusq15;
    } else {
        constexpr int sgn = (A == 0) ? B : A;  // sign of v_i . u relative to xi below
        const L xi = (A == 0) ? uy : (B == 0) ? ux : (A == B) ? sxy : dxy;
        return fmaL(xi, fmaL(L(4.5), xi, L(3 * sgn)), nusq15);
    }
}

// storage-unit multiplicity m_i = 36 W_i: 1 (diagonal), 4 (axis), 16 (rest)
__host__ __device__ constexpr double unit_m(int i)
{
    return (va(i) != 0 && vb(i) != 0) ? 1.0 : (va(i) == 0 && vb(i) == 0) ? 16.0 : 4.0;
}

// df_i = d_i - (f^eq_i - W_i), with f^eq - W = W (rho - 1 + rho P); in
// storage units (d_i = e_i W_i / S) the factor W_i becomes S for every i
template <int I, bool U, class L>
__device__ __forceinline__ L neq(L d, L rho, L drho, L P, L unit_s)
{
    if constexpr (U) return fmaL(-unit_s, fmaL(rho, P, drho), d);
    else return fmaL(L(-wgt(I)), fmaL(rho, P, drho), d);
}

// Montgomery's simultaneous inversion: w_i = 1 / x_i for nine x_i with one
// reciprocal and 24 multiplications.  The weights enter gamma* only through
// the ratio <ds|dh> / <dh|dh>, so the rounding of the single shared
// reciprocal cancels there; nine independent approximate reciprocals do not
// (measured: three times the FP32-FP64 divergence of a turbulent run and a
// much noisier FP32 adjoint).
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

// Collision of one node in a lane type (Lf: float, Ld: double).  Returns
// gamma; rho_out receives rho (NaN/Inf flags a blown-up node); guard_hits is
// 1 when the entropic denominator falls to or below the guard.
//
// Only six non-equilibrium parts are formed from the equilibrium; the other
// three follow from sum df = sum a df = sum b df = 0 (the collision
// conserves rho and rho u).  The rounding of f^eq (about eps |f^eq - W|)
// then never leaks into the conserved moments, where nothing would damp it.
//
// U (storage units, FP16 only): d_i holds e_i = (f_i - W_i) S / W_i, the
// half-precision code itself, and so do df, ds, dh and the result.  With
// c = 1/(36 S) the deviation is c m_i e_i, m_i = 36 W_i = 1, 4, 16 (diagonal,
// axis, rest), exact powers of two: the moment sums weight e_i by m_i, the
// second moments and ds come out in units of c and are divided by m_i in
// their constants, and the entropic weights become m_i^2 rho / f^eq_i, which
// scales <ds|dh> and <dh|dh> alike by 1/c^2 (the guard threshold with them).
// The codec then needs no multiplication on either side.
template <int VAR, class L, bool U = false>
__device__ __forceinline__ L collide(L (&d)[9], const CollideParams<typename L::S>& p, L& rho_out,
                                     unsigned& guard_hits)
{
    constexpr bool dbl = std::is_same<typename L::S, double>::value;
    static_assert(!(U && dbl), "storage units are a single-precision path");
    // column sums (a = +1, -1, 0) and row sums (b = +1, -1); in units, cM is
    // a quarter of the middle column
    L cR, cL, cM, rT, rB, drho, jx, jy;
    if constexpr (U) {
        cR = fmaL(L(4), d[5], d[2] + d[8]);
        cL = fmaL(L(4), d[3], d[0] + d[6]);
        cM = fmaL(L(4), d[4], d[1] + d[7]);
        rT = fmaL(L(4), d[7], d[6] + d[8]);
        rB = fmaL(L(4), d[1], d[0] + d[2]);
        drho = L(p.unit_c) * fmaL(L(4), cM, cR + cL);
    } else {
        cR = (d[2] + d[5]) + d[8];
        cL = (d[0] + d[3]) + d[6];
        cM = (d[1] + d[4]) + d[7];
        rT = (d[6] + d[7]) + d[8];
        rB = (d[0] + d[1]) + d[2];
        drho = (cR + cL) + cM;
    }
    jx = cR - cL;
    jy = rT - rB;
    const L rho = L(1) + drho;
    rho_out = rho;
    L irho = rcp_fast(rho);
    if constexpr (U) irho = irho * L(p.unit_c);  // j is in units of c
    const L ux = jx * irho, uy = jy * irho;
    const L uxx = ux * ux, uyy = uy * uy;
    // storage units also collide in packed node pairs (Lf2), where a packed
    // product whose only use is an addition may be fused with it into one
    // fma: there |u|^2 is formed by an explicit fma, the same operation in
    // both lane types (elsewhere every product has a second use or scales by
    // a power of two, exact either way)
    L nusq15;
    if constexpr (U) nusq15 = L(-1.5) * fmaL(ux, ux, uyy);
    else nusq15 = L(-1.5) * (uxx + uyy);
    const L sxy = ux + uy, dxy = ux - uy;

    L P[9], df[9];
    P[0] = eq_poly<0>(ux, uy, sxy, dxy, nusq15);
    P[1] = eq_poly<1>(ux, uy, sxy, dxy, nusq15);
    P[2] = eq_poly<2>(ux, uy, sxy, dxy, nusq15);
    P[3] = eq_poly<3>(ux, uy, sxy, dxy, nusq15);
    P[6] = eq_poly<6>(ux, uy, sxy, dxy, nusq15);
    P[8] = eq_poly<8>(ux, uy, sxy, dxy, nusq15);
    const L us(p.unit_s);
    df[0] = neq<0, U>(d[0], rho, drho, P[0], us);
    df[1] = neq<1, U>(d[1], rho, drho, P[1], us);
    df[2] = neq<2, U>(d[2], rho, drho, P[2], us);
    df[3] = neq<3, U>(d[3], rho, drho, P[3], us);
    df[6] = neq<6, U>(d[6], rho, drho, P[6], us);
    df[8] = neq<8, U>(d[8], rho, drho, P[8], us);
    // second moments of df; df carries no mass or momentum, so its central
    // and natural second moments coincide (see header)
    L m20, m02, s08, s26;
    if constexpr (U) {
        df[5] = fmaL(L(0.25), (df[0] + df[6]) - (df[2] + df[8]), df[3]);  // sum a m df = 0
        df[7] = fmaL(L(0.25), (df[0] + df[2]) - (df[6] + df[8]), df[1]);  // sum b m df = 0
        s08 = df[0] + df[8];
        s26 = df[2] + df[6];
        const L corner = s08 + s26, s17 = df[1] + df[7];
        m20 = fmaL(L(4), df[3] + df[5], corner);
        m02 = fmaL(L(4), s17, corner);
        df[4] = L(-0.0625) * fmaL(L(4), s17, m20);                      // sum m df = 0
    } else {
        df[5] = (df[3] - (df[2] + df[8])) + (df[0] + df[6]);  // sum a df = 0
        df[7] = (df[1] - (df[6] + df[8])) + (df[0] + df[2]);  // sum b df = 0
        s08 = df[0] + df[8];
        s26 = df[2] + df[6];
        const L corner = s08 + s26, s17 = df[1] + df[7];
        m20 = corner + (df[3] + df[5]);
        m02 = corner + s17;
        df[4] = -(m20 + s17);                                 // sum df = 0
    }

    const L n2b(-p.two_beta);
    if constexpr (VAR == kLBGK) {
        guard_hits = 0u;
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = fmaL(n2b, df[i], d[i]);
        return L(2);
    } else {
        const L m11 = s08 - s26;
        // ds carries the variant's second moments c20, c02, c11 = m11 and no
        // other moment: A/C carry T, N, Pi (c20 = m20, c02 = m02); B/D carry N
        // and Pi only, the traceless part c20 = -c02 = (m20 - m02)/2
        L ds[9];
        if constexpr (VAR == kA || VAR == kB) {
            // Central basis about c = u: the other central moments of ds
            // vanish.  The binomial shift a = (a - ux) + ux turns that into
            // natural moments (mass and momentum stay zero)
            //   M21 = uy c20 + 2 ux c11,  M12 = ux c02 + 2 uy c11,
            //   M22 = uy^2 c20 + ux^2 c02 + 4 ux uy c11,
            // and the natural dual vectors e0 = (0,1,0), e1 = (-1/2,0,1/2),
            // e2 = (1/2,-1,1/2) give the same population as the central ones
            // e_p(c) would, in about 30 operations instead of 46.  With
            // q = c/4 and Q = M/4:
            //   ds(0,0) = 4 (Q22 - q20 - q02),  ds(a,0) = 2 (q20 - Q22 - a Q12),
            //   ds(0,b) = 2 (q02 - Q22 - b Q21),
            //   ds(a,b) = Q22 + a Q12 + b Q21 + a b q11   (a, b = +-1)
            // (in storage units the centre and edge factors are divided by
            // m = 16 and 4)
            constexpr double kc = U ? 0.25 : 4.0, ke = U ? 0.5 : 2.0;
            L q20, q02;
            if constexpr (VAR == kA) {
                q20 = L(0.25) * m20;
                q02 = L(0.25) * m02;
            } else {
                q20 = L(0.125) * (m20 - m02);
                q02 = -q20;
            }
            const L q11 = L(0.25) * m11, h11 = L(0.5) * m11;
            const L Q21 = fmaL(ux, h11, uy * q20);
            const L Q12 = fmaL(uy, h11, ux * q02);
            const L Q22 = fmaL(uyy, q20, fmaL(uxx, q02, (ux * uy) * m11));
            if constexpr (VAR == kA) ds[4] = L(kc) * (Q22 - (q20 + q02));
            else ds[4] = L(kc) * Q22;  // q20 + q02 = 0
            const L ex2 = L(ke) * (q20 - Q22), ey2 = L(ke) * (q02 - Q22);
            ds[3] = fmaL(L(ke), Q12, ex2);
            ds[5] = fmaL(L(-ke), Q12, ex2);
            ds[1] = fmaL(L(ke), Q21, ey2);
            ds[7] = fmaL(L(-ke), Q21, ey2);
            const L sp = Q22 + Q12, sm = Q22 - Q12, rp = Q21 + q11, rm = Q21 - q11;
            ds[8] = sp + rp;
            ds[2] = sp - rp;
            ds[6] = sm + rm;
            ds[0] = sm - rm;
        } else {
            // natural basis (c = 0): e0 = (0,1,0), e1 = (-1/2, 0, 1/2);
            // hc = half the coefficient (a quarter of that in storage units,
            // where the edges are divided by m = 4 and the centre by 16)
            constexpr double kh = U ? 0.25 : 1.0;
            L hc20, hc02;
            if constexpr (VAR == kC) {
                hc20 = L(0.5 * kh) * m20;
                hc02 = L(0.5 * kh) * m02;
            } else {
                hc20 = L(0.25 * kh) * (m20 - m02);
                hc02 = -hc20;
            }
            const L q = L(0.25) * m11;
            ds[4] = L(U ? -0.5 : -2.0) * (hc20 + hc02);
            ds[3] = ds[5] = hc20;
            ds[1] = ds[7] = hc02;
            ds[0] = ds[8] = q;
            ds[2] = ds[6] = -q;
        }
        P[4] = nusq15;
        P[5] = eq_poly<5>(ux, uy, sxy, dxy, nusq15);
        P[7] = eq_poly<7>(ux, uy, sxy, dxy, nusq15);
        L x[9], w[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {  // f^eq_i / rho (over m_i^2 in storage units)
            const double wx = U ? 1.0 / (36.0 * unit_m(i)) : wgt(i);  // W_i / m_i^2
            x[i] = fmaL(L(wx), P[i], L(wx));
        }
        L xprod;  // double lanes: prod_i x_i, the common factor of their weights
        if constexpr (dbl) {
            // gamma* uses the weights only through <ds|dh> / <dh|dh>, which a
            // common factor leaves unchanged: w_i = prod_{j != i} x_j from
            // prefix and suffix products, with no division (the FP64 pipe is
            // the bound of the double path)
            L pre[8], suf[9];
            pre[0] = x[0];
#pragma unroll
            for (int k = 1; k < 8; ++k) pre[k] = pre[k - 1] * x[k];
            suf[8] = x[8];
#pragma unroll
            for (int k = 7; k >= 1; --k) suf[k] = suf[k + 1] * x[k];
            w[0] = suf[1];
            w[8] = pre[7];
#pragma unroll
            for (int k = 1; k < 8; ++k) w[k] = pre[k - 1] * suf[k + 1];
            xprod = pre[7] * x[8];
        } else {
            inv9(x, w);  // w_i = rho / f^eq_i
        }
        L dh[9];
        L sh, hh;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            dh[i] = df[i] - ds[i];
            const L t = dh[i] * w[i];
            if (i == 0) {
                sh = ds[0] * t;
                hh = dh[0] * t;
            } else {
                sh = fmaL(ds[i], t, sh);
                hh = fmaL(dh[i], t, hh);
            }
        }
        L nch, gamma;  // nch = -beta (gamma - 2)
        guard_hits = 0u;
        if (p.fixed) {
            nch = L(-p.ch_fixed);
            gamma = L(p.gamma_fixed);
        } else {
            // the guard concerns single precision (double lanes never flag)
            const typename L::S gthr = U ? p.guard_u : p.guard;
            if (!dbl && gthr > 0) guard_hits = ~gt_mask(hh, L(gthr)) & ((1u << L::kLanes) - 1u);
            // <dh|dh> = 0 means dh = 0: gamma multiplies nothing; report 2
            // (double lanes: the sign of <dh|dh> is that of hh * prod x)
            unsigned pos;
            if constexpr (dbl) pos = gt_mask(hh * xprod, L(0));
            else pos = gt_mask(hh, L(0));
            const L R = ratio(sh, hh);
            const L nb = L(-p.one_m_2beta);
            nch = select(pos, fmaL(nb, R, nb), L(0));
            gamma = select(pos, fmaL(L(-p.two_m_inv_beta), R, L(p.inv_beta)), L(2));
            if constexpr (std::is_same<L, Ld>::value) {
                if (p.exact && pos) {
                    double dsd[9], dhd[9], wd[9];
                    const double iprod = 1.0 / xprod.v;  // weights normalised: rho / f^eq_i
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        dsd[i] = ds[i].v;
                        dhd[i] = dh[i].v;
                        wd[i] = w[i].v * iprod;
                    }
                    const double beta = 0.5 * p.two_beta;
                    gamma = Ld(exact_gamma(dsd, dhd, wd, rho.v, beta, gamma.v));
                    nch = Ld(beta * (2.0 - gamma.v));
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = fmaL(nch, dh[i], fmaL(n2b, df[i], d[i]));
        return gamma;
    }
}

// One node in float or double (wraps the scalar into its lane type); U:
// f holds storage units (see collide).
template <int VAR, bool U = false, typename T>
__device__ __forceinline__ T collide_node(T (&f)[9], const CollideParams<T>& p, T& rho, bool& hit)
{
    using L = typename LaneOf<T>::type;
    L d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = L(f[i]);
    L r;
    unsigned h;
    const L g = collide<VAR, L, U>(d, p, r, h);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = d[i].v;
    rho = r.v;
    hit = (h & 1u) != 0u;
    return g.v;
}

// Two nodes in one packed lane pair (float only); the same bits as two
// collide_node calls.  hits: bit 0 / 1 for node 0 / 1.
template <int VAR, bool U = false>
__device__ __forceinline__ void collide_pair(float (&f0)[9], float (&f1)[9],
                                             const CollideParams<float>& p, float& rho0,
                                             float& rho1, unsigned& hits)
{
    Lf2 d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = Lf2(f0[i], f1[i]);
    Lf2 r;
    collide<VAR, Lf2, U>(d, p, r, hits);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        f0[i] = d[i].lo();
        f1[i] = d[i].hi();
    }
    rho0 = r.lo();
    rho1 = r.hi();
}

}  // namespace kbc
