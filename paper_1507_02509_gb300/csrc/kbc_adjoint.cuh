// Discrete adjoint of the stream-collide step (not part of the paper; it
// gives gradients of an objective of the final field with respect to the
// initial velocity and beta).
//
// Forward map of one step: g^{n+1} = C(P g^n), P the periodic pull
// f_i(x) = g_i(x - v_i), C the per-node collision of kbc_collide.cuh.
// Reverse: lambda^n = P^T (dC/df)^T lambda^{n+1}, where P^T sends the
// adjoint of the population pulled from x - v_i back there, and
// dJ/dbeta = sum_n sum_x lambda^{n+1}(x) . dC/dbeta.
//
// collide_adjoint() is the hand-written reverse mode of collide(): it
// recomputes the forward quantities and propagates lambda back through the
// update f' = f - 2 beta df - beta (gamma - 2) dh, the entropic products and
// gamma* (Eq. result21, including the dependence of gamma on f), the split
// (Table 1 bases, with the velocity dependence of the central basis), the
// equilibrium (Eq. Eq) and the moments.  It differentiates the exact map:
// all nine non-equilibrium parts are taken from the equilibrium (the
// forward kernel derives three of them from conservation, which is the same
// function).
#pragma once

#include <type_traits>

#include "kbc_kernels.cuh"

namespace kbc {

// Threads per block of the reverse step, and resident blocks per SM it is
// compiled for: the natural-basis variants (C, D) fit 96 registers (5 blocks,
// 20 warps per SM) without spilling; the central-basis ones keep 128 (4
// blocks), where a 96-register cap spills and runs slower.  Measured at
// 4096^2 (200 steps, FP32): B 0.203 s with 256-thread blocks -> 0.199 s,
// C 0.197 s -> 0.185 s with the 96-register cap; 512^2: B 0.063 -> 0.055 s.
// Double arithmetic is bound by the FP64 pipe, not by occupancy: no cap.
constexpr int kAdjBlock = 128;
template <int VAR, typename T> constexpr int adj_min_blocks()
{
    return std::is_same<T, double>::value ? 1 : ((VAR == kC || VAR == kD) ? 5 : 4);
}

// Single-precision reverse collision in opposite-pair lanes: population
// pair k = 0..3 holds (i = k, i = 8 - k) in one packed FP32x2 lane (Lf2).
// The two members have velocities v and -v and the same weight, so every
// per-population step of the reverse (equilibrium, split, entropic
// products, their adjoints) is one packed operation for two populations,
// with sign pairs (a, -a), (b, -b) for the velocity components; the rest
// population i = 4 and the scalar moments stay scalar.  Same mathematics as
// the generic collide_adjoint below, in a different rounding order.
template <int VAR>
__device__ __forceinline__ bool collide_adjoint_pairs(const float (&d)[9], const float (&lam)[9],
                                                      const CollideParams<float>& p,
                                                      float (&mu)[9], float& beta_bar)
{
    using L = Lf2;
    constexpr bool central = (VAR == kA || VAR == kB);
    bool guarded = false;
    // ---------------------------------------------------------------- forward
    // the pairwise moment sums of the generic path
    const float drho = ((d[0] + d[8]) + (d[2] + d[6])) + ((d[1] + d[7]) + (d[3] + d[5])) + d[4];
    const float jx = ((d[2] - d[0]) + (d[8] - d[6])) + (d[5] - d[3]);
    const float jy = ((d[6] - d[0]) + (d[8] - d[2])) + (d[7] - d[1]);
    const float rho = 1.0f + drho;
    const float irho = rcp_fast(rho);
    const float ux = jx * irho, uy = jy * irho;
    const float usq15 = 1.5f * (ux * ux + uy * uy);
    const L nusq(-usq15), lrho(rho), ldrho(drho), c3(3.0f), c45(4.5f);
    // xi of pair k's first member (v_k . u); the second has -xi
    auto xi_of = [&](int k) {
        const int a = va(k), b = vb(k);
        const float x = (a == 0) ? 0.0f : (a > 0 ? ux : -ux);
        return (b == 0) ? x : (b > 0 ? x + uy : x - uy);
    };
    L D[4], LM[4], P[4], DF[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        D[k] = L(d[k], d[8 - k]);
        LM[k] = L(lam[k], lam[8 - k]);
        const float x = xi_of(k);
        const L X(x, -x);
        P[k] = fmaL(X, fmaL(c45, X, c3), nusq);
        DF[k] = fmaL(L(-(float)wgt(k)), fmaL(lrho, P[k], ldrho), D[k]);
    }
    const float P4 = -usq15;
    const float df4 = d[4] - (float)wgt(4) * (drho + rho * P4);
    L DFB[4], PB[4];
    const L n2b(-p.two_beta);
    L BB(0.0f);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        DFB[k] = n2b * LM[k];
        PB[k] = L(0.0f);
        BB = fmaL(LM[k], DF[k], BB);
    }
    float dfb4 = -p.two_beta * lam[4], pb4 = 0.0f;
    float bb = -2.0f * ((BB.lo() + BB.hi()) + lam[4] * df4);
    float uxb = 0.0f, uyb = 0.0f;
    if constexpr (VAR != kLBGK) {
        const L s02 = DF[0] + DF[2];  // (df0 + df2, df8 + df6)
        const float corner = s02.lo() + s02.hi();
        const float m20 = corner + (DF[3].lo() + DF[3].hi());
        const float m02 = corner + (DF[1].lo() + DF[1].hi());
        const float m11 = (DF[0].lo() + DF[0].hi()) - (DF[2].lo() + DF[2].hi());
        float c20, c02;
        if constexpr (VAR == kA || VAR == kC) {
            c20 = m20;
            c02 = m02;
        } else {
            c20 = 0.5f * (m20 - m02);
            c02 = -c20;
        }
        // 1-D dual vectors at c (u for the central basis, 0 for the natural):
        // e0 = (c(c-1)/2, 1 - c^2, c(c+1)/2), e1 = (c - 1/2, -2c, c + 1/2),
        // e2 = (1/2, -1, 1/2); the outer entries as pairs (in both orders)
        const float cx = central ? ux : 0.0f, cy = central ? uy : 0.0f;
        const L lcx(cx), lcy(cy), h(0.5f);
        const L e0x02 = (h * lcx) * (lcx + L(-1.0f, 1.0f)), e0x20 = (h * lcx) * (lcx + L(1.0f, -1.0f));
        const L e0y02 = (h * lcy) * (lcy + L(-1.0f, 1.0f));
        const L e1x02 = lcx + L(-0.5f, 0.5f), e1x20 = lcx + L(0.5f, -0.5f);
        const L e1y02 = lcy + L(-0.5f, 0.5f), e1y20 = lcy + L(0.5f, -0.5f);
        const float e0x1 = 1.0f - cx * cx, e0y1 = 1.0f - cy * cy, e1x1 = -2.0f * cx, e1y1 = -2.0f * cy;
        // ds(a,b) = m11 e1x[a] e1y[b] + (e2[a] c20 e0y[b] + e2[b] c02 e0x[a])
        const L lm11(m11), lc20(c20), lc02(c02);
        const L Cx02 = lm11 * e1x02, Cx20 = lm11 * e1x20, Bx02 = lc02 * e0x02, Bx20 = lc02 * e0x20;
        const L Ay02 = lc20 * e0y02;
        const float cx1 = m11 * e1x1, bx1 = c02 * e0x1, ay1 = c20 * e0y1;
        L DS[4];
        DS[0] = fmaL(Cx02, e1y02, fmaL(h, Ay02, h * Bx02));
        DS[1] = fmaL(L(cx1), e1y02, fmaL(L(-1.0f), Ay02, L(0.5f * bx1)));
        DS[2] = fmaL(Cx20, e1y02, fmaL(h, Ay02, h * Bx20));
        DS[3] = fmaL(Cx02, L(e1y1), fmaL(h, L(ay1), -Bx02));
        const float ds4 = cx1 * e1y1 - (ay1 + bx1);
        // entropic weights q_i = 1 / (W_i (1 + P_i)) by Montgomery's
        // simultaneous inversion over the pairs (one reciprocal)
        L X1[4], PRE[4], WI[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) X1[k] = L(1.0f) + P[k];
        const float x4 = 1.0f + P4;
        PRE[0] = X1[0];
#pragma unroll
        for (int k = 1; k < 4; ++k) PRE[k] = PRE[k - 1] * X1[k];
        const float prod8 = PRE[3].lo() * PRE[3].hi();
        const float r = rcp_fast(prod8 * x4);
        const float wi4 = r * prod8;
        const float rx4 = r * x4;
        L R(rx4 * PRE[3].hi(), rx4 * PRE[3].lo());  // 1 / PRE[3], per member
#pragma unroll
        for (int k = 3; k >= 1; --k) {
            WI[k] = R * PRE[k - 1];
            R = R * X1[k];
        }
        WI[0] = R;
        L DH[4], Q[4];
        L SH(0.0f), HH(0.0f);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            DH[k] = DF[k] - DS[k];
            Q[k] = L((float)inv_wgt(k)) * WI[k];
            const L t = DH[k] * Q[k];
            SH = fmaL(DS[k], t, SH);
            HH = fmaL(DH[k], t, HH);
        }
        const float dh4 = df4 - ds4, q4 = (float)inv_wgt(4) * wi4;
        const float sh = (SH.lo() + SH.hi()) + ds4 * dh4 * q4;
        const float hh = (HH.lo() + HH.hi()) + dh4 * dh4 * q4;
        float ch, Rr = 0.0f;
        const bool has_h = hh > 0.0f;
        guarded = !p.fixed && p.guard > 0.0f && !(hh > p.guard);
        const float ihh = has_h ? rcp_fast(hh) : 0.0f;
        if (p.fixed) {
            ch = p.ch_fixed;
        } else if (has_h) {
            Rr = sh * ihh;
            ch = p.one_m_2beta * (1.0f + Rr);
        } else {
            ch = 0.0f;
        }
        // ---------------------------------------------------------- reverse
        const L nch(-ch);
        L DHB[4], DSB[4];
        L CHB(0.0f);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            DHB[k] = nch * LM[k];
            CHB = fmaL(LM[k], DH[k], CHB);
        }
        float dhb4 = -ch * lam[4];
        const float chb = -((CHB.lo() + CHB.hi()) + lam[4] * dh4);
        float Rb = 0.0f;
        if (p.fixed) {
            bb += chb * (p.gamma_fixed - 2.0f);
        } else if (has_h) {
            bb += chb * (-2.0f * (1.0f + Rr));
            Rb = chb * p.one_m_2beta;
        }
        const float shb = Rb * ihh;
        const float hhb = -Rb * Rr * ihh;
        const L lshb(shb), lhhb(hhb), lhhb2(2.0f * hhb);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const L t = DH[k] * Q[k];
            DSB[k] = lshb * t;
            DHB[k] = fmaL(lshb, DS[k] * Q[k], fmaL(lhhb2, t, DHB[k]));
            const L qb = DH[k] * fmaL(lshb, DS[k], lhhb * DH[k]);
            PB[k] = PB[k] - (qb * (Q[k] * Q[k])) * L((float)wgt(k));  // q_i / x_i = W_i q_i^2
            DFB[k] = DFB[k] + DHB[k];
            DSB[k] = DSB[k] - DHB[k];
        }
        float dsb4 = shb * dh4 * q4;
        dhb4 += shb * ds4 * q4 + 2.0f * hhb * dh4 * q4;
        pb4 -= (shb * ds4 * dh4 + hhb * dh4 * dh4) * (q4 * q4) * (float)wgt(4);
        dfb4 += dhb4;
        dsb4 -= dhb4;
        // reverse of ds through per-axis partial sums of D(a,b) = dsb[3b + a]
        // (rows b: S, V; columns a: Ta, U), outer entries as pairs
        const L DSB2s(DSB[2].hi(), DSB[2].lo());  // (dsb6, dsb2)
        const L S02 = fmaL(h, DSB[0] + DSB[2], -DSB[1]);
        const float S1 = 0.5f * (DSB[3].lo() + DSB[3].hi()) - dsb4;
        const L T02 = fmaL(h, DSB[0] + DSB2s, -DSB[3]);
        const float T1 = 0.5f * (DSB[1].lo() + DSB[1].hi()) - dsb4;
        const L U02 = fmaL(e1y02, DSB[0], fmaL(L(e1y1), DSB[3], e1y20 * DSB2s));
        const float U1 = e1y02.lo() * DSB[1].lo() + e1y1 * dsb4 + e1y02.hi() * DSB[1].hi();
        const L V02 = fmaL(e1x02, DSB[0], fmaL(L(e1x1), DSB[1], e1x20 * DSB[2]));
        const float V1 = e1x02.lo() * DSB[3].lo() + e1x1 * dsb4 + e1x02.hi() * DSB[3].hi();
        const L pc20 = e0y02 * S02, pc02 = e0x02 * T02, pm11 = e1x02 * U02;
        const float c20b = (pc20.lo() + pc20.hi()) + e0y1 * S1;
        const float c02b = (pc02.lo() + pc02.hi()) + e0x1 * T1;
        const float m11b = (pm11.lo() + pm11.hi()) + e1x1 * U1;
        if constexpr (central) {
            // d e0(c)/dc = e1(c), d e1(c)/dc = (1, -2, 1), with e0xb = c02 Ta,
            // e1xb = m11 U, e0yb = c20 S, e1yb = m11 V
            const L tx = e1x02 * T02, ty = e1y02 * S02;
            uxb += c02 * ((tx.lo() + tx.hi()) + e1x1 * T1) + m11 * ((U02.lo() + U02.hi()) - 2.0f * U1);
            uyb += c20 * ((ty.lo() + ty.hi()) + e1y1 * S1) + m11 * ((V02.lo() + V02.hi()) - 2.0f * V1);
        }
        float m20b, m02b;
        if constexpr (VAR == kA || VAR == kC) {
            m20b = c20b;
            m02b = c02b;
        } else {
            m20b = 0.5f * (c20b - c02b);
            m02b = -m20b;
        }
        // df_i += a^2 m20b + b^2 m02b + a b m11b: the same for both members
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int a = va(k), b = vb(k);
            float inc = 0.0f;
            if (a != 0) inc = m20b;
            if (b != 0) inc = (a != 0) ? inc + m02b : m02b;
            if (a != 0 && b != 0) inc = (a == b) ? inc + m11b : inc - m11b;
            DFB[k] = DFB[k] + L(inc);
        }
    }
    // ------------------------------------------------- equilibrium and moments
    L MU[4];
    L DRHOB(0.0f), USQB(0.0f), UXB(0.0f), UYB(0.0f);
    const L c9(9.0f);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int a = va(k), b = vb(k);
        const float x = xi_of(k);
        const L X(x, -x);
        const L PR = fmaL(X, fmaL(c45, X, c3), nusq);
        const L W((float)wgt(k));
        MU[k] = LM[k] + DFB[k];
        DRHOB = DRHOB - DFB[k] * fmaL(W, PR, W);
        PB[k] = PB[k] - DFB[k] * L((float)wgt(k) * rho);
        USQB = USQB - PB[k];
        const L XIB = PB[k] * fmaL(c9, X, c3);
        if (a != 0) UXB = fmaL(L((float)a, (float)-a), XIB, UXB);
        if (b != 0) UYB = fmaL(L((float)b, (float)-b), XIB, UYB);
    }
    mu[4] = lam[4] + dfb4;
    float drhob = (DRHOB.lo() + DRHOB.hi()) - dfb4 * (float)wgt(4) * (1.0f + P4);
    pb4 -= dfb4 * (float)wgt(4) * rho;
    const float usqb = (USQB.lo() + USQB.hi()) - pb4;
    uxb += (UXB.lo() + UXB.hi()) + 3.0f * ux * usqb;
    uyb += (UYB.lo() + UYB.hi()) + 3.0f * uy * usqb;
    const float jxb = uxb * irho, jyb = uyb * irho;
    const float irhob = uxb * jx + uyb * jy;
    drhob -= irhob * irho * irho;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int a = va(k), b = vb(k);
        const float c = (a == 0 ? 0.0f : (a > 0 ? jxb : -jxb)) + (b == 0 ? 0.0f : (b > 0 ? jyb : -jyb));
        MU[k] = MU[k] + L(drhob + c, drhob - c);
        mu[k] = MU[k].lo();
        mu[8 - k] = MU[k].hi();
    }
    mu[4] += drhob;
    beta_bar = bb;
    return guarded;
}

// Returns true when the entropic denominator rho <dh|dh> is at or below
// p.guard (entropic gamma only): there the derivative of gamma* with respect
// to f, which carries 1 / <dh|dh>, is not resolved in the lane's precision,
// and the caller re-evaluates the node in double (as the forward step does).
template <int VAR, typename T>
__device__ __forceinline__ bool collide_adjoint(const T (&d)[9], const T (&lam)[9],
                                                const CollideParams<T>& p, T (&mu)[9],
                                                T& beta_bar)
{
    if constexpr (std::is_same<T, float>::value)
        return collide_adjoint_pairs<VAR>(d, lam, p, mu, beta_bar);
    bool guarded = false;
    constexpr bool central = (VAR == kA || VAR == kB);
    const T two_beta = p.two_beta;
    // ---------------------------------------------------------------- forward
    // pairwise sums (this order keeps the single-precision reverse closest
    // to the double one on long turbulent runs, where the linearised map
    // amplifies rounding; measured against column sums)
    const T drho = ((d[0] + d[8]) + (d[2] + d[6])) + ((d[1] + d[7]) + (d[3] + d[5])) + d[4];
    const T jx = ((d[2] - d[0]) + (d[8] - d[6])) + (d[5] - d[3]);
    const T jy = ((d[6] - d[0]) + (d[8] - d[2])) + (d[7] - d[1]);
    const T rho = T(1) + drho;
    const T irho = rcp_fast(rho);
    const T ux = jx * irho, uy = jy * irho;
    const T usq15 = T(1.5) * (ux * ux + uy * uy);
    T xi[9], P[9], df[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        xi[i] = T(va(i)) * ux + T(vb(i)) * uy;
        P[i] = xi[i] * (T(3) + T(4.5) * xi[i]) - usq15;
        df[i] = d[i] - T(wgt(i)) * (drho + rho * P[i]);
    }
    T dfb[9], Pb[9];
    T uxb = T(0), uyb = T(0);
    T bb = T(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        dfb[i] = -two_beta * lam[i];
        Pb[i] = T(0);
        bb -= T(2) * lam[i] * df[i];
    }
    if constexpr (VAR != kLBGK) {
        const T corner = (df[0] + df[2]) + (df[6] + df[8]);
        const T m20 = corner + (df[3] + df[5]);
        const T m02 = corner + (df[1] + df[7]);
        const T m11 = (df[0] + df[8]) - (df[2] + df[6]);
        T c20, c02;
        if constexpr (VAR == kA || VAR == kC) {
            c20 = m20;
            c02 = m02;
        } else {
            c20 = T(0.5) * (m20 - m02);
            c02 = -c20;
        }
        const T cx = central ? ux : T(0), cy = central ? uy : T(0);
        const T e0x[3] = {T(0.5) * cx * (cx - T(1)), T(1) - cx * cx, T(0.5) * cx * (cx + T(1))};
        const T e0y[3] = {T(0.5) * cy * (cy - T(1)), T(1) - cy * cy, T(0.5) * cy * (cy + T(1))};
        const T e1x[3] = {cx - T(0.5), T(-2) * cx, cx + T(0.5)};
        const T e1y[3] = {cy - T(0.5), T(-2) * cy, cy + T(0.5)};
        const T e2[3] = {T(0.5), T(-1), T(0.5)};
        T ds[9], dh[9], x[9], xi_inv[9], q[9];
        T sh = T(0), hh = T(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) x[i] = T(1) + P[i];
        inv9(x, xi_inv);  // 1 / x_i
        // ds_(a,b) = c20 e2[a] e0y[b] + c02 e0x[a] e2[b] + m11 e1x[a] e1y[b]
        T Ay[3], Bx[3], Cx[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Ay[k] = c20 * e0y[k];
            Bx[k] = c02 * e0x[k];
            Cx[k] = m11 * e1x[k];
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int a = i % 3, b = i / 3;
            ds[i] = Cx[a] * e1y[b] + (e2[a] * Ay[b] + e2[b] * Bx[a]);
            dh[i] = df[i] - ds[i];
            q[i] = T(inv_wgt(i)) * xi_inv[i];
            sh += ds[i] * dh[i] * q[i];
            hh += dh[i] * dh[i] * q[i];
        }
        T ch, R = T(0);
        const bool has_h = hh > T(0);
        guarded = !p.fixed && p.guard > T(0) && !(hh > p.guard);
        const T ihh = has_h ? rcp_fast(hh) : T(0);
        if (p.fixed) {
            ch = p.ch_fixed;
        } else if (has_h) {
            R = sh * ihh;
            ch = p.one_m_2beta * (T(1) + R);
        } else {
            ch = T(0);
        }
        // ---------------------------------------------------------- reverse
        T dhb[9], dsb[9];
        T chb = T(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            dhb[i] = -ch * lam[i];
            chb -= lam[i] * dh[i];
        }
        T Rb = T(0);
        if (p.fixed) {
            bb += chb * (p.gamma_fixed - T(2));
        } else if (has_h) {
            bb += chb * (T(-2) * (T(1) + R));
            Rb = chb * p.one_m_2beta;
        }
        const T shb = Rb * ihh;
        const T hhb = -Rb * R * ihh;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            dsb[i] = shb * dh[i] * q[i];
            dhb[i] += shb * ds[i] * q[i] + T(2) * hhb * dh[i] * q[i];
            const T qb = shb * ds[i] * dh[i] + hhb * dh[i] * dh[i];
            Pb[i] -= qb * (q[i] * q[i]) * T(wgt(i));  // q_i / x_i = W_i q_i^2
            dfb[i] += dhb[i];
            dsb[i] -= dhb[i];
        }
        // reverse of ds through per-axis partial sums of D(a,b) = dsb[3b + a]:
        // S_b = sum_a e2[a] D, T_a = sum_b e2[b] D, U_a = sum_b e1y[b] D,
        // V_b = sum_a e1x[a] D
        T S[3], Ta[3], U[3], V[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            S[k] = T(0.5) * (dsb[3 * k] + dsb[3 * k + 2]) - dsb[3 * k + 1];
            Ta[k] = T(0.5) * (dsb[k] + dsb[6 + k]) - dsb[3 + k];
            U[k] = e1y[0] * dsb[k] + e1y[1] * dsb[3 + k] + e1y[2] * dsb[6 + k];
            V[k] = e1x[0] * dsb[3 * k] + e1x[1] * dsb[3 * k + 1] + e1x[2] * dsb[3 * k + 2];
        }
        const T c20b = e0y[0] * S[0] + e0y[1] * S[1] + e0y[2] * S[2];
        const T c02b = e0x[0] * Ta[0] + e0x[1] * Ta[1] + e0x[2] * Ta[2];
        const T m11b = e1x[0] * U[0] + e1x[1] * U[1] + e1x[2] * U[2];
        T e0xb[3], e0yb[3], e1xb[3], e1yb[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            e0yb[k] = c20 * S[k];
            e0xb[k] = c02 * Ta[k];
            e1xb[k] = m11 * U[k];
            e1yb[k] = m11 * V[k];
        }
        if constexpr (central) {
            // d e0(c)/dc = e1(c), d e1(c)/dc = (1, -2, 1)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                uxb += e0xb[k] * e1x[k] + e1xb[k] * (k == 1 ? T(-2) : T(1));
                uyb += e0yb[k] * e1y[k] + e1yb[k] * (k == 1 ? T(-2) : T(1));
            }
        }
        T m20b, m02b;
        if constexpr (VAR == kA || VAR == kC) {
            m20b = c20b;
            m02b = c02b;
        } else {
            m20b = T(0.5) * (c20b - c02b);
            m02b = -m20b;
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const T a = T(va(i)), b = T(vb(i));
            dfb[i] += a * a * m20b + b * b * m02b + a * b * m11b;
        }
    }
    // ------------------------------------------------- equilibrium and moments
    T drhob = T(0), usqb = T(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        // xi and P again from u (cheaper than keeping nine of each live)
        const T xr = T(va(i)) * ux + T(vb(i)) * uy;
        const T Pr = xr * (T(3) + T(4.5) * xr) - usq15;
        mu[i] = lam[i] + dfb[i];
        drhob -= dfb[i] * T(wgt(i)) * (T(1) + Pr);
        Pb[i] -= dfb[i] * T(wgt(i)) * rho;
        usqb -= Pb[i];
        const T xib = Pb[i] * (T(3) + T(9) * xr);
        uxb += T(va(i)) * xib;
        uyb += T(vb(i)) * xib;
    }
    uxb += T(3) * ux * usqb;
    uyb += T(3) * uy * usqb;
    const T jxb = uxb * irho, jyb = uyb * irho;
    const T irhob = uxb * jx + uyb * jy;
    drhob -= irhob * irho * irho;
#pragma unroll
    for (int i = 0; i < 9; ++i) mu[i] += drhob + T(va(i)) * jxb + T(vb(i)) * jyb;
    beta_bar = bb;
    return guarded;
}

// block-wide FP64 sum of v, added by thread 0 to *acc (fixed order)
__device__ __forceinline__ void block_add(double v, double* acc)
{
    __shared__ double sm[256];
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *acc += sm[0];
}

// Reverse step of node (x, y) entirely in double: pulls the forward state,
// writes lambda^n to the nine sources and returns the node's beta adjoint.
template <int VAR, class C>
__device__ __forceinline__ double adj_node_f64(const typename C::S* __restrict__ g,
                                               const typename C::T* __restrict__ lam_in,
                                               typename C::T* __restrict__ lam_out, long long n,
                                               int x, int y, const StepArgs& a)
{
    double dd[9], ll[9], mm[9], bnode;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ai = i % 3 - 1, bi = i / 3 - 1;
        int sx = x - ai, sy = y - bi;
        sx = sx < 0 ? sx + a.nx : (sx >= a.nx ? sx - a.nx : sx);
        sy = sy < 0 ? sy + a.ny : (sy >= a.ny ? sy - a.ny : sy);
        dd[i] = C::to_f64(g[(long long)i * a.plane + (long long)sy * a.nx + sx], i, a.cs);
        ll[i] = (double)lam_in[(long long)i * a.plane + n];
    }
    CollideParams<double> q = a.pd;
    q.guard = 0.0;
    collide_adjoint<VAR>(dd, ll, q, mm, bnode);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ai = i % 3 - 1, bi = i / 3 - 1;
        int sx = x - ai, sy = y - bi;
        sx = sx < 0 ? sx + a.nx : (sx >= a.nx ? sx - a.nx : sx);
        sy = sy < 0 ? sy + a.ny : (sy >= a.ny ? sy - a.ny : sy);
        lam_out[(long long)i * a.plane + (long long)sy * a.nx + sx] = (typename C::T)mm[i];
    }
    return bnode;
}

// Reverse step of one node: g, lam_in and lam_out point at the node's row
// position minus t (t is added to every access), dn / up are the offsets of
// the rows y - 1 / y + 1 and cl / cr those of the columns x - 1 / x + 1.
// Writes lambda^n to the nine pull sources and returns the beta adjoint
// (0 for a node left to the double redo, which it marks in fixmask).
template <int VAR, class C>
__device__ __forceinline__ double adj_node(const typename C::S* __restrict__ g,
                                           const typename C::T* __restrict__ lam_in,
                                           typename C::T* __restrict__ lam_out, int t, long long dn,
                                           long long up, int cl, int cr, long long n,
                                           unsigned* __restrict__ fixmask,
                                           const CollideParams<typename C::T>& p, const StepArgs& a)
{
    using T = typename C::T;
    T d[9], lam[9], mu[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ai = i % 3 - 1, bi = i / 3 - 1;
        const long long off = (long long)i * a.plane + (bi == 1 ? dn : (bi == -1 ? up : 0)) +
                              (ai == 1 ? cl : (ai == -1 ? cr : 0));
        d[i] = C::decode(g[off + t], i, a.cs);
        lam[i] = lam_in[(long long)i * a.plane + t];
    }
    T bbar;
    const bool guarded = collide_adjoint<VAR>(d, lam, p, mu, bbar);
    if constexpr (!std::is_same<T, double>::value && VAR != kLBGK) {
        if (guarded) {
            atomicOr(fixmask + (n >> 5), 1u << (n & 31));
            bbar = T(0);  // summed by adj_fixup
        }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ai = i % 3 - 1, bi = i / 3 - 1;
        const long long off = (long long)i * a.plane + (bi == 1 ? dn : (bi == -1 ? up : 0)) +
                              (ai == 1 ? cl : (ai == -1 ? cr : 0));
        lam_out[off + t] = mu[i];
    }
    return (double)bbar;
}

// lambda^n from lambda^{n+1} and the forward state g^n; beta adjoint summed
// into part[blockIdx.x] (same grid every step, so the sum order is fixed).
// One node per thread; the grid strides over row segments of kAdjBlock
// nodes.  A segment away from the row ends addresses every population as
// the segment's base plus an offset that is the same for the whole block
// (plane, source row, source column) plus the thread index; the segments at
// the row ends take the periodic wrap of the columns per thread.
// Single precision: a node whose entropic denominator is at or below the
// guard (the nodes the forward step re-evaluates in double) is marked in
// fixmask (bit n % 32 of word n / 32) and left to adj_fixup, which redoes it
// in double.
template <int VAR, class C>
__global__ void __launch_bounds__(kAdjBlock, adj_min_blocks<VAR, typename C::T>())
adj_step(const typename C::S* __restrict__ g, const typename C::T* __restrict__ lam_in,
         typename C::T* __restrict__ lam_out, double* __restrict__ part, unsigned* __restrict__ fixmask,
         StepArgs a)
{
    using T = typename C::T;
    const CollideParams<T>& p = params_of<T>(a);
    const int nbx = (a.nx + kAdjBlock - 1) / kAdjBlock;
    const int segs = nbx * a.ny;  // nx * ny < 2^31
    double bsum = 0.0;
    for (int sg = blockIdx.x; sg < segs; sg += gridDim.x) {
        const int y = sg / nbx;
        const int x0 = (sg - y * nbx) * kAdjBlock;
        const int x = x0 + (int)threadIdx.x;
        // offsets of the source rows y - b (b = +1, -1; periodic), the same
        // for the whole segment
        const long long dn = (y == 0) ? (long long)(a.ny - 1) * a.nx : -(long long)a.nx;
        const long long up = (y == a.ny - 1) ? -(long long)(a.ny - 1) * a.nx : (long long)a.nx;
        if (x0 > 0 && x0 + kAdjBlock < a.nx) {
            // interior segment: the source column of population i is x - a_i
            // for every thread, so each address is the segment's base plus an
            // offset shared by the block plus the thread index
            const long long base = (long long)y * a.nx + x0;
            bsum += adj_node<VAR, C>(g + base, lam_in + base, lam_out + base, (int)threadIdx.x, dn, up,
                                     -1, 1, base + threadIdx.x, fixmask, p, a);
        } else if (x < a.nx) {
            // row ends: the columns x -+ 1 wrap
            const long long base = (long long)y * a.nx + x;
            const int cl = (x == 0) ? a.nx - 1 : -1;
            const int cr = (x == a.nx - 1) ? 1 - a.nx : 1;
            bsum += adj_node<VAR, C>(g + base, lam_in + base, lam_out + base, 0, dn, up, cl, cr, base,
                                     fixmask, p, a);
        }
    }
    block_add(bsum, part + blockIdx.x);
}

// Double-precision redo of the nodes adj_step marked: the mask is scanned in
// a fixed order by the same grid, so the beta sum stays deterministic; each
// word is cleared for the next step.
template <int VAR, class C>
__global__ void __launch_bounds__(256)
adj_fixup(const typename C::S* __restrict__ g, const typename C::T* __restrict__ lam_in,
          typename C::T* __restrict__ lam_out, double* __restrict__ part, unsigned* __restrict__ fixmask,
          StepArgs a)
{
    const long long total = (long long)a.nx * a.ny;
    const long long words = (total + 31) >> 5;
    double bsum = 0.0;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < words;
         w += (long long)gridDim.x * blockDim.x) {
        unsigned m = fixmask[w];
        if (m == 0u) continue;
        fixmask[w] = 0u;
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1u;
            const long long n = (w << 5) + b;
            const int y = (int)(n / a.nx), x = (int)(n - (long long)y * a.nx);
            bsum += adj_node_f64<VAR, C>(g, lam_in, lam_out, n, x, y, a);
        }
    }
    block_add(bsum, part + blockIdx.x);
}

// J of the final field and lambda^N = dJ/dg^N.  objective 0: kinetic energy
// sum_x rho |u|^2 / 2; objective 1: misfit sum_x |u - u_target|^2 / 2.
template <class C>
__global__ void __launch_bounds__(256)
adj_objective(const typename C::S* __restrict__ g, const double* __restrict__ tx,
              const double* __restrict__ ty, int objective, typename C::T* __restrict__ lam,
              double* __restrict__ part, StepArgs a)
{
    using T = typename C::T;
    const long long total = (long long)a.nx * a.ny;
    double jsum = 0.0;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < total;
         n += (long long)gridDim.x * blockDim.x) {
        double r, ux, uy;
        node_macro<C>(g, n, a, r, ux, uy);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double vx = va(i), vy = vb(i);
            double l;
            if (objective == 0) {
                l = vx * ux + vy * uy - 0.5 * (ux * ux + uy * uy);
            } else {
                l = ((ux - tx[n]) * (vx - ux) + (uy - ty[n]) * (vy - uy)) / r;
            }
            lam[(long long)i * a.plane + n] = (T)l;
        }
        if (objective == 0)
            jsum += 0.5 * r * (ux * ux + uy * uy);
        else
            jsum += 0.5 * ((ux - tx[n]) * (ux - tx[n]) + (uy - ty[n]) * (uy - ty[n]));
    }
    block_add(jsum, part + blockIdx.x);
}

// dJ/du0 = (d f^eq / du)^T lambda^0 for the equilibrium initialisation.
template <class C>
__global__ void __launch_bounds__(256)
adj_grad_u0(const double* __restrict__ rho0, const double* __restrict__ ux0,
            const double* __restrict__ uy0, const typename C::T* __restrict__ lam,
            double* __restrict__ gx, double* __restrict__ gy, StepArgs a)
{
    const long long total = (long long)a.nx * a.ny;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < total;
         n += (long long)gridDim.x * blockDim.x) {
        const double r = rho0[n], x = ux0[n], y = uy0[n];
        double sx = 0.0, sy = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double vx = va(i), vy = vb(i);
            const double xi = vx * x + vy * y;
            const double l = (double)lam[(long long)i * a.plane + n];
            // f^eq_i = W_i rho (1 + 3 xi + 4.5 xi^2 - 1.5 u^2)
            sx += l * wgt(i) * r * (3.0 * vx + 9.0 * xi * vx - 3.0 * x);
            sy += l * wgt(i) * r * (3.0 * vy + 9.0 * xi * vy - 3.0 * y);
        }
        gx[n] = sx;
        gy[n] = sy;
        if (!isfinite(sx) || !isfinite(sy)) atomicOr(a.flag, 8);  // adjoint overflowed
    }
}

__global__ void sum_partials(const double* __restrict__ part, int n, double* __restrict__ out);

}  // namespace kbc
