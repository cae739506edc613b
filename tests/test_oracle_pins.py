"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, invariants, a brute-force numeric inverse or maximisation, the exact
root of the entropic condition, or values printed in the paper.  A plausible
slip anywhere in the oracle (a dropped term, a wrong sign or index, a
transposed operand, a wrong weight) fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq, minimize_scalar

import oracle as O

VA = O.VA.astype(np.float64)
VB = O.VB.astype(np.float64)
CS2 = 1.0 / 3.0
KBC = (O.A, O.B, O.C, O.D)


def random_states(n, seed, amp=0.05, umax=0.1):
    """Positive populations near equilibrium with random rho, u and a random
    non-equilibrium part of relative size amp."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.8, 1.2, n)
    ux = rng.uniform(-umax, umax, n)
    uy = rng.uniform(-umax, umax, n)
    f = O.feq(rho, ux, uy) * (1.0 + amp * rng.standard_normal((n, 9)))
    assert (f > 0).all()
    return f


def mom(f, px, py, cx=0.0, cy=0.0):
    """sum_i (a - cx)^px (b - cy)^py f_i per node (plain numpy)."""
    cx = np.asarray(cx)[..., None] if np.ndim(cx) else cx
    cy = np.asarray(cy)[..., None] if np.ndim(cy) else cy
    return np.sum((VA - cx) ** px * (VB - cy) ** py * f, axis=-1)


# ---------------------------------------------------------------- lattice


def test_weights_and_equilibrium_moments():
    """Eq. Peq and Eq. Qeq hold exactly for the D2Q9 product weights with
    cs^2 = 1/3 (and for no other choice): this pins W_i and cs^2, which the
    paper leaves unprinted, together with the equilibrium of Eq. Eq."""
    rng = np.random.default_rng(1)
    n = 64
    rho = rng.uniform(0.5, 2.0, n)
    ux = rng.uniform(-0.3, 0.3, n)
    uy = rng.uniform(-0.3, 0.3, n)
    fe = O.feq(rho, ux, uy)
    u = np.stack([ux, uy], 1)
    v = np.stack([VA, VB], 1)  # [9][2]
    assert np.allclose(fe.sum(1), rho, rtol=0, atol=1e-15)
    assert np.allclose(fe @ v, rho[:, None] * u, rtol=0, atol=1e-15)
    for a in range(2):
        for b in range(2):
            Pi = np.sum(fe * v[:, a] * v[:, b], 1)
            assert np.allclose(Pi, rho * CS2 * (a == b) + rho * u[:, a] * u[:, b], atol=1e-15)
            for c in range(2):
                Q = np.sum(fe * v[:, a] * v[:, b] * v[:, c], 1)
                expect = rho * CS2 * (u[:, a] * (b == c) + u[:, b] * (a == c) + u[:, c] * (a == b))
                assert np.allclose(Q, expect, atol=1e-15)
    # the weights themselves: product form, normalised
    W = O.weights()
    assert W.sum() == pytest.approx(1.0, abs=1e-16)
    assert W[4] == pytest.approx(4 / 9) and W[0] == pytest.approx(1 / 36) and W[1] == pytest.approx(1 / 9)


# ---------------------------------------------------------------- moment maps


@pytest.mark.parametrize("central", [False, True])
def test_populations_from_moments_reconstructs(central):
    """Eq. momentsD2Q9 (and its central form through Eq. cm) inverts the
    moment definitions: f -> (rho, u, T, N, Pi, Q, A) -> f is the identity."""
    f = random_states(200, 2, amp=0.2, umax=0.2)
    rho, ux, uy, m6 = O.moments(f, central)
    back = O.populations_from_moments(central, rho, ux, uy, m6)
    assert np.allclose(back, f, rtol=0, atol=2e-15)


def test_moment_definitions_against_direct_sums():
    f = random_states(50, 3, amp=0.2, umax=0.2)
    rho, ux, uy, nat = O.moments(f, False)
    _, _, _, cen = O.moments(f, True)
    assert np.allclose(rho, f.sum(1), atol=1e-15)
    assert np.allclose(ux, mom(f, 1, 0) / rho, atol=1e-15)
    # natural: T = M20 + M02, N = M20 - M02, Pi = M11, Qxyy = M12, Qyxx = M21, A = M22
    exp_nat = np.stack([mom(f, 2, 0) + mom(f, 0, 2), mom(f, 2, 0) - mom(f, 0, 2), mom(f, 1, 1),
                        mom(f, 1, 2), mom(f, 2, 1), mom(f, 2, 2)], 1) / rho[:, None]
    assert np.allclose(nat, exp_nat, atol=1e-15)
    exp_cen = np.stack([mom(f, 2, 0, ux, uy) + mom(f, 0, 2, ux, uy),
                        mom(f, 2, 0, ux, uy) - mom(f, 0, 2, ux, uy),
                        mom(f, 1, 1, ux, uy), mom(f, 1, 2, ux, uy), mom(f, 2, 1, ux, uy),
                        mom(f, 2, 2, ux, uy)], 1) / rho[:, None]
    assert np.allclose(cen, exp_cen, atol=1e-15)


def test_natural_from_central_matches_direct():
    """Eq. cm maps the directly summed central moments onto the directly
    summed natural moments."""
    f = random_states(300, 4, amp=0.15, umax=0.25)
    rho, ux, uy, nat = O.moments(f, False)
    _, _, _, cen = O.moments(f, True)
    assert np.allclose(O.natural_from_central(ux, uy, cen), nat, rtol=0, atol=1e-15)


# ---------------------------------------------------------------- k-s-h split


def _moment_matrix(cx, cy):
    """Rows: the nine central monomials (a-cx)^p (b-cy)^q, p,q in {0,1,2}."""
    rows = []
    for p in range(3):
        for q in range(3):
            rows.append((VA - cx) ** p * (VB - cy) ** q)
    return np.array(rows)  # [9 monomials][9 populations]


def _row(p, q):
    return 3 * p + q


@pytest.mark.parametrize("variant", KBC)
def test_split_against_numeric_inverse(variant):
    """Delta s from the paper's representation equals the population that
    carries exactly the variant's shear-moment deviations (and no other
    moment), obtained by numerically inverting the 9x9 moment matrix."""
    f = random_states(40, 5 + variant, amp=0.1, umax=0.15)
    sp = O.split(variant, f)
    central = variant in (O.A, O.B)
    for n in range(f.shape[0]):
        rho = f[n].sum()
        ux, uy = mom(f[n], 1, 0) / rho, mom(f[n], 0, 1) / rho
        cx, cy = (ux, uy) if central else (0.0, 0.0)
        M = _moment_matrix(cx, cy)
        Minv = np.linalg.inv(M)
        dm = M @ (f[n] - sp["feq"][n])
        target = np.zeros(9)  # moment deviations that s must carry
        if variant in (O.A, O.C):  # T, N, Pi -> all of m20, m02, m11
            for pq in ((2, 0), (0, 2), (1, 1)):
                target[_row(*pq)] = dm[_row(*pq)]
        else:  # N, Pi only: m20 - m02 split evenly, trace left to h
            half = 0.5 * (dm[_row(2, 0)] - dm[_row(0, 2)])
            target[_row(2, 0)] = half
            target[_row(0, 2)] = -half
            target[_row(1, 1)] = dm[_row(1, 1)]
        ds = Minv @ target
        assert np.allclose(sp["ds"][n], ds, rtol=0, atol=1e-13), n
        assert np.allclose(sp["dh"][n], (f[n] - sp["feq"][n]) - ds, rtol=0, atol=1e-13)


@pytest.mark.parametrize("variant", KBC)
def test_split_conservation_and_table2(variant):
    """k carries rho and rho u; s and h carry none (Eq. k_conservation,
    Eq. sh_conservation); second moments of s and h follow Table 2."""
    f = random_states(100, 11 + variant, amp=0.1, umax=0.15)
    sp = O.split(variant, f)
    rho, ux, uy, cen = O.moments(f, True)
    _, _, _, nat = O.moments(f, False)
    k, s, h = sp["k"], sp["s"], sp["h"]
    assert np.allclose(k + s + h, f, atol=1e-15)
    assert np.allclose(k.sum(1), rho, atol=1e-15)
    assert np.allclose(mom(k, 1, 0), rho * ux, atol=1e-15)
    assert np.allclose(mom(k, 0, 1), rho * uy, atol=1e-15)
    for part in (s, h, sp["ds"], sp["dh"]):
        assert np.allclose(part.sum(1), 0, atol=1e-15)
        assert np.allclose(mom(part, 1, 0), 0, atol=1e-15)
        assert np.allclose(mom(part, 0, 1), 0, atol=1e-15)
    m = cen if variant in (O.A, O.B) else nat
    T, N, P = m[:, 0], m[:, 1], m[:, 2]
    if variant in (O.A, O.C):
        exp_s = (0.5 * rho * (T + N), 0.5 * rho * (T - N), rho * P)
        exp_h = (0 * rho, 0 * rho, 0 * rho)
    else:
        exp_s = (0.5 * rho * N, -0.5 * rho * N, rho * P)
        exp_h = (0.5 * rho * T, 0.5 * rho * T, 0 * rho)
    got_s = (mom(s, 2, 0), mom(s, 0, 2), mom(s, 1, 1))
    got_h = (mom(h, 2, 0), mom(h, 0, 2), mom(h, 1, 1))
    for g, e in zip(got_s + got_h, exp_s + exp_h):
        assert np.allclose(g, e, rtol=0, atol=1e-14)
    # the kinematic part has no higher moments in its own basis (Sec. 5)
    central = variant in (O.A, O.B)
    _, _, _, mk = O.moments(k, central)
    assert np.allclose(mk, 0, atol=1e-14)


def test_lbgk_row_of_table1_puts_everything_in_s():
    f = random_states(30, 21)
    sp = O.split(O.LBGK, f)
    assert np.allclose(sp["dh"], 0, atol=1e-15)
    assert np.allclose(sp["ds"], f - sp["feq"], atol=1e-15)


# ---------------------------------------------------------------- stabiliser


def _entropic(x, y, feq):
    return np.sum(x * y / feq)


@pytest.mark.parametrize("variant", KBC)
@pytest.mark.parametrize("beta", [0.55, 0.9, 0.999])
def test_gamma_maximises_quadratic_entropy(variant, beta):
    """Eq. result21 is the maximiser over gamma of the quadratic entropy
    -<df'|df'>/2 of the post-collision deviation
    df' = (1 - 2 beta) ds + (1 - beta gamma) dh (brute-force 1-D search)."""
    f = random_states(20, 31 + variant, amp=0.05)
    sp = O.split(variant, f)
    _, gam = O.collide(variant, beta, f)
    for n in range(f.shape[0]):
        ds, dh, fe = sp["ds"][n], sp["dh"][n], sp["feq"][n]

        def neg_entropy(g):
            d = (1 - 2 * beta) * ds + (1 - beta * g) * dh
            return 0.5 * _entropic(d, d, fe)

        res = minimize_scalar(neg_entropy, bracket=(-50.0, 0.0, 50.0), tol=1e-14)
        assert gam[n] == pytest.approx(res.x, rel=1e-6, abs=1e-6)
        # and the neighbours of the oracle's gamma are never better
        for dg in (1e-4, -1e-4):
            assert neg_entropy(gam[n]) <= neg_entropy(gam[n] + dg)


@pytest.mark.parametrize("variant", KBC)
def test_gamma_star_approximates_exact_entropic_root(variant):
    """gamma* of Eq. result21 is the first-order expansion of the exact
    condition Eq. result1: the gap to the exact root shrinks linearly with the
    size eps of the non-equilibrium part."""
    beta = 0.95
    gaps = []
    for eps in (1e-2, 1e-3, 1e-4):
        f = random_states(10, 41 + variant, amp=eps)
        sp = O.split(variant, f)
        _, gam = O.collide(variant, beta, f)
        g = []
        for n in range(f.shape[0]):
            ds, dh, fe = sp["ds"][n], sp["dh"][n], sp["feq"][n]

            def cond(x):
                return np.sum(dh * np.log(1 + ((1 - beta * x) * dh - (2 * beta - 1) * ds) / fe))

            gs = gam[n]
            exact = brentq(cond, gs - 5.0, gs + 5.0, xtol=1e-15)
            g.append(abs(exact - gs))
        gaps.append(max(g))
    assert gaps[1] < 0.2 * gaps[0] and gaps[2] < 0.2 * gaps[1], gaps
    assert gaps[2] < 1e-2


def _states_at_rest(n, seed, amp):
    """Populations with zero momentum: W_i rho (1 + noise) with the momentum
    removed by symmetrising the noise between opposite velocities."""
    rng = np.random.default_rng(seed)
    W = O.weights()
    rho = rng.uniform(0.9, 1.1, n)
    e = amp * rng.standard_normal((n, 9))
    opp = np.array([8 - i for i in range(9)])
    e = 0.5 * (e + e[:, opp])
    f = W * rho[:, None] * (1 + e)
    assert np.allclose(mom(f, 1, 0), 0, atol=1e-16) and np.allclose(mom(f, 0, 1), 0, atol=1e-16)
    return f


@pytest.mark.parametrize("variant", KBC)
def test_zeroth_order_scalar_product(variant):
    """At u = 0: <ds|dh> = -rho (9A - 1)(3T - 2)/4 for A and C, 0 for B and D
    (the zeroth-order asymptotics of Sec. 4), hence gamma = 1/beta for B, D."""
    f = _states_at_rest(50, 51 + variant, 0.1)
    sp = O.split(variant, f)
    rho, _, _, m = O.moments(f, True)
    T, A = m[:, 0], m[:, 5]
    sh = np.sum(sp["ds"] * sp["dh"] / sp["feq"], 1)
    if variant in (O.A, O.C):
        assert np.allclose(sh, -0.25 * rho * (9 * A - 1) * (3 * T - 2), rtol=1e-12, atol=1e-17)
        assert np.max(np.abs(sh)) > 1e-6
    else:
        assert np.allclose(sh, 0, atol=1e-17)
        beta = 0.8
        _, gam = O.collide(variant, beta, f)
        assert np.allclose(gam, 1 / beta, rtol=1e-12)


# ---------------------------------------------------------------- relaxation


@pytest.mark.parametrize("variant", KBC)
def test_gamma_two_is_lbgk(variant):
    """With gamma forced to 2, KBC is LBGK (Sec. 3): bit for bit in the
    generalised-equilibrium form (Eq. EGE, Eq. GE), to rounding against the
    mirror form of Eq. LBGKmirr."""
    f = random_states(100, 61 + variant)
    beta = 0.93
    kbc_ge, _ = O.collide(variant, beta, f, gamma_mode=1, gamma_fixed=2.0, form=1)
    lbgk_ge, _ = O.collide(O.LBGK, beta, f, form=1)
    assert np.array_equal(kbc_ge, lbgk_ge)
    kbc_m, _ = O.collide(variant, beta, f, gamma_mode=1, gamma_fixed=2.0, form=0)
    lbgk_m, _ = O.collide(O.LBGK, beta, f, form=0)
    assert np.max(np.abs(kbc_m - lbgk_m) / np.abs(lbgk_m)) < 8 * np.finfo(float).eps
    # and LBGK is f + 2 beta (f^eq - f)
    plain = f + 2 * beta * (O.feq(*O.moments(f, False)[:3]) - f)
    assert np.allclose(lbgk_m, plain, rtol=1e-15, atol=1e-17)


@pytest.mark.parametrize("variant", KBC)
def test_mirror_and_generalised_equilibrium_forms_agree(variant):
    f = random_states(60, 71 + variant)
    for beta in (0.6, 0.97):
        a, ga = O.collide(variant, beta, f, form=0)
        b, gb = O.collide(variant, beta, f, form=1)
        assert np.array_equal(ga, gb)
        assert np.allclose(a, b, rtol=0, atol=1e-15)


@pytest.mark.parametrize("variant", KBC)
def test_post_collision_moment_relaxation(variant):
    """After one collision: ds' = (1 - 2 beta) ds, dh' = (1 - beta gamma) dh
    (Eq. ksh-mirror); for A and C the stress relaxes as
    Pi' - Pi^eq = (1 - 2 beta)(Pi - Pi^eq)."""
    f = random_states(60, 81 + variant)
    beta = 0.9
    out, gam = O.collide(variant, beta, f)
    sp0 = O.split(variant, f)
    sp1 = O.split(variant, out)
    assert np.allclose(sp1["feq"], sp0["feq"], atol=1e-15)
    assert np.allclose(sp1["ds"], (1 - 2 * beta) * sp0["ds"], rtol=0, atol=1e-15)
    assert np.allclose(sp1["dh"], (1 - beta * gam[:, None]) * sp0["dh"], rtol=0, atol=1e-15)
    if variant in (O.A, O.C):
        for px, py in ((2, 0), (0, 2), (1, 1)):
            d0 = mom(f - sp0["feq"], px, py)
            d1 = mom(out - sp0["feq"], px, py)
            assert np.allclose(d1, (1 - 2 * beta) * d0, atol=1e-15)


@pytest.mark.parametrize("variant", KBC)
def test_regularised_limit(variant):
    """gamma = 1/beta gives f' = f^eq + (1 - 2 beta) ds: all higher moments
    brought to equilibrium (regularised LB, Sec. 4)."""
    f = random_states(40, 91 + variant)
    beta = 0.85
    out, _ = O.collide(variant, beta, f, gamma_mode=1, gamma_fixed=1 / beta)
    sp = O.split(variant, f)
    assert np.allclose(out, sp["feq"] + (1 - 2 * beta) * sp["ds"], atol=1e-15)


def test_collision_conserves_and_equilibrium_is_fixed_point():
    f = random_states(100, 101)
    for v in (O.LBGK,) + KBC:
        out, _ = O.collide(v, 0.97, f)
        assert np.allclose(out.sum(1), f.sum(1), rtol=1e-15)
        assert np.allclose(mom(out, 1, 0), mom(f, 1, 0), atol=1e-16)
        assert np.allclose(mom(out, 0, 1), mom(f, 0, 1), atol=1e-16)
        fe = O.feq([1.0, 1.1], [0.05, -0.02], [0.01, 0.03])
        o2, g2 = O.collide(v, 0.97, fe)
        assert np.allclose(o2, fe, rtol=1e-15)


# ---------------------------------------------------------------- grid step


def test_uniform_flow_is_a_fixed_point():
    n = 8
    rho = np.full((n, n), 1.05)
    ux = np.full((n, n), 0.07)
    uy = np.full((n, n), -0.03)
    g0 = O.init_feq(rho, ux, uy)
    for v in (O.LBGK,) + KBC:
        g = O.step(g0, v, 0.99, nsteps=5)
        assert np.allclose(g, g0, rtol=2e-15, atol=0)


def test_streaming_is_the_periodic_pull():
    """At beta -> 0+ the collision of Eq. Egeneral is the identity, so one
    step is the pure periodic pull f_i(x) = f'_i(x - v_i)."""
    rng = np.random.default_rng(5)
    g = O.init_feq(np.ones((5, 7)), 0.01 * rng.standard_normal((5, 7)),
                   0.01 * rng.standard_normal((5, 7)))
    beta = 1e-12
    g1 = O.step(g, O.LBGK, beta, 1)
    for i in range(9):
        shifted = np.roll(np.roll(g[i], int(O.VA[i]), axis=1), int(O.VB[i]), axis=0)
        assert np.allclose(g1[i], shifted, rtol=0, atol=1e-12)


@pytest.mark.parametrize("variant", (O.LBGK,) + KBC)
def test_mass_and_momentum_conserved_over_steps(variant):
    rng = np.random.default_rng(7)
    n = 16
    rho = 1 + 0.01 * rng.standard_normal((n, n))
    ux, uy = 0.05 * rng.standard_normal((n, n)), 0.05 * rng.standard_normal((n, n))
    g = O.init_feq(rho, ux, uy)
    g2 = O.step(g, variant, 0.98, nsteps=20)
    m0 = g.sum()
    assert abs(g2.sum() - m0) <= 1e-14 * m0
    for vel in (VA, VB):
        p0 = np.tensordot(vel, g, 1).sum()
        p1 = np.tensordot(vel, g2, 1).sum()
        assert abs(p1 - p0) <= 1e-14 * m0


def _rot90_field(g):
    """Rotate the lattice by +90 degrees: node (x, y) -> (-y, x) and velocity
    (a, b) -> (-b, a)."""
    out = np.empty_like(g)
    for i in range(9):
        a, b = int(O.VA[i]), int(O.VB[i])
        j = 3 * (a + 1) + (-b + 1)  # index of (-b, a)
        # new[y', x'] with x' = -y, y' = x  (mod n)
        n = g.shape[1]
        src = g[i]
        new = np.empty_like(src)
        for y in range(n):
            for x in range(n):
                new[x % n, (-y) % n] = src[y, x]
        out[j] = new
    return out


@pytest.mark.parametrize("variant", (O.LBGK,) + KBC)
def test_rotation_equivariance(variant):
    rng = np.random.default_rng(9)
    n = 8
    g = O.init_feq(1 + 0.01 * rng.standard_normal((n, n)), 0.05 * rng.standard_normal((n, n)),
                   0.05 * rng.standard_normal((n, n)))
    g = O.step(g, variant, 0.9, 2)
    a = _rot90_field(O.step(g, variant, 0.9, 3))
    b = O.step(_rot90_field(g), variant, 0.9, 3)
    assert np.allclose(a, b, rtol=0, atol=1e-14)


def _mirror_x_field(g):
    """Reflect the lattice in x: node (x, y) -> (-x, y) and velocity
    (a, b) -> (-a, b)."""
    out = np.empty_like(g)
    for i in range(9):
        a, b = int(O.VA[i]), int(O.VB[i])
        j = 3 * (b + 1) + (-a + 1)  # index of (-a, b)
        out[j] = np.roll(g[i][:, ::-1], 1, axis=1)  # column x -> (-x) mod n
    return out


@pytest.mark.parametrize("variant", (O.LBGK,) + KBC)
def test_mirror_equivariance(variant):
    """The D2Q9 velocity set, the weights, the equilibrium and each variant's
    split are symmetric under x -> -x, so stepping commutes with the
    reflection (a handedness slip, which a 90 degree rotation can map onto
    itself, would not)."""
    rng = np.random.default_rng(19)
    n = 8
    g = O.init_feq(1 + 0.01 * rng.standard_normal((n, n)), 0.05 * rng.standard_normal((n, n)),
                   0.05 * rng.standard_normal((n, n)))
    g = O.step(g, variant, 0.9, 2)
    a = _mirror_x_field(O.step(g, variant, 0.9, 3))
    b = O.step(_mirror_x_field(g), variant, 0.9, 3)
    assert np.allclose(a, b, rtol=0, atol=1e-14)
    assert not np.allclose(g, _mirror_x_field(g), rtol=0, atol=1e-6)  # the field is not symmetric


def _tg_rate(variant, n, u0, nu, steps):
    from paper_1507_02509_gb300 import flows

    beta = 1.0 / (6 * nu + 1)  # Eq. viscosity solved for beta (cs^2 = 1/3)
    rho, ux, uy = flows.taylor_green(n, u0=u0, pressure_rho=True)
    x = np.arange(n)[None, :]
    y = np.arange(n)[:, None]
    k = 2 * math.pi / n
    shape_x = -np.cos(k * x) * np.sin(k * y)
    g = O.init_grad(beta, rho, ux, uy)
    amps, ts = [], []
    for t in range(0, steps + 1, steps // 4):
        if t:
            g = O.step(g, variant, beta, steps // 4, nthreads=4)
        _, vx, _ = O.macro(g)
        amps.append(np.sum(vx * shape_x) / np.sum(shape_x * shape_x))
        ts.append(t)
    rate = -np.polyfit(ts, np.log(amps), 1)[0]
    return rate / (2 * nu * k * k) - 1.0


def test_taylor_green_decay_rate():
    """The vortex amplitude decays as exp(-2 nu k^2 t) with
    nu = cs^2 (1/(2 beta) - 1/2) (Eq. viscosity): at 64^2 (u0 = 0.04,
    nu = 0.01) the fitted rate is within 2% for every model, and the
    discretisation gap shrinks at least 3x from 64^2 to 128^2."""
    for variant in (O.LBGK, O.A, O.B, O.C, O.D):
        err64 = _tg_rate(variant, 64, 0.04, 0.01, 1000)
        assert abs(err64) < 2e-2, (variant, err64)
    for variant in (O.LBGK, O.B):
        err64 = _tg_rate(variant, 64, 0.04, 0.01, 1000)
        err128 = _tg_rate(variant, 128, 0.04, 0.01, 4000)
        assert abs(err128) < abs(err64) / 3, (variant, err64, err128)


def test_second_order_convergence_taylor_green():
    """Error against the analytic vortex at a fixed fraction of the decay
    time falls as N^-2 under diffusive refinement (u0 ~ 1/N at fixed nu and
    Re), the second-order accuracy the paper reports for all models."""
    from paper_1507_02509_gb300 import flows

    nu = 0.02
    beta = 1.0 / (6 * nu + 1)
    errs = []
    Ns = (16, 32, 64)
    for n in Ns:
        u0 = 0.04 * 16 / n
        k = 2 * math.pi / n
        t_end = int(round(0.25 / (2 * nu * k * k)))
        rho, ux, uy = flows.taylor_green(n, u0=u0, pressure_rho=True)
        g = O.init_grad(beta, rho, ux, uy)
        g = O.step(g, O.B, beta, t_end, nthreads=4)
        _, vx, vy = O.macro(g)
        decay = math.exp(-2 * nu * k * k * t_end)
        ex, ey = ux * decay, uy * decay
        errs.append(math.sqrt(np.sum((vx - ex) ** 2 + (vy - ey) ** 2) / np.sum(ex ** 2 + ey ** 2)))
    slope = -np.polyfit(np.log(Ns), np.log(errs), 1)[0]
    assert 1.8 <= slope <= 2.3, (errs, slope)


# ---------------------------------------------------------------- init / diagnostics


def test_grad_initialisation_moments():
    """Eq. Grad carries rho, rho u and Pi = Pi^eq + Pi^(1) exactly, with
    Pi^(1) = -rho cs^2/(2 beta) (du + du^T) (Eq. P1AC) from central
    differences."""
    from paper_1507_02509_gb300 import flows

    n, beta = 16, 0.9
    rho, ux, uy = flows.turbulence(n, k0=3, urms=0.05, seed=3, kcut=6)
    rho = rho + 0.01 * np.cos(2 * math.pi * np.arange(n) / n)[None, :]
    g = O.init_grad(beta, rho, ux, uy)
    gn = np.moveaxis(g, 0, -1)
    assert np.allclose(gn.sum(-1), rho, atol=1e-15)
    assert np.allclose(mom(gn, 1, 0), rho * ux, atol=1e-16)
    dxx = 0.5 * (np.roll(ux, -1, 1) - np.roll(ux, 1, 1))
    dyy = 0.5 * (np.roll(uy, -1, 0) - np.roll(uy, 1, 0))
    dxy = 0.5 * (np.roll(uy, -1, 1) - np.roll(uy, 1, 1)) + 0.5 * (np.roll(ux, -1, 0) - np.roll(ux, 1, 0))
    c = rho * CS2 / (2 * beta)
    assert np.allclose(mom(gn, 2, 0), rho * CS2 + rho * ux * ux - c * 2 * dxx, atol=1e-16)
    assert np.allclose(mom(gn, 0, 2), rho * CS2 + rho * uy * uy - c * 2 * dyy, atol=1e-16)
    assert np.allclose(mom(gn, 1, 1), rho * ux * uy - c * dxy, atol=1e-16)


@pytest.mark.parametrize("n", [8, 12, 32])
def test_diagnostics_taylor_green_closed_forms(n):
    """For the discrete vortex at equilibrium, with C, S = cos, sin(kx) and
    c, s = cos, sin(ky): |u|^2/2 = (u0^2/2)(C^2 s^2 + S^2 c^2) and, with
    central differences, w = 2 u0 sin(k) C c.  Grid means of cos^2, cos^4 and
    cos^2 sin^2 are 1/2, 3/8 and 1/8 (n > 4), so E = u0^2/4 with spatial std
    u0^2/8, and Z = u0^2 sin(k)^2/2 with std (sqrt(5)/4) u0^2 sin(k)^2 (the
    RMS histories of the shear-layer and turbulence sections).  The momentum
    sums vanish; LBGK reports gamma = 2 everywhere."""
    from paper_1507_02509_gb300 import flows

    u0 = 0.03
    rho, ux, uy = flows.taylor_green(n, u0=u0)
    g = O.init_feq(rho, ux, uy)
    d = O.diagnostics(g, O.B, 0.9)
    k = 2 * math.pi / n
    assert d[0] == pytest.approx(n * n, rel=1e-15)
    assert abs(d[1]) < 1e-13 and abs(d[2]) < 1e-13
    assert d[3] == pytest.approx(u0 * u0 / 4, rel=1e-13)
    assert d[4] == pytest.approx(0.5 * u0 * u0 * math.sin(k) ** 2, rel=1e-12)
    assert d[8] == pytest.approx(u0 * u0 / 8, rel=1e-13)
    assert d[9] == pytest.approx(math.sqrt(5) / 4 * u0 * u0 * math.sin(k) ** 2, rel=1e-12)
    assert d[6] <= d[5] <= d[7]
    dl = O.diagnostics(g, O.LBGK, 0.9)
    assert dl[5] == dl[6] == dl[7] == 2.0


def test_diagnostics_std_of_two_valued_fields():
    """A field whose nodes take one of two values with equal frequency has
    spatial std |v1 - v2| / 2: uniform flows (U1, 0) and (U2, 0) on
    alternating pairs of rows for |u|^2/2; every row then has one neighbour
    row of each kind, so central differences give w = +-(U1 - U2)/2 and
    w^2/2 is uniform (std 0)."""
    nx, ny, U1, U2 = 6, 8, 0.05, -0.02
    ux = np.full((ny, nx), U1)
    ux[2::4, :] = U2
    ux[3::4, :] = U2
    rho, uy = np.ones((ny, nx)), np.zeros((ny, nx))
    d = O.diagnostics(O.init_feq(rho, ux, uy), O.LBGK, 0.9)
    assert d[3] == pytest.approx(0.25 * (U1 * U1 + U2 * U2), rel=1e-14)
    assert d[8] == pytest.approx(0.25 * abs(U1 * U1 - U2 * U2), rel=1e-13)
    assert d[4] == pytest.approx(0.5 * (0.5 * (U1 - U2)) ** 2, rel=1e-14)
    assert d[9] < 1e-15 * d[4]


# ---------------------------------------------------------------- adjoint oracle


@pytest.mark.parametrize("variant", (O.LBGK, O.B, O.C))
def test_collision_jacobian_matches_finite_differences(variant):
    """Complex-step Jacobian against a fourth-order central difference."""
    f = random_states(5, 111 + variant)
    beta = 0.9
    J, db = O.collide_jacobian(variant, beta, f)
    h = 2e-6

    def d4(fun):
        return (8 * (fun(h) - fun(-h)) - (fun(2 * h) - fun(-2 * h))) / (12 * h)

    for k in range(9):
        def fk(e, k=k):
            g = f.copy()
            g[:, k] += e
            return O.collide(variant, beta, g)[0]

        assert np.allclose(J[:, :, k], d4(fk), rtol=1e-8, atol=1e-8)
    assert np.allclose(db, d4(lambda e: O.collide(variant, beta + e, f)[0]), rtol=1e-8, atol=1e-8)


@pytest.mark.parametrize("objective", [0, 1])
def test_adjoint_matches_central_differences(objective):
    """Gradients of J with respect to u0 and beta from the oracle's reverse
    sweep agree with central finite differences of the forward oracle."""
    from paper_1507_02509_gb300 import flows

    n, steps, beta, variant = 6, 4, 0.9, O.B
    rho, ux, uy = flows.turbulence(n, k0=1.5, urms=0.05, seed=13, kcut=2)
    rng = np.random.default_rng(2)
    tx, ty = 0.02 * rng.standard_normal((n, n)), 0.02 * rng.standard_normal((n, n))

    def J_of(ux_, uy_, b):
        g = O.step(O.init_feq(rho, ux_, uy_), variant, b, steps)
        r, vx, vy = O.macro(g)
        if objective == 0:
            return 0.5 * np.sum(r * (vx ** 2 + vy ** 2))
        return 0.5 * np.sum((vx - tx) ** 2 + (vy - ty) ** 2)

    J, gx, gy, gb = O.adjoint(variant, beta, rho, ux, uy, steps, objective, tx, ty)
    assert J == pytest.approx(J_of(ux, uy, beta), rel=1e-14)
    h = 1e-6
    for (yy, xx) in ((0, 0), (2, 3), (5, 1)):
        p, m = ux.copy(), ux.copy()
        p[yy, xx] += h
        m[yy, xx] -= h
        fd = (J_of(p, uy, beta) - J_of(m, uy, beta)) / (2 * h)
        assert gx[yy, xx] == pytest.approx(fd, rel=1e-6, abs=1e-10)
        p, m = uy.copy(), uy.copy()
        p[yy, xx] += h
        m[yy, xx] -= h
        fd = (J_of(ux, p, beta) - J_of(ux, m, beta)) / (2 * h)
        assert gy[yy, xx] == pytest.approx(fd, rel=1e-6, abs=1e-10)
    fd = (J_of(ux, uy, beta + h) - J_of(ux, uy, beta - h)) / (2 * h)
    assert gb == pytest.approx(fd, rel=1e-6, abs=1e-10)


# ---------------------------------------------------------------- exact stabiliser


@pytest.mark.parametrize("variant", KBC)
def test_exact_gamma_is_the_root_of_the_entropic_condition(variant):
    """gamma mode 2 returns the root of Eq. result1 (found independently with
    brentq) and that root maximises the relative entropy
    -sum f' ln(f'/f^eq) of the post-collision state over gamma (the condition
    is beta times the derivative of that entropy)."""
    beta = 0.93
    f = random_states(25, 151 + variant, amp=0.03)
    sp = O.split(variant, f)
    _, gex = O.collide(variant, beta, f, gamma_mode=2)
    _, gst = O.collide(variant, beta, f)
    for n in range(f.shape[0]):
        ds, dh, fe = sp["ds"][n], sp["dh"][n], sp["feq"][n]

        def cond(x):
            return np.sum(dh * np.log1p(((1 - beta * x) * dh - (2 * beta - 1) * ds) / fe))

        root = brentq(cond, gst[n] - 3.0, gst[n] + 3.0, xtol=1e-15)
        assert gex[n] == pytest.approx(root, rel=1e-11, abs=1e-11)

        def neg_rel_entropy(g):
            fp = fe + (1 - 2 * beta) * ds + (1 - beta * g) * dh
            return np.sum(fp * np.log(fp / fe))

        res = minimize_scalar(neg_rel_entropy, bracket=(gst[n] - 1, gst[n], gst[n] + 1),
                              tol=1e-12)
        assert gex[n] == pytest.approx(res.x, rel=1e-5, abs=1e-5)


def test_exact_gamma_limits():
    """At equilibrium the exact mode leaves the state unchanged (whatever
    gamma the rounding-level dh yields); the exact mode is rejected by the
    derivative routines."""
    fe = O.feq([1.0], [0.02], [0.01])
    out, _ = O.collide(O.B, 0.9, fe, gamma_mode=2)
    assert np.allclose(out, fe, rtol=1e-15, atol=0)
    with pytest.raises(ValueError):
        O.collide_jacobian(O.B, 0.9, fe, gamma_mode=2)


def test_diagnostics_ext_closed_forms():
    """Palinstrophy of the discrete vortex with central differences is
    u0^2 sin(k)^4 with spatial std u0^2 sin(k)^4 / 2; the entropy density of
    Eq. S vanishes at rest with unit density and is -rho ln rho for a density
    at rest, so a two-valued density gives the mean and std of two values."""
    from paper_1507_02509_gb300 import flows

    n, u0 = 32, 0.03
    rho, ux, uy = flows.taylor_green(n, u0=u0)
    k = 2 * math.pi / n
    d = O.diagnostics_ext(O.init_feq(rho, ux, uy))
    assert d[0] == pytest.approx(u0 * u0 * math.sin(k) ** 4, rel=1e-11)
    # |grad w|^2/2 = 2 u0^2 sin(k)^4 (S^2 c^2 + C^2 s^2): std u0^2 sin(k)^4 / 2
    assert d[1] == pytest.approx(0.5 * u0 * u0 * math.sin(k) ** 4, rel=1e-11)
    rest = O.init_feq(np.ones((4, 6)), np.zeros((4, 6)), np.zeros((4, 6)))
    d = O.diagnostics_ext(rest)
    assert abs(d[2]) < 1e-16 and d[0] == 0.0 and d[1] == 0.0
    r0 = 1.3
    d = O.diagnostics_ext(O.init_feq(np.full((4, 6), r0), np.zeros((4, 6)), np.zeros((4, 6))))
    assert d[2] == pytest.approx(-r0 * math.log(r0), rel=1e-14)
    assert d[3] <= 1e-15 * abs(d[2])  # identical values: std at the rounding of the mean
    # two densities on alternate rows at rest: s = -rho ln rho takes two values
    r = np.full((4, 6), r0)
    r[1::2, :] = 0.7
    d = O.diagnostics_ext(O.init_feq(r, np.zeros((4, 6)), np.zeros((4, 6))))
    s1, s2 = -r0 * math.log(r0), -0.7 * math.log(0.7)
    assert d[2] == pytest.approx(0.5 * (s1 + s2), rel=1e-14)
    assert d[3] == pytest.approx(0.5 * abs(s1 - s2), rel=1e-13)


def test_spectra_oracle_parseval_and_single_mode():
    """sum_k E(k) equals mean |u|^2 / 2 (Parseval); the Taylor-Green vortex
    with m modes puts all its energy in the shell round(sqrt(2) m)."""
    from oracle import spectra
    from paper_1507_02509_gb300 import flows

    rho, ux, uy = flows.turbulence(32, k0=4, urms=0.05, seed=3, kcut=12)
    k, E, Z = spectra.energy_spectrum(ux, uy)
    assert E.sum() == pytest.approx(0.5 * np.mean(ux ** 2 + uy ** 2), rel=1e-12)
    _, ux, uy = flows.taylor_green(32, u0=0.02, modes=3)
    k, E, Z = spectra.energy_spectrum(ux, uy)
    assert E[4] == pytest.approx(0.02 ** 2 / 4, rel=1e-12)
    assert E.sum() - E[4] < 1e-20
    assert Z[4] == pytest.approx((2 * math.pi * 4 / 32) ** 2 * E[4])


def test_taylor_green_k1k2_is_divergence_free_curl():
    """The paper's vortex: spectral divergence vanishes and the vorticity is
    the Laplacian-scaled stream function, for k1 = 1, k2 = 4."""
    from paper_1507_02509_gb300 import flows

    n = 64
    _, ux, uy = flows.taylor_green_k1k2(n, u0=0.03, k1=1, k2=4)
    kx = 2 * np.pi * np.fft.fftfreq(n, d=1.0 / n) / n
    KX, KY = np.meshgrid(kx, kx)
    div = np.fft.ifft2(1j * KX * np.fft.fft2(ux) + 1j * KY * np.fft.fft2(uy)).real
    assert np.max(np.abs(div)) < 1e-15
    w = np.fft.ifft2(1j * KX * np.fft.fft2(uy) - 1j * KY * np.fft.fft2(ux)).real
    x = 2 * np.pi * np.arange(n)[None, :] / n
    y = 2 * np.pi * np.arange(n)[:, None] / n
    k2l = (2 * np.pi / n) ** 2 * 17
    psi = (0.03 / 4) * np.cos(x) * np.cos(4 * y) * (n / (2 * np.pi))
    assert np.allclose(w, k2l * psi, atol=1e-15)
