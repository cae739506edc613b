"""Second-order convergence of every model on the paper's Green-Taylor vortex
(k1 = 1, k2 = 4 on [0, 2 pi)^2, Grad initialisation), error against the
analytic decaying solution at t_c = ln 2 / (nu (k1^2 + k2^2)) for
Re = u0 N / nu = 100 with u0 = 0.03 and Re = 1000 with u0 = 0.04 on
N = 64, 128, 256 (the paper's convergence figure).

The initial density carries the vortex's pressure (p = cs^2 rho).  With the
constant density the paper states, the initial pressure mismatch launches
sound waves of relative amplitude ~ u0 / cs that the low viscosity of the
Re = 1000 case barely damps: the error then stalls near 3.5% for LBGK, A and
C alike (a collision-independent plateau), which is why the pressure-carrying
start is used here.

The shear-layer test checks the paper's convergence figure for the doubly
periodic shear layer: under-resolved LBGK blows up while the KBC models stay
stable, B (and A) are the most accurate KBC variants there, and all models
agree once resolved."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1507_02509_gb300 import KBCError, Lattice, beta_from_viscosity, capi, flows  # noqa: E402

pytestmark = pytest.mark.gpu


def _error(variant, n, re, u0):
    nu = u0 * n / re
    kk = (2 * math.pi / n) ** 2 * 17
    tc = int(round(math.log(2.0) / (nu * kk)))
    rho, ux, uy = flows.taylor_green_k1k2(n, u0, pressure_rho=True)
    lat = Lattice(n, n, variant=variant, beta=beta_from_viscosity(nu), dtype="f64")
    lat.init(rho, ux, uy, grad=True).step(tc)
    _, vx, vy = (t.cpu().numpy() for t in lat.moments())
    lat.close()
    _, ex, ey = flows.taylor_green_k1k2(n, u0, t=tc, nu=nu)
    return math.sqrt(np.sum((vx - ex) ** 2 + (vy - ey) ** 2) / np.sum(ex ** 2 + ey ** 2))


@pytest.mark.parametrize("re,u0,ns", [(100, 0.03, (64, 128, 256)), (1000, 0.04, (64, 128, 256))])
@pytest.mark.parametrize("variant", ["lbgk", "A", "B", "C", "D"])
def test_taylor_green_second_order(variant, re, u0, ns):
    errs = [_error(variant, n, re, u0) for n in ns]
    slope = -np.polyfit(np.log(ns), np.log(errs), 1)[0]
    print(f"Re {re}, {variant}: errors {['%.3e' % e for e in errs]}, slope {slope:.2f}")
    assert 1.6 <= slope <= 2.4, (errs, slope)


def _shear(variant, n, dtype, re=30000.0, u0=0.04):
    """Shear layer (kappa = 80, delta = 0.05), Re = u0 N / nu, Grad
    initialisation, advanced to t_c = N / u0 (the same physical time on every
    grid); (finite, u_x, u_y)."""
    rho, ux, uy = flows.shear_layer(n, u0=u0)
    lat = Lattice(n, n, variant=variant, beta=beta_from_viscosity(u0 * n / re), dtype=dtype)
    lat.init(rho, ux, uy, grad=True)
    try:
        lat.step(int(round(n / u0)))
        lat.sync()
        _, vx, vy = (t.cpu().numpy() for t in lat.moments())
        ok = bool(np.isfinite(vx).all() and np.isfinite(vy).all())
    except KBCError as e:
        assert e.status == capi.KBC_ERR_NONFINITE
        ok, vx, vy = False, None, None
    lat.close()
    return ok, vx, vy


def test_shear_layer_under_resolution_ranking():
    """Re = 30000: relative L2 velocity error at t_c against a 2048^2 LBGK
    reference (FP32) at the coincident nodes.  N = 128: LBGK turns
    non-finite, A-D stay finite, B beats C and D and A beats C; N = 512: all
    five models agree within 10% (measured: B 0.050, A 0.062, D 0.093,
    C 0.153 at 128; 2.7e-3 to 2.8e-3 at 512)."""
    ref_ok, rx, ry = _shear("lbgk", 2048, "f32")
    assert ref_ok
    errs = {}
    for n in (128, 512):
        s = 2048 // n
        ex, ey = rx[::s, ::s], ry[::s, ::s]
        for v in ("lbgk", "A", "B", "C", "D"):
            ok, vx, vy = _shear(v, n, "f64")
            errs[(n, v)] = (math.sqrt(np.sum((vx - ex) ** 2 + (vy - ey) ** 2)
                                      / np.sum(ex ** 2 + ey ** 2)) if ok else math.inf)
    print({f"{n}/{v}": round(e, 5) for (n, v), e in errs.items()})
    assert errs[(128, "lbgk")] == math.inf
    for v in "ABCD":
        assert math.isfinite(errs[(128, v)])
    assert errs[(128, "B")] < errs[(128, "C")] and errs[(128, "B")] < errs[(128, "D")]
    assert errs[(128, "A")] < errs[(128, "C")]
    e512 = [errs[(512, v)] for v in ("lbgk", "A", "B", "C", "D")]
    assert max(e512) < 5e-3 and max(e512) < 1.1 * min(e512)
