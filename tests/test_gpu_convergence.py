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
start is used here."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1507_02509_gb300 import Lattice, beta_from_viscosity, flows  # noqa: E402

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
