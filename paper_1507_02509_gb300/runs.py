"""Histories of the paper's decaying-turbulence and shear-layer runs on the
GPU: the FP64 device diagnostics (mass, energy, enstrophy, gamma statistics,
palinstrophy, entropy) sampled every ``every`` steps while the field is
advanced.  Stops early and records the step when the field stops being
finite (the paper's LBGK runs "crash" in under-resolved cases).
"""
from __future__ import annotations

import math
import time

from . import DIAG_EXT_NAMES, DIAG_NAMES, KBCError, Lattice, beta_from_viscosity, capi, flows


def history(lat: Lattice, steps: int, every: int, ext: bool = True) -> dict:
    """Advance ``lat`` by ``steps`` steps, sampling the diagnostics at step 0
    and every ``every`` steps.  Returns lists keyed by diagnostic name plus
    ``step``, ``seconds`` and ``blew_up`` (the first step found non-finite, or
    None)."""
    out = {"step": []}
    for k in DIAG_NAMES + (DIAG_EXT_NAMES if ext else ()):
        out[k] = []

    def sample(t):
        d = lat.diagnostics()
        if ext:
            d.update(lat.diagnostics_ext())
        out["step"].append(t)
        for k, v in d.items():
            out[k].append(v)

    blew = None
    t0 = time.perf_counter()
    sample(0)
    done = 0
    while done < steps:
        k = min(every, steps - done)
        try:
            lat.step(k)
            lat.sync()
        except KBCError as e:
            if e.status != capi.KBC_ERR_NONFINITE:
                raise
            blew = done + k
            break
        done += k
        sample(done)
        if not math.isfinite(out["E"][-1]):
            blew = done
            break
    out["seconds"] = time.perf_counter() - t0
    out["blew_up"] = blew
    return out


def turbulence_run(n: int = 4096, steps: int = 50000, every: int = 500, variant="B",
                   dtype="f32", k0: float = 16.0, urms: float = 0.03, reynolds: float = 1e5,
                   seed: int = 0, f16_scale: float = 1.0, backend: str = "torch",
                   spectrum: str = "k4") -> dict:
    """Decaying two-dimensional turbulence, equilibrium initialisation, nu from
    Re = N sqrt(2E)/nu.  spectrum "k4": E(k) ~ k^4 exp(-2 (k/k0)^2); "paper":
    E(k) ~ k^6 / (1 + (k/k0)^18), the narrow-band spectrum of the paper's
    turbulence section."""
    from . import viscosity_for_reynolds

    nu = viscosity_for_reynolds(n, 0.5 * urms * urms, reynolds)
    beta = beta_from_viscosity(nu)
    spec = flows.spectrum_k4_gauss if spectrum == "k4" else flows.spectrum_paper
    rho, ux, uy = flows.turbulence(n, k0=k0, urms=urms, seed=seed, backend=backend,
                                   spectrum=spec,
                                   kcut=None if spectrum == "k4" else min(n // 2 - 1, int(4 * k0)))
    lat = Lattice(n, n, variant=variant, beta=beta, dtype=dtype)
    if dtype == "f16":
        lat.set_f16_scale(f16_scale)
    lat.init(rho, ux, uy)
    del rho, ux, uy
    h = history(lat, steps, every)
    lat.close()
    h.update({"n": n, "variant": variant, "dtype": dtype, "nu": nu, "beta": beta})
    return h


def shear_layer_run(n: int = 1024, steps: int = 20000, every: int = 500, variant="B",
                    dtype="f64", reynolds: float = 30000.0, u0: float = 0.04) -> dict:
    nu = u0 * n / reynolds
    beta = beta_from_viscosity(nu)
    rho, ux, uy = flows.shear_layer(n, u0=u0)
    lat = Lattice(n, n, variant=variant, beta=beta, dtype=dtype)
    lat.init(rho, ux, uy)
    h = history(lat, steps, every)
    lat.close()
    h.update({"n": n, "variant": variant, "dtype": dtype, "nu": nu, "beta": beta})
    return h
