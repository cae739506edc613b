"""FP64 CPU oracle of the D2Q9 KBC / LBGK step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it (see ``kbc_oracle.c`` for what each function follows
in the paper).  Arrays are numpy float64; populations are ``[9][ny][nx]``
(x fastest, ``i = 3(b+1) + (a+1)`` for ``v_i = (a, b)``) for grids and
``[n][9]`` for per-node batches.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libkbc_oracle.so")
_SRC = [os.path.join(_HERE, "kbc_oracle.c"), os.path.join(_HERE, "kbc_oracle_core.inc")]
_lock = threading.Lock()
_lib = None

LBGK, A, B, C, D = 0, 1, 2, 3, 4
VARIANTS = {"lbgk": LBGK, "A": A, "B": B, "C": C, "D": D}

# velocity of population i
VA = np.array([i % 3 - 1 for i in range(9)], dtype=np.int64)
VB = np.array([i // 3 - 1 for i in range(9)], dtype=np.int64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP)."""
    newest = max(os.path.getmtime(s) for s in _SRC)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC[0], "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            d = ctypes.POINTER(ctypes.c_double)
            i = ctypes.c_int
            db = ctypes.c_double
            sig = {
                "kbco_version": (i, []),
                "kbco_weight": (db, [i]),
                "kbco_feq_batch": (None, [i, d, d, d, d]),
                "kbco_moments_batch": (None, [i, i, d, d, d, d, d]),
                "kbco_natural_from_central_batch": (None, [i, d, d, d, d]),
                "kbco_populations_from_moments_batch": (None, [i, i, d, d, d, d, d]),
                "kbco_split_batch": (i, [i, i, d, d, d, d, d, d, d]),
                "kbco_collide_batch": (i, [i, i, db, i, db, i, d, d, d]),
                "kbco_collide_jacobian_batch": (i, [i, i, db, i, db, d, d, d]),
                "kbco_init_feq": (None, [i, i, d, d, d, d]),
                "kbco_init_grad": (None, [i, i, db, d, d, d, d]),
                "kbco_step": (i, [i, i, i, db, i, db, i, d, d, d, i]),
                "kbco_macro": (None, [i, i, d, d, d, d]),
                "kbco_diagnostics": (i, [i, i, i, db, i, db, d, d]),
                "kbco_diagnostics_ext": (i, [i, i, d, d]),
                "kbco_adjoint": (i, [i, i, i, db, i, db, d, d, d, i, i, d, d, d, d, d, d]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def weights() -> np.ndarray:
    return np.array([lib().kbco_weight(i) for i in range(9)])


# ---- per-node batches -----------------------------------------------------

def feq(rho, ux, uy) -> np.ndarray:
    rho, ux, uy = (_f64(np.atleast_1d(v)) for v in (rho, ux, uy))
    n = rho.size
    out = np.empty((n, 9))
    lib().kbco_feq_batch(n, _p(rho), _p(ux), _p(uy), _p(out))
    return out


def moments(f, central: bool):
    """rho, ux, uy and (T, N, Pi_xy, Q_xyy, Q_yxx, A) per node."""
    f = _f64(np.atleast_2d(f))
    n = f.shape[0]
    rho, ux, uy = np.empty(n), np.empty(n), np.empty(n)
    m6 = np.empty((n, 6))
    lib().kbco_moments_batch(n, int(central), _p(f), _p(rho), _p(ux), _p(uy), _p(m6))
    return rho, ux, uy, m6


def natural_from_central(ux, uy, c6) -> np.ndarray:
    ux, uy, c6 = _f64(np.atleast_1d(ux)), _f64(np.atleast_1d(uy)), _f64(np.atleast_2d(c6))
    n = ux.size
    out = np.empty((n, 6))
    lib().kbco_natural_from_central_batch(n, _p(ux), _p(uy), _p(c6), _p(out))
    return out


def populations_from_moments(central: bool, rho, ux, uy, m6) -> np.ndarray:
    rho, ux, uy = (_f64(np.atleast_1d(v)) for v in (rho, ux, uy))
    m6 = _f64(np.atleast_2d(m6))
    n = rho.size
    out = np.empty((n, 9))
    lib().kbco_populations_from_moments_batch(n, int(central), _p(rho), _p(ux), _p(uy),
                                              _p(m6), _p(out))
    return out


def split(variant: int, f):
    """dict with feq, ds, dh, k, s, h per node."""
    f = _f64(np.atleast_2d(f))
    n = f.shape[0]
    r = {k: np.empty((n, 9)) for k in ("feq", "ds", "dh", "k", "s", "h")}
    rc = lib().kbco_split_batch(n, variant, _p(f), _p(r["feq"]), _p(r["ds"]), _p(r["dh"]),
                                _p(r["k"]), _p(r["s"]), _p(r["h"]))
    if rc != 0:
        raise ValueError("bad variant")
    return r


def collide(variant: int, beta: float, f, gamma_mode: int = 0, gamma_fixed: float = 2.0,
            form: int = 0):
    """post-collision populations and gamma per node."""
    f = _f64(np.atleast_2d(f))
    n = f.shape[0]
    out = np.empty((n, 9))
    gm = np.empty(n)
    rc = lib().kbco_collide_batch(n, variant, float(beta), int(gamma_mode), float(gamma_fixed),
                                  int(form), _p(f), _p(out), _p(gm))
    if rc != 0:
        raise ValueError("bad arguments")
    return out, gm


def collide_jacobian(variant: int, beta: float, f, gamma_mode: int = 0,
                     gamma_fixed: float = 2.0):
    f = _f64(np.atleast_2d(f))
    n = f.shape[0]
    J = np.empty((n, 9, 9))
    db = np.empty((n, 9))
    rc = lib().kbco_collide_jacobian_batch(n, variant, float(beta), int(gamma_mode),
                                           float(gamma_fixed), _p(f), _p(J), _p(db))
    if rc != 0:
        raise ValueError("bad arguments")
    return J, db


# ---- grids ------------------------------------------------------------------

def init_feq(rho, ux, uy) -> np.ndarray:
    rho, ux, uy = (_f64(v) for v in (rho, ux, uy))
    ny, nx = rho.shape
    g = np.empty((9, ny, nx))
    lib().kbco_init_feq(nx, ny, _p(rho), _p(ux), _p(uy), _p(g))
    return g


def init_grad(beta: float, rho, ux, uy) -> np.ndarray:
    rho, ux, uy = (_f64(v) for v in (rho, ux, uy))
    ny, nx = rho.shape
    g = np.empty((9, ny, nx))
    lib().kbco_init_grad(nx, ny, float(beta), _p(rho), _p(ux), _p(uy), _p(g))
    return g


def step(g, variant: int, beta: float, nsteps: int = 1, gamma_mode: int = 0,
         gamma_fixed: float = 2.0, nthreads: int = 1, want_gamma: bool = False):
    """Advance a copy of g by nsteps; returns g (and the last step's gamma)."""
    g = _f64(g).copy()
    _, ny, nx = g.shape
    work = np.empty_like(g)
    gam = np.empty((ny, nx)) if want_gamma else None
    rc = lib().kbco_step(nx, ny, variant, float(beta), int(gamma_mode), float(gamma_fixed),
                         int(nsteps), _p(g), _p(work), _p(gam), int(nthreads))
    if rc != 0:
        raise ValueError("bad arguments")
    return (g, gam) if want_gamma else g


def macro(g):
    g = _f64(g)
    _, ny, nx = g.shape
    rho, ux, uy = np.empty((ny, nx)), np.empty((ny, nx)), np.empty((ny, nx))
    lib().kbco_macro(nx, ny, _p(g), _p(rho), _p(ux), _p(uy))
    return rho, ux, uy


DIAG_NAMES = ("mass", "px", "py", "E", "Z", "gamma_mean", "gamma_min", "gamma_max",
              "E_std", "Z_std")


def diagnostics(g, variant: int, beta: float, gamma_mode: int = 0,
                gamma_fixed: float = 2.0) -> np.ndarray:
    g = _f64(g)
    _, ny, nx = g.shape
    out = np.empty(10)
    rc = lib().kbco_diagnostics(nx, ny, variant, float(beta), int(gamma_mode),
                                float(gamma_fixed), _p(g), _p(out))
    if rc != 0:
        raise ValueError("bad arguments")
    return out


DIAG_EXT_NAMES = ("P", "P_std", "S", "S_std")


def diagnostics_ext(g) -> np.ndarray:
    """palinstrophy (mean, std) and entropy density of Eq. S (mean, std)."""
    g = _f64(g)
    _, ny, nx = g.shape
    out = np.empty(4)
    if lib().kbco_diagnostics_ext(nx, ny, _p(g), _p(out)) != 0:
        raise ValueError("bad arguments")
    return out


def adjoint(variant: int, beta: float, rho0, ux0, uy0, nsteps: int, objective: int = 0,
            utx=None, uty=None, gamma_mode: int = 0, gamma_fixed: float = 2.0):
    """J, dJ/du0 (ux, uy) and dJ/dbeta of the discrete forward map."""
    rho0, ux0, uy0 = (_f64(v) for v in (rho0, ux0, uy0))
    ny, nx = rho0.shape
    if objective == 1:
        utx, uty = _f64(utx), _f64(uty)
    else:
        utx = uty = np.zeros((ny, nx))
    J = np.zeros(1)
    gbeta = np.zeros(1)
    gux, guy = np.empty((ny, nx)), np.empty((ny, nx))
    rc = lib().kbco_adjoint(nx, ny, variant, float(beta), int(gamma_mode), float(gamma_fixed),
                            _p(rho0), _p(ux0), _p(uy0), int(nsteps), int(objective),
                            _p(utx), _p(uty), _p(J), _p(gux), _p(guy), _p(gbeta))
    if rc != 0:
        raise ValueError(f"oracle adjoint failed ({rc})")
    return float(J[0]), gux, guy, float(gbeta[0])
