"""ctypes binding of the C ABI in ``include/kbc.h`` (same names, argument
marshalling only).

Every computation runs in ``libkbc_gb300.so``; this module never computes a
lattice Boltzmann quantity itself and has no fallback: if the library is
missing it raises.  Pointers may be torch tensors (CUDA or CPU), numpy
arrays, or raw integers.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkbc_gb300.so")

KBC_LBGK, KBC_A, KBC_B, KBC_C, KBC_D = 0, 1, 2, 3, 4
KBC_F64, KBC_F32_DEV, KBC_F16_DEV = 0, 1, 2
KBC_GAMMA_ENTROPIC, KBC_GAMMA_FIXED, KBC_GAMMA_EXACT = 0, 1, 2
KBC_OK, KBC_ERR_ARG, KBC_ERR_CUDA, KBC_ERR_NOMEM = 0, -1, -2, -3
KBC_ERR_NONFINITE, KBC_ERR_TIMEOUT, KBC_ERR_STATE = -4, -5, -6
KBC_DIAG_N = 10
KBC_DIAG_EXT_N = 4
KBC_DIAG_PART_N = 11
KBC_KERNEL_AUTO, KBC_KERNEL_ROWS, KBC_KERNEL_NODES, KBC_KERNEL_BULK = 0, 1, 2, 3

STATUS_NAMES = {
    0: "KBC_OK", -1: "KBC_ERR_ARG", -2: "KBC_ERR_CUDA", -3: "KBC_ERR_NOMEM",
    -4: "KBC_ERR_NONFINITE", -5: "KBC_ERR_TIMEOUT", -6: "KBC_ERR_STATE",
}

# every entry point of include/kbc.h: name -> (restype, argtypes)
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
SIGNATURES = {
    "kbc_set_allocator": (_i, [ALLOC_FN, FREE_FN, _vp]),
    "kbc_create": (_i, [_i, _i, _i, _d, _i, ctypes.POINTER(_vp)]),
    "kbc_create_slab": (_i, [_i, _i, _i, _d, _i, ctypes.POINTER(_vp)]),
    "kbc_halo_send": (_i, [_vp, _i, _i, _vp]),
    "kbc_halo_recv": (_i, [_vp, _i, _i, _vp]),
    "kbc_halo_bytes": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_size_t)]),
    "kbc_destroy": (_i, [_vp]),
    "kbc_set_stream": (_i, [_vp, _vp]),
    "kbc_set_gamma_mode": (_i, [_vp, _i, _d]),
    "kbc_set_kernel": (_i, [_vp, _i]),
    "kbc_set_graph_steps": (_i, [_vp, _i]),
    "kbc_set_guard": (_i, [_vp, _d]),
    "kbc_guard_count": (_i, [_vp, ctypes.POINTER(ctypes.c_longlong)]),
    "kbc_set_f16_scale": (_i, [_vp, _d]),
    "kbc_init": (_i, [_vp, _vp, _vp]),
    "kbc_init_grad": (_i, [_vp, _vp, _vp]),
    "kbc_set_populations": (_i, [_vp, _vp]),
    "kbc_get_populations": (_i, [_vp, _vp]),
    "kbc_step": (_i, [_vp, _i]),
    "kbc_sync": (_i, [_vp, _d]),
    "kbc_probe": (_i, [_vp, _i, _vp, _vp]),
    "kbc_moments": (_i, [_vp, _vp, _vp]),
    "kbc_diagnostics": (_i, [_vp, _vp]),
    "kbc_diagnostics_ext": (_i, [_vp, _vp]),
    "kbc_diagnostics_partial": (_i, [_vp, _vp]),
    "kbc_diagnostics_merge": (_i, [_i, _vp, _vp]),
    "kbc_spectrum": (_i, [_i, _vp, _i, _vp, _vp, _vp]),
    "kbc_diagnostics_noalloc": (_i, [_i, _i, _i, _d, _vp, _vp, _vp]),
    "kbc_adjoint": (_i, [_vp, _vp, _vp, _i, _i, _i, _vp, ctypes.POINTER(_d), _vp,
                         ctypes.POINTER(_d)]),
    "kbc_bytes_per_update": (_i, [_vp, ctypes.POINTER(_d)]),
    "kbc_fp64_fma_rate": (_i, [_vp, ctypes.POINTER(_d)]),
    "kbc_last_error": (ctypes.c_char_p, [_vp]),
}

_lock = threading.Lock()
_lib = None


class KBCError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(
                    f"{p} is missing: build the CUDA library first "
                    "(python -c 'import __graft_entry__ as g; g.build()')")
            L = ctypes.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def ptr(x) -> int | None:
    """Address of a torch tensor / numpy array / integer (None stays None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)!r}")


def check(h, status: int):
    if status != KBC_OK:
        msg = load().kbc_last_error(h)
        raise KBCError(status, msg.decode() if msg else "")
    return status


# ---- thin wrappers, one per entry point -----------------------------------

def kbc_set_allocator(alloc, release, user=None):
    return check(None, load().kbc_set_allocator(alloc, release, user))


def kbc_create(nx: int, ny: int, variant: int, beta: float, dtype: int):
    h = ctypes.c_void_p()
    check(None, load().kbc_create(int(nx), int(ny), int(variant), float(beta), int(dtype),
                                  ctypes.byref(h)))
    return h


def kbc_create_slab(nx: int, ny: int, variant: int, beta: float, dtype: int):
    h = ctypes.c_void_p()
    check(None, load().kbc_create_slab(int(nx), int(ny), int(variant), float(beta), int(dtype),
                                       ctypes.byref(h)))
    return h


def kbc_halo_send(h, face: int, full: int, buf):
    return check(h, load().kbc_halo_send(h, int(face), int(full), ptr(buf)))


def kbc_halo_recv(h, face: int, full: int, buf):
    return check(h, load().kbc_halo_recv(h, int(face), int(full), ptr(buf)))


def kbc_halo_bytes(h, full: int = 0) -> int:
    b = ctypes.c_size_t()
    check(h, load().kbc_halo_bytes(h, int(full), ctypes.byref(b)))
    return b.value


def kbc_destroy(h):
    return check(h, load().kbc_destroy(h))


def kbc_set_stream(h, stream):
    return check(h, load().kbc_set_stream(h, stream))


def kbc_set_gamma_mode(h, mode: int, gamma_fixed: float = 2.0):
    return check(h, load().kbc_set_gamma_mode(h, int(mode), float(gamma_fixed)))


def kbc_set_kernel(h, kernel: int):
    return check(h, load().kbc_set_kernel(h, int(kernel)))


def kbc_set_graph_steps(h, steps: int):
    return check(h, load().kbc_set_graph_steps(h, int(steps)))


def kbc_set_guard(h, threshold: float):
    return check(h, load().kbc_set_guard(h, float(threshold)))


def kbc_guard_count(h) -> int:
    c = ctypes.c_longlong()
    check(h, load().kbc_guard_count(h, ctypes.byref(c)))
    return c.value


def kbc_set_f16_scale(h, scale: float):
    return check(h, load().kbc_set_f16_scale(h, float(scale)))


def kbc_init(h, rho, u):
    return check(h, load().kbc_init(h, ptr(rho), ptr(u)))


def kbc_init_grad(h, rho, u):
    return check(h, load().kbc_init_grad(h, ptr(rho), ptr(u)))


def kbc_set_populations(h, f):
    return check(h, load().kbc_set_populations(h, ptr(f)))


def kbc_get_populations(h, f):
    return check(h, load().kbc_get_populations(h, ptr(f)))


def kbc_step(h, nsteps: int):
    return check(h, load().kbc_step(h, int(nsteps)))


def kbc_sync(h, timeout_s: float = 0.0):
    return check(h, load().kbc_sync(h, float(timeout_s)))


def kbc_probe(h, count: int, nodes, f):
    return check(h, load().kbc_probe(h, int(count), ptr(nodes), ptr(f)))


def kbc_moments(h, rho, u):
    return check(h, load().kbc_moments(h, ptr(rho), ptr(u)))


def kbc_diagnostics(h, out):
    return check(h, load().kbc_diagnostics(h, ptr(out)))


def kbc_diagnostics_ext(h, out):
    return check(h, load().kbc_diagnostics_ext(h, ptr(out)))


def kbc_diagnostics_partial(h, out):
    return check(h, load().kbc_diagnostics_partial(h, ptr(out)))


def kbc_diagnostics_merge(n: int, parts, out):
    return check(None, load().kbc_diagnostics_merge(int(n), ptr(parts), ptr(out)))


def kbc_spectrum(n: int, u, nbins: int, E, Z, stream=None):
    return check(None, load().kbc_spectrum(int(n), ptr(u), int(nbins), ptr(E), ptr(Z),
                                           ptr(stream)))


def kbc_diagnostics_noalloc(nx: int, ny: int, variant: int, beta: float, f, out,
                            stream=None):
    """Diagnostics of a caller-owned FP64 device field, no device allocation."""
    return check(None, load().kbc_diagnostics_noalloc(int(nx), int(ny), int(variant), float(beta),
                                                      ptr(f), ptr(out), stream))


def kbc_adjoint(h, rho0, u0, nsteps: int, ckpt_every: int, objective: int, u_target,
                grad_u0):
    """Returns (J, dJ/dbeta); dJ/du0 is written into grad_u0 [2][ny][nx]."""
    J = ctypes.c_double()
    gb = ctypes.c_double()
    check(h, load().kbc_adjoint(h, ptr(rho0), ptr(u0), int(nsteps), int(ckpt_every),
                                int(objective), ptr(u_target), ctypes.byref(J), ptr(grad_u0),
                                ctypes.byref(gb)))
    return J.value, gb.value


def kbc_bytes_per_update(h) -> float:
    b = ctypes.c_double()
    check(h, load().kbc_bytes_per_update(h, ctypes.byref(b)))
    return b.value


def kbc_fp64_fma_rate(stream=None) -> float:
    """Measured thread DFMA operations per second of the current device."""
    r = ctypes.c_double()
    st = load().kbc_fp64_fma_rate(stream, ctypes.byref(r))
    if st != KBC_OK:
        raise KBCError(st, "kbc_fp64_fma_rate failed")
    return r.value


def kbc_last_error(h) -> str:
    m = load().kbc_last_error(h)
    return m.decode() if m else ""
