"""GB300-native D2Q9 KBC entropic multi-relaxation lattice Boltzmann solver.

The hot path -- the fused pull-stream + KBC collide step of Bosch,
Chikatamarla and Karlin, "Entropic multi-relaxation models for simulation of
fluid turbulence" -- runs in hand-written sm_103a CUDA kernels behind the C
ABI of ``include/kbc.h``.  This package is the Python face of that ABI:

* ``capi``     -- ctypes binding with the C names (``kbc_create``, ...);
* ``Lattice``  -- a small object wrapper that allocates through PyTorch's
  caching allocator and runs on PyTorch's current CUDA stream;
* ``flows``    -- seeded initial fields of the paper's benchmark flows;
* ``build``    -- in-tree nvcc build of ``libkbc_gb300.so``.
"""
from __future__ import annotations

import ctypes
import math

from . import capi
from .capi import (KBC_A, KBC_B, KBC_C, KBC_D, KBC_F16_DEV, KBC_F32_DEV, KBC_F64,  # noqa: F401
                   KBC_GAMMA_ENTROPIC, KBC_GAMMA_FIXED, KBC_LBGK, KBCError)

VARIANTS = {"lbgk": KBC_LBGK, "A": KBC_A, "B": KBC_B, "C": KBC_C, "D": KBC_D}
DTYPES = {"f64": KBC_F64, "f32": KBC_F32_DEV, "f16": KBC_F16_DEV}
DIAG_NAMES = ("mass", "px", "py", "E", "Z", "gamma_mean", "gamma_min", "gamma_max",
              "E_std", "Z_std")
DIAG_EXT_NAMES = ("P", "P_std", "S", "S_std")


def beta_from_viscosity(nu: float) -> float:
    """nu = cs^2 (1/(2 beta) - 1/2) with cs^2 = 1/3 (Eq. viscosity), solved for beta."""
    return 1.0 / (6.0 * nu + 1.0)


def viscosity_from_beta(beta: float) -> float:
    return (1.0 / (2.0 * beta) - 0.5) / 3.0


def viscosity_for_reynolds(n: int, energy: float, reynolds: float) -> float:
    """nu from Re = N sqrt(2 E) / nu (turbulence section, E = mean |u|^2/2)."""
    return n * math.sqrt(2.0 * energy) / reynolds


# ---- PyTorch caching allocator as the library's device allocator ------------

_torch_hooks = None


def use_torch_allocator():
    """Route the library's device allocations through torch's caching allocator."""
    global _torch_hooks
    if _torch_hooks is not None:
        return
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream or 0))
        except Exception:  # out of memory: the library reports KBC_ERR_NOMEM
            return None

    def _free(p, stream, user):
        try:
            torch.cuda.caching_allocator_delete(int(p))
        except Exception:
            pass

    hooks = (capi.ALLOC_FN(_alloc), capi.FREE_FN(_free))
    capi.kbc_set_allocator(hooks[0], hooks[1], None)
    _torch_hooks = hooks


class Lattice:
    """One doubly periodic nx x ny D2Q9 field advanced on the GPU.

    variant: "lbgk" or "A".."D" (Table 1); dtype: "f64", "f32" (float
    deviations f - W) or "f16" (scaled half deviations).  beta is the
    relaxation parameter of Eq. Egeneral.  slab=True makes the field ny rows
    of a larger grid split into y-slabs, with ghost rows filled by halo
    exchange between steps (kbc_create_slab; see slabs.py).
    """

    def __init__(self, nx: int, ny: int, variant="B", beta: float = 0.99, dtype="f32",
                 stream=None, torch_allocator: bool = True, slab: bool = False):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("Lattice needs a CUDA device")
        capi.load()
        if torch_allocator:
            use_torch_allocator()
        self.nx, self.ny = int(nx), int(ny)
        self.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        self.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        self.beta = float(beta)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._stream = stream
        self.slab = bool(slab)
        create = capi.kbc_create_slab if self.slab else capi.kbc_create
        self.h = create(self.nx, self.ny, self.variant, self.beta, self.dtype)
        self._bind_stream()

    # -- plumbing
    def _bind_stream(self):
        import torch

        s = self._stream if self._stream is not None else torch.cuda.current_stream(self.device)
        capi.kbc_set_stream(self.h, ctypes.c_void_p(s.cuda_stream))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            capi.kbc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- configuration
    def set_gamma(self, gamma_fixed):
        """None: entropic gamma* (Eq. result21); "exact": root of Eq. result1;
        a number: gamma fixed to it."""
        if gamma_fixed is None:
            capi.kbc_set_gamma_mode(self.h, KBC_GAMMA_ENTROPIC, 2.0)
        elif gamma_fixed == "exact":
            capi.kbc_set_gamma_mode(self.h, capi.KBC_GAMMA_EXACT, 2.0)
        else:
            capi.kbc_set_gamma_mode(self.h, KBC_GAMMA_FIXED, float(gamma_fixed))

    def set_kernel(self, kernel: str):
        """"auto", "rows", "nodes" or "bulk" (see kbc_set_kernel)."""
        k = {"auto": capi.KBC_KERNEL_AUTO, "rows": capi.KBC_KERNEL_ROWS,
             "nodes": capi.KBC_KERNEL_NODES, "bulk": capi.KBC_KERNEL_BULK}[kernel]
        capi.kbc_set_kernel(self.h, k)

    def set_graph_steps(self, steps: int):
        """Steps per CUDA graph replayed by step() (even; 0 = no graphs)."""
        capi.kbc_set_graph_steps(self.h, steps)

    def set_guard(self, threshold: float):
        capi.kbc_set_guard(self.h, threshold)

    def guard_count(self) -> int:
        """Nodes re-evaluated in FP64 by the guard pass in the last step."""
        return capi.kbc_guard_count(self.h)

    def set_f16_scale(self, scale: float):
        capi.kbc_set_f16_scale(self.h, scale)

    # -- state
    @staticmethod
    def _velocity(ux, uy):
        import torch

        if hasattr(ux, "data_ptr"):
            return torch.stack((ux, uy)).to(torch.float64).contiguous()
        import numpy as np

        return np.ascontiguousarray(np.stack((ux, uy)).astype(np.float64))

    @staticmethod
    def _f64(x):
        import numpy as np

        if hasattr(x, "data_ptr"):
            import torch

            return x.to(torch.float64).contiguous()
        return np.ascontiguousarray(np.asarray(x, dtype=np.float64))

    def init(self, rho, ux, uy, grad: bool = False):
        """f = f^eq(rho, u) (or Grad's approximation with grad=True)."""
        self._bind_stream()
        rho = self._f64(rho)
        u = self._velocity(ux, uy)
        (capi.kbc_init_grad if grad else capi.kbc_init)(self.h, rho, u)
        self._keep = (rho, u)  # alive until the stream has consumed them
        return self

    def step(self, n: int = 1):
        self._bind_stream()
        capi.kbc_step(self.h, n)
        return self

    def sync(self, timeout_s: float = 0.0):
        capi.kbc_sync(self.h, timeout_s)

    def moments(self):
        """(rho, ux, uy) as float64 CUDA tensors."""
        import torch

        self._bind_stream()
        rho = torch.empty((self.ny, self.nx), dtype=torch.float64, device=self.device)
        u = torch.empty((2, self.ny, self.nx), dtype=torch.float64, device=self.device)
        capi.kbc_moments(self.h, rho, u)
        return rho, u[0], u[1]

    def populations(self):
        """f[9][ny][nx] as a float64 CUDA tensor."""
        import torch

        self._bind_stream()
        f = torch.empty((9, self.ny, self.nx), dtype=torch.float64, device=self.device)
        capi.kbc_get_populations(self.h, f)
        return f

    def probe(self, nodes):
        """f[k][9] (float64 numpy) of node indices y * nx + x."""
        import numpy as np

        nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.int64))
        out = np.empty((nodes.size, 9))
        self._bind_stream()
        capi.kbc_probe(self.h, nodes.size, nodes, out)
        return out

    def set_populations(self, f):
        self._bind_stream()
        f = self._f64(f)
        capi.kbc_set_populations(self.h, f)
        self._keep = (f,)

    def diagnostics(self) -> dict:
        import numpy as np

        self._bind_stream()
        out = np.zeros(capi.KBC_DIAG_N)
        capi.kbc_diagnostics(self.h, out)
        return dict(zip(DIAG_NAMES, out.tolist()))

    def diagnostics_ext(self) -> dict:
        """Palinstrophy and entropy density (mean and spatial std)."""
        import numpy as np

        self._bind_stream()
        out = np.zeros(capi.KBC_DIAG_EXT_N)
        capi.kbc_diagnostics_ext(self.h, out)
        return dict(zip(DIAG_EXT_NAMES, out.tolist()))

    @property
    def bytes_per_update(self) -> float:
        return capi.kbc_bytes_per_update(self.h)

    @property
    def halo_bytes(self) -> int:
        """Bytes of one face's halo of a y-slab handle ([3][nx] stored elements)."""
        return capi.kbc_halo_bytes(self.h)

    @property
    def full_halo_bytes(self) -> int:
        """Bytes of one face's full halo ([9][nx] stored elements)."""
        return capi.kbc_halo_bytes(self.h, 1)

    def diagnostics_partial(self):
        """This handle's nodes as one partial diagnostics set (float64 numpy,
        KBC_DIAG_PART_N values; combine with kbc_diagnostics_merge)."""
        import numpy as np

        self._bind_stream()
        out = np.zeros(capi.KBC_DIAG_PART_N)
        capi.kbc_diagnostics_partial(self.h, out)
        return out
