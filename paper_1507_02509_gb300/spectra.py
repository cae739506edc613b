"""Shell-averaged energy and enstrophy spectra of a velocity field on the
device (the spectra of the paper's two-dimensional turbulence figures),
through the library's kbc_spectrum: cuFFT for the transform, the library's
own kernel for the shell sums.

E(k) = sum over wavevectors with round(|k|) = k of |u_hat(k)|^2 / 2, with
u_hat the discrete Fourier coefficients normalised by the node count, so that
sum_k E(k) = mean |u|^2 / 2 (Parseval); Z(k) = (2 pi k / N)^2 E(k).
"""
from __future__ import annotations

import math

import torch

from . import capi


def shell_count(n: int) -> int:
    """Number of shells round(|k|) of an n x n grid: round(n sqrt(2) / 2) + 1."""
    return int(round(n * math.sqrt(2.0) / 2.0)) + 1


def energy_spectrum(ux: torch.Tensor, uy: torch.Tensor):
    """(k, E(k), Z(k)) for a square periodic field on the current CUDA device;
    k = 0 .. round(N sqrt(2) / 2)."""
    n = ux.shape[-1]
    if ux.shape[-2] != n or uy.shape != ux.shape:
        raise ValueError("spectra need a square grid")
    dev = ux.device if ux.is_cuda else torch.device("cuda")
    u = torch.stack((ux.to(dev, torch.float64), uy.to(dev, torch.float64))).contiguous()
    nb = shell_count(n)
    E = torch.empty(nb, dtype=torch.float64, device=dev)
    Z = torch.empty(nb, dtype=torch.float64, device=dev)
    capi.kbc_spectrum(n, u, nb, E, Z, torch.cuda.current_stream(dev).cuda_stream)
    k = torch.arange(nb, dtype=torch.float64, device=dev)
    return k, E, Z
