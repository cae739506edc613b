"""Shell-averaged energy and enstrophy spectra of a velocity field on the
device (the spectra of the paper's turbulence figures).

E(k) = sum over wavevectors with round(|k|) = k of |u_hat(k)|^2 / 2, with
u_hat the discrete Fourier coefficients normalised by the node count, so that
sum_k E(k) = mean |u|^2 / 2 (Parseval); Z(k) = (2 pi k / N)^2 E(k).  The FFT
is cuFFT through torch (a library step); the binning is a scatter-add.
"""
from __future__ import annotations

import math

import torch


def energy_spectrum(ux: torch.Tensor, uy: torch.Tensor):
    """(k, E(k), Z(k)) for a square periodic field; k = 0 .. N/2 * sqrt(2)."""
    n = ux.shape[-1]
    if ux.shape[-2] != n:
        raise ValueError("spectra need a square grid")
    uh = torch.fft.fft2(ux.to(torch.float64)) / (n * n)
    vh = torch.fft.fft2(uy.to(torch.float64)) / (n * n)
    e = 0.5 * (uh.real ** 2 + uh.imag ** 2 + vh.real ** 2 + vh.imag ** 2)
    f = torch.fft.fftfreq(n, d=1.0 / n, device=ux.device, dtype=torch.float64)
    kk = torch.sqrt(f[:, None] ** 2 + f[None, :] ** 2)
    shell = torch.round(kk).to(torch.int64)
    nbins = int(shell.max().item()) + 1
    E = torch.zeros(nbins, dtype=torch.float64, device=ux.device)
    E.scatter_add_(0, shell.reshape(-1), e.reshape(-1))
    k = torch.arange(nbins, dtype=torch.float64, device=ux.device)
    Z = (2.0 * math.pi * k / n) ** 2 * E
    return k, E, Z
