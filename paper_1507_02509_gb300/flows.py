"""Seeded initial fields (rho, u) of the paper's three benchmark flows.

These generators hold none of the lattice Boltzmann arithmetic: they only
produce macroscopic fields in lattice units on a doubly periodic nx x ny grid
(node coordinates x = i, y = j, arrays ``[ny][nx]``, float64).  Both the CUDA
path and the CPU oracle take their inputs from here.

* Taylor-Green vortex (Sec. "Green-Taylor vortex flow"): the curl of
  (u0/k) cos(k x) cos(k y) with k = 2 pi m / N.
* Doubly periodic shear layer (Sec. "Doubly periodic shear layer"): tanh
  profiles of width 1/kappa and a sine perturbation of relative size delta.
* Decaying two-dimensional turbulence (Sec. "Decaying two-dimensional
  turbulence"): a zero-mean Gaussian random stream function with random
  Fourier phases whose velocity has the energy spectrum E(k), rescaled to a
  given rms speed.
"""
from __future__ import annotations

import math

import numpy as np


def taylor_green(nx: int, ny: int | None = None, u0: float = 0.04, modes: int = 1,
                 rho0: float = 1.0, pressure_rho: bool = False):
    """u = curl[(u0/k) cos(kx) cos(ky) e_z], k = 2 pi modes / nx (square grid).

    u_x = -u0 cos(kx) sin(ky), u_y = u0 sin(kx) cos(ky).  With
    ``pressure_rho`` the density carries the vortex's pressure field,
    rho = rho0 - rho0 u0^2 / (4 cs^2) (cos 2kx + cos 2ky) with cs^2 = 1/3,
    instead of a constant.
    """
    ny = nx if ny is None else ny
    if nx != ny:
        raise ValueError("Taylor-Green vortex needs a square grid")
    k = 2.0 * math.pi * modes / nx
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    ux = -u0 * np.cos(k * x) * np.sin(k * y)
    uy = u0 * np.sin(k * x) * np.cos(k * y)
    if pressure_rho:
        rho = rho0 - rho0 * u0 * u0 * 0.75 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    else:
        rho = np.full((ny, nx), rho0)
    return np.ascontiguousarray(rho), np.ascontiguousarray(ux), np.ascontiguousarray(uy)


def taylor_green_decay_rate(nu: float, n: int, modes: int = 1) -> float:
    """Amplitude decay rate nu (k1^2 + k2^2) = 2 nu k^2 of the vortex above."""
    k = 2.0 * math.pi * modes / n
    return 2.0 * nu * k * k


def taylor_green_k1k2(n: int, u0: float, k1: int = 1, k2: int = 4, t: float = 0.0,
                      nu: float = 0.0, rho0: float = 1.0, pressure_rho: bool = False):
    """The vortex of the paper's Green-Taylor section on [0, 2 pi)^2 sampled on
    an n x n grid (node x_i = 2 pi i / n): the curl of
    (u0/k2) cos(k1 x) cos(k2 y) exp(-nu (k1^2 + k2^2) t), i.e.
    u_x = -u0 cos(k1 x) sin(k2 y) e, u_y = u0 (k1/k2) sin(k1 x) cos(k2 y) e,
    with nu and t in lattice units (wavenumbers 2 pi k / n per node).
    Constant density rho0, or with ``pressure_rho`` the density that carries
    the vortex's pressure p = -(rho0 u0^2 / 4) (cos 2 k1 x + (k1/k2)^2 cos 2 k2 y)
    through p = cs^2 rho, cs^2 = 1/3."""
    x = 2.0 * math.pi * np.arange(n, dtype=np.float64)[None, :] / n
    y = 2.0 * math.pi * np.arange(n, dtype=np.float64)[:, None] / n
    kk = (2.0 * math.pi / n) ** 2 * (k1 * k1 + k2 * k2)
    e = math.exp(-nu * kk * t)
    ux = -u0 * np.cos(k1 * x) * np.sin(k2 * y) * e
    uy = u0 * (k1 / k2) * np.sin(k1 * x) * np.cos(k2 * y) * e
    if pressure_rho:
        p = -0.25 * rho0 * u0 * u0 * e * e * (np.cos(2 * k1 * x) + (k1 / k2) ** 2 * np.cos(2 * k2 * y))
        rho = rho0 + 3.0 * p
    else:
        rho = np.full((n, n), rho0)
    return np.ascontiguousarray(rho), np.ascontiguousarray(ux), np.ascontiguousarray(uy)


def shear_layer(n: int, u0: float = 0.04, kappa: float = 80.0, delta: float = 0.05,
                rho0: float = 1.0):
    """Doubly periodic shear layer on an n x n grid.

    u_x = u0 tanh(kappa (y/n - 1/4)) for y <= n/2, u0 tanh(kappa (3/4 - y/n))
    above; u_y = delta u0 sin(2 pi (x/n + 1/4)).
    """
    x = np.arange(n, dtype=np.float64)[None, :]
    y = np.arange(n, dtype=np.float64)[:, None]
    lower = u0 * np.tanh(kappa * (y / n - 0.25))
    upper = u0 * np.tanh(kappa * (0.75 - y / n))
    ux = np.where(y <= n / 2, lower, upper) * np.ones((1, n))
    uy = delta * u0 * np.sin(2 * math.pi * (x / n + 0.25)) * np.ones((n, 1))
    rho = np.full((n, n), rho0)
    return np.ascontiguousarray(rho), np.ascontiguousarray(ux), np.ascontiguousarray(uy)


def spectrum_k4_gauss(k, k0: float):
    """E(k) ~ k^4 exp(-2 (k/k0)^2)."""
    return k ** 4 * np.exp(-2.0 * (k / k0) ** 2)


def spectrum_paper(k, k0: float, A: float = 6.0, B: float = 17.0):
    """E(k) ~ k^A / (1 + (k/k0)^(B+1)), the paper's narrow-band spectrum."""
    return k ** A / (1.0 + (k / k0) ** (B + 1))


def _stream_coefficients(n: int, k0: float, seed: int, spectrum, kcut: int):
    """Random stream-function coefficients psi_hat[m, l] for |m|, |l| <= kcut
    (integer wavenumbers), amplitude sqrt(E(k) / (pi k^3)) and uniform phases.

    The block is drawn with numpy's PCG64 from ``seed`` and does not depend
    on n, so grids of different sizes share the same large scales.
    """
    rng = np.random.default_rng(seed)
    m = np.arange(-kcut, kcut + 1, dtype=np.float64)
    KX, KY = np.meshgrid(m, m, indexing="xy")  # KX along x (columns)
    K = np.hypot(KX, KY)
    phase = rng.uniform(0.0, 2.0 * math.pi, size=K.shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        amp = np.where(K > 0, np.sqrt(spectrum(K, k0) / (math.pi * K ** 3)), 0.0)
    coef = amp * np.exp(1j * phase)
    # a real field needs Hermitian symmetry: c(-k) = conj(c(k))
    coef = 0.5 * (coef + np.conj(coef[::-1, ::-1]))
    if 2 * kcut + 1 > n:
        raise ValueError("grid too small for the spectral cut-off")
    return KX, KY, coef


def turbulence(n: int, k0: float = 16.0, urms: float = 0.03, seed: int = 0,
               spectrum=spectrum_k4_gauss, kcut: int | None = None, rho0: float = 1.0,
               backend: str = "numpy", device=None):
    """Divergence-free random velocity on an n x n grid.

    psi has random phases and amplitudes from E(k); u = (d psi/dy,
    -d psi/dx) by spectral differentiation; the field is rescaled so that
    sqrt(mean |u|^2) = urms.  Wavenumbers above ``kcut`` (default
    min(8 k0, n/2 - 1)) are left empty; for the default spectrum their energy
    is below exp(-128) of the peak.

    backend "numpy" returns numpy arrays; backend "torch" evaluates the inverse
    FFT with torch on ``device`` (for very large grids) and returns torch
    float64 tensors.  Both take the same coefficients.
    """
    if kcut is None:
        kcut = int(min(8 * k0, n // 2 - 1))
    KX, KY, coef = _stream_coefficients(n, k0, seed, spectrum, kcut)
    # spectral derivatives of psi: u_x = d psi/dy = i ky psi, u_y = -i kx psi
    two_pi_n = 2.0 * math.pi / n
    cx = 1j * KY * two_pi_n * coef
    cy = -1j * KX * two_pi_n * coef
    idx = np.arange(-kcut, kcut + 1) % n
    if backend == "numpy":
        fields = []
        for c in (cx, cy):
            full = np.zeros((n, n), dtype=np.complex128)
            full[np.ix_(idx, idx)] = c
            fields.append(np.real(np.fft.ifft2(full)) * (n * n))
        ux, uy = fields
        scale = urms / math.sqrt(float(np.mean(ux * ux + uy * uy)))
        ux *= scale
        uy *= scale
        rho = np.full((n, n), rho0)
        return rho, np.ascontiguousarray(ux), np.ascontiguousarray(uy)
    if backend == "torch":
        import torch

        dev = torch.device(device if device is not None else "cuda")
        out = []
        iy = torch.as_tensor(idx, device=dev)
        for c in (cx, cy):
            full = torch.zeros((n, n), dtype=torch.complex128, device=dev)
            full[iy[:, None], iy[None, :]] = torch.as_tensor(c, device=dev)
            out.append(torch.fft.ifft2(full).real.mul_(n * n).contiguous())
            del full
        ux, uy = out
        scale = urms / math.sqrt(float((ux * ux + uy * uy).mean()))
        ux.mul_(scale)
        uy.mul_(scale)
        rho = torch.full((n, n), rho0, dtype=torch.float64, device=dev)
        return rho, ux, uy
    raise ValueError(f"unknown backend {backend!r}")
