"""The seeded input generators (paper_1507_02509_gb300/flows.py) against the
recipe they state: the decaying-turbulence field is divergence-free, has the
requested u_rms and the energy spectrum E(k) it draws from (shell sums by the
oracle's plain spectrum routine), is the same on both backends and on grids of
different sizes; the shear layer follows its printed formula."""
import math

import numpy as np
import pytest

import oracle.spectra as OS
from paper_1507_02509_gb300 import flows


def _modes(u, n):
    return np.fft.fft2(u) / (n * n)


def test_turbulence_divergence_free_with_requested_rms():
    n, urms = 128, 0.03
    _, ux, uy = flows.turbulence(n, k0=8, urms=urms, seed=4)
    assert math.sqrt(float(np.mean(ux * ux + uy * uy))) == pytest.approx(urms, rel=1e-13)
    k = np.fft.fftfreq(n, 1.0 / n)
    KX, KY = np.meshgrid(k, k, indexing="xy")
    uh, vh = _modes(ux, n), _modes(uy, n)
    div = np.abs(KX * uh + KY * vh)
    scale = np.max(np.hypot(KX, KY) * np.hypot(np.abs(uh), np.abs(vh)))
    assert np.max(div) <= 1e-12 * scale


@pytest.mark.parametrize("spectrum,k0", [(flows.spectrum_k4_gauss, 16.0),
                                          (flows.spectrum_paper, 12.0)])
def test_turbulence_shell_spectrum_follows_the_drawn_spectrum(spectrum, k0):
    """Each stream-function mode has amplitude sqrt(E(k)/(pi k^3)) and a
    random phase; Hermitian symmetrisation leaves a random cos^2 factor of
    mean 1/2.  The expected shell energy is therefore proportional to the sum
    of E(|k|)/|k| over the shell's integer wavevectors: the measured shells
    between k0/2 and 2 k0 follow it within the sampling spread of about a
    hundred modes per shell, and the most energetic shell lies near the
    spectrum's peak."""
    n = 256
    _, ux, uy = flows.turbulence(n, k0=k0, urms=0.03, seed=9, spectrum=spectrum)
    k, E, _ = OS.energy_spectrum(ux, uy)
    expect = np.zeros_like(E)
    m = np.arange(-(n // 2) + 1, n // 2)
    MX, MY = np.meshgrid(m, m)
    K = np.hypot(MX, MY)
    nz = K > 0
    shells = np.rint(K[nz]).astype(int)
    np.add.at(expect, shells, spectrum(K[nz], k0) / K[nz])
    band = (k >= k0 / 2) & (k <= 2 * k0)
    ratio = (E[band] / E[band].sum()) / (expect[band] / expect[band].sum())
    assert np.all(np.abs(ratio - 1.0) < 0.45), ratio
    assert abs(np.mean(ratio) - 1.0) < 0.1
    kpeak = k[np.argmax(E)]
    kstar = k[np.argmax(expect)]
    assert abs(kpeak - kstar) <= 0.25 * kstar


def test_turbulence_backends_agree():
    torch = pytest.importorskip("torch")
    n = 96
    _, ux, uy = flows.turbulence(n, k0=6, urms=0.03, seed=2)
    _, tx, ty = flows.turbulence(n, k0=6, urms=0.03, seed=2, backend="torch", device="cpu")
    assert isinstance(tx, torch.Tensor)
    assert np.max(np.abs(tx.numpy() - ux)) <= 1e-15
    assert np.max(np.abs(ty.numpy() - uy)) <= 1e-15


def test_turbulence_large_scales_do_not_depend_on_the_grid():
    """The coefficient block depends on the seed and the cut-off only, so a
    band-limited field sampled on a grid twice as fine agrees at the common
    nodes after the u_rms rescaling."""
    _, ux, uy = flows.turbulence(64, k0=3, urms=0.03, seed=7, kcut=8)
    _, vx, vy = flows.turbulence(128, k0=3, urms=0.03, seed=7, kcut=8)
    assert np.max(np.abs(vx[::2, ::2] - ux)) <= 1e-15
    assert np.max(np.abs(vy[::2, ::2] - uy)) <= 1e-15


def test_shear_layer_follows_the_printed_formula():
    """u_x = u0 tanh(kappa (y/N - 1/4)) for y <= N/2, u0 tanh(kappa (3/4 - y/N))
    above, u_y = delta u0 sin(2 pi (x/N + 1/4)); node coordinates x = i, y = j."""
    n, u0, kappa, delta = 64, 0.04, 80.0, 0.05
    rho, ux, uy = flows.shear_layer(n, u0=u0, kappa=kappa, delta=delta)
    assert np.all(rho == 1.0)
    assert np.all(ux[n // 4] == 0.0) and np.all(ux[3 * n // 4] == 0.0)
    assert ux[n // 2, 0] == u0 * math.tanh(kappa * 0.25)          # y = N/2: lower branch
    assert ux[n // 2 + 1, 0] == u0 * math.tanh(kappa * (0.75 - (n // 2 + 1) / n))
    assert np.all(ux == ux[:, :1])                                   # depends on y only
    assert uy[0, 0] == pytest.approx(delta * u0, rel=1e-15)          # sin(pi/2)
    assert uy[0, n // 4] == pytest.approx(0.0, abs=1e-18)
    assert np.all(uy == uy[:1, :])                                   # depends on x only
