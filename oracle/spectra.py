"""Shell-averaged spectra in plain numpy -- TEST INFRASTRUCTURE ONLY.

E(k) = sum over integer wavevectors with round(|k|) = k of |u_hat|^2 / 2,
u_hat = fft2(u) / N^2; Z(k) = (2 pi k / N)^2 E(k).  Written with an explicit
loop over wavevectors (slow, plain).
"""
import math

import numpy as np


def energy_spectrum(ux, uy):
    n = ux.shape[1]
    uh = np.fft.fft2(ux) / (n * n)
    vh = np.fft.fft2(uy) / (n * n)
    freqs = [m if m <= n // 2 else m - n for m in range(n)]
    kmax = int(round(math.sqrt(2) * (n // 2)))
    E = np.zeros(kmax + 1)
    for a in range(n):
        for b in range(n):
            k = int(round(math.hypot(freqs[a], freqs[b])))
            E[k] += 0.5 * (abs(uh[a, b]) ** 2 + abs(vh[a, b]) ** 2)
    k = np.arange(kmax + 1, dtype=float)
    return k, E, (2 * math.pi * k / n) ** 2 * E
