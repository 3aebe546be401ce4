"""Oracle of the three-dimensional spectra of kinetic energy and dissipation
(test infrastructure).

TEST INFRASTRUCTURE ONLY: plain numpy statement of the spectra that the CUDA
library computes with its own FFT kernels. The paper compares 3D spectra of
the turbulent kinetic energy and of the dissipation rate between IBB and IBM,
with the velocity inside the particles masked or not (Sec. 3.2). Reading:

- Fourier coefficients of each velocity component on the periodic n^3 box,
  u_hat(k) = (1/N) sum_x u(x) exp(-2 pi i k.x / n), N = n^3, integer wave
  vectors k with components in (-n/2, n/2];
- E(K) = sum over |k| in the shell K (|k| rounded to the nearest integer)
  of (1/2) |u_hat(k)|^2 summed over the three components, so that
  sum_K E(K) = (1/2) <|u|^2> (Parseval);
- D(K) = sum over the same shell of 2 nu |kappa|^2 (1/2) |u_hat(k)|^2 with
  the physical wavenumber kappa = 2 pi k / n (lattice units), so that
  sum_K D(K) = nu <|grad u|^2>, the spectral dissipation of an
  incompressible field.
"""
from __future__ import annotations

import numpy as np


def shells(n: int):
    """Shell index round(|k|) of every wave vector of an n^3 FFT (numpy
    layout, axes (z, y, x)) and |kappa|^2."""
    k1 = np.fft.fftfreq(n, d=1.0 / n)  # 0, 1, ..., n/2 - 1, -n/2, ..., -1
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    shell = np.floor(np.sqrt(k2) + 0.5).astype(np.int64)
    kappa2 = (2.0 * np.pi / n) ** 2 * k2
    return shell, kappa2


def spectra(u, n: int, nu: float, nbins: int):
    """u: velocity, shape (3, n*n*n) (x fastest) or (3, n, n, n) as (z, y,
    x). Returns E, D of length nbins (shells beyond nbins - 1 dropped)."""
    u = np.asarray(u, dtype=np.float64).reshape(3, n, n, n)
    shell, kappa2 = shells(n)
    N = float(n) ** 3
    e = np.zeros((n, n, n))
    for d in range(3):
        uh = np.fft.fftn(u[d]) / N
        e += 0.5 * (uh.real ** 2 + uh.imag ** 2)
    keep = shell < nbins
    E = np.bincount(shell[keep], weights=e[keep], minlength=nbins)[:nbins]
    D = np.bincount(shell[keep], weights=(2.0 * nu * kappa2 * e)[keep], minlength=nbins)[:nbins]
    return E, D
