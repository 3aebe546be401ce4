"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds no arithmetic of the lattice Boltzmann method or of its
boundary treatments: it only draws the initial velocity fields and particle
layouts that stand in for the data the paper used (the de Motta et al.
decaying-turbulence field and particle positions of Sec. 3.1, and the
developed pipe flow of Sec. 2.1, neither of which is available). Every
random number comes from numpy's PCG64 generator seeded by the caller.

Array layout used everywhere in this project: a scalar field of an
``nx*ny*nz`` grid is stored with x fastest, ``idx = x + nx*(y + ny*z)``; a
vector field is three such planes, component-major (``u[c*N + idx]``), which
as a numpy array is ``u[c, z, y, x]``.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "hit_velocity",
    "pipe_velocity",
    "place_spheres",
    "noise_velocity",
    "random_populations",
    "PIPE_148",
    "HIT_256",
    "HIT_512",
    "SPHERE_32",
]


def _wavenumbers(n: int) -> np.ndarray:
    return np.fft.fftfreq(n, d=1.0 / n)


def hit_velocity(n: int, seed: int, k_peak: float = 8.0, u_rms: float = 0.03,
                 dtype=np.float64) -> np.ndarray:
    """Random solenoidal periodic field on an n^3 grid, shape (3, n, n, n).

    Fourier amplitudes are complex Gaussians, projected onto the plane normal
    to k (divergence-free), and rescaled shell by shell (shells of integer
    |k|) so the shell energy follows E(k) ~ k^4 exp(-2 (k/k_peak)^2). The real
    field is then scaled so that u_rms = sqrt(<u.u>/3) equals ``u_rms``.
    """
    rng = np.random.default_rng(seed)
    k = _wavenumbers(n)
    kr = np.fft.rfftfreq(n, d=1.0 / n)
    kz, ky, kx = np.meshgrid(k, k, kr, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    shape = k2.shape
    a = (rng.standard_normal((3,) + shape) + 1j * rng.standard_normal((3,) + shape))
    a = a.astype(np.complex128)
    kdota = kx * a[0] + ky * a[1] + kz * a[2]
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.where(k2 > 0, 1.0 / k2, 0.0)
    a[0] -= kx * kdota * inv
    a[1] -= ky * kdota * inv
    a[2] -= kz * kdota * inv
    a[:, k2 == 0] = 0.0
    # Nyquist modes have no divergence-free real counterpart: drop them
    nyq = (np.abs(kx) >= n / 2) | (np.abs(ky) >= n / 2) | (np.abs(kz) >= n / 2)
    a[:, nyq] = 0.0
    kmag = np.sqrt(k2)
    shell = np.rint(kmag).astype(np.int64)
    # the half spectrum counts every mode with kx>0 twice
    mult = np.where((kx > 0) & (kx < n / 2), 2.0, 1.0)
    e_mode = 0.5 * mult * (np.abs(a[0]) ** 2 + np.abs(a[1]) ** 2 + np.abs(a[2]) ** 2)
    nshell = shell.max() + 1
    e_shell = np.bincount(shell.ravel(), weights=e_mode.ravel(), minlength=nshell)
    ks = np.arange(nshell, dtype=np.float64)
    target = ks ** 4 * np.exp(-2.0 * (ks / k_peak) ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        fac = np.where(e_shell > 0, np.sqrt(target / e_shell), 0.0)
    a *= fac[shell][None]
    u = np.empty((3, n, n, n), dtype=np.float64)
    for c in range(3):
        u[c] = np.fft.irfftn(a[c], s=(n, n, n), axes=(0, 1, 2))
    rms = math.sqrt(float(np.mean(u[0] ** 2 + u[1] ** 2 + u[2] ** 2)) / 3.0)
    u *= u_rms / rms
    return u.astype(dtype, copy=False)


def pipe_velocity(nx: int, ny: int, nz: int, radius: float, u_bulk: float,
                  perturbation: float = 0.05, seed: int = 0) -> np.ndarray:
    """Initial pipe field, shape (3, nz, ny, nx): axis along z through
    ((nx-1)/2, (ny-1)/2).

    A parabolic streamwise profile with bulk velocity ``u_bulk`` inside
    r < radius plus a divergence-free perturbation: the spectral curl of a
    random vector potential tapered by (1 - r^2/R^2)^2, scaled so that its rms
    over the pipe interior is ``perturbation * u_bulk``.
    """
    rng = np.random.default_rng(seed)
    cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
    x = np.arange(nx, dtype=np.float64) - cx
    y = np.arange(ny, dtype=np.float64) - cy
    r2 = (y[:, None] ** 2 + x[None, :] ** 2)
    inside = r2 < radius * radius
    prof = np.where(inside, 2.0 * u_bulk * (1.0 - r2 / (radius * radius)), 0.0)
    taper = np.where(inside, (1.0 - r2 / (radius * radius)) ** 2, 0.0)
    u = np.zeros((3, nz, ny, nx), dtype=np.float64)
    u[2] = prof[None, :, :]
    if perturbation > 0.0:
        # smooth random potential: low-pass Gaussian noise in Fourier space
        kz = _wavenumbers(nz)[:, None, None]
        ky = _wavenumbers(ny)[None, :, None]
        kx = _wavenumbers(nx)[None, None, :]
        k2 = kx * kx + ky * ky + kz * kz
        lowpass = np.exp(-k2 / (2.0 * 6.0 ** 2))
        pot = []
        for _ in range(3):
            w = rng.standard_normal((nz, ny, nx))
            w = np.real(np.fft.ifftn(np.fft.fftn(w) * lowpass))
            pot.append(w * taper[None, :, :])
        fa = [np.fft.fftn(p) for p in pot]
        tx = 2.0 * np.pi * kx / nx
        ty = 2.0 * np.pi * ky / ny
        tz = 2.0 * np.pi * kz / nz
        cur = [
            np.real(np.fft.ifftn(1j * (ty * fa[2] - tz * fa[1]))),
            np.real(np.fft.ifftn(1j * (tz * fa[0] - tx * fa[2]))),
            np.real(np.fft.ifftn(1j * (tx * fa[1] - ty * fa[0]))),
        ]
        pert = np.stack(cur)
        pert *= inside[None, None, :, :]
        rms = math.sqrt(float(np.sum(pert ** 2)) / max(1, int(inside.sum()) * nz))
        if rms > 0:
            pert *= perturbation * u_bulk / rms
        u += pert
    return u


def place_spheres(box, n_particles: int, radius: float, min_gap: float,
                  seed: int, max_tries: int = 2_000_000) -> np.ndarray:
    """Random sequential placement of non-overlapping spheres in a periodic
    box; returns centres, shape (n, 3) as (x, y, z). Any two centres are at
    least 2*radius + min_gap apart (minimum image)."""
    rng = np.random.default_rng(seed)
    box = np.asarray(box, dtype=np.float64)
    dmin = 2.0 * radius + min_gap
    out = np.empty((n_particles, 3), dtype=np.float64)
    m = 0
    tries = 0
    while m < n_particles:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place spheres: volume fraction too high")
        p = rng.random(3) * box
        if m:
            d = out[:m] - p
            d -= box * np.rint(d / box)
            if np.min(np.einsum("ij,ij->i", d, d)) < dmin * dmin:
                continue
        out[m] = p
        m += 1
    return out


def noise_velocity(shape_zyx, amplitude: float, seed: int) -> np.ndarray:
    """Uniform velocity noise in [-amplitude, amplitude] per component,
    shape (3, nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape_zyx
    return rng.uniform(-amplitude, amplitude, size=(3, nz, ny, nx))


def random_populations(ncell: int, seed: int, lo: float = 0.01, hi: float = 0.1) -> np.ndarray:
    """Arbitrary positive populations, shape (19, ncell): a state far from any
    equilibrium, for single-step comparisons of the collision."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(19, ncell))


# Workload descriptions (sizes and parameters of the synthetic stand-ins).
SPHERE_32 = dict(n=32, radius=4.0, centre=(15.5, 15.5, 15.5), force=(1e-6, 0.0, 0.0),
                 tau=0.6, noise=1e-4, steps=500)
PIPE_148 = dict(nx=148, ny=148, nz=438, radius=73.0, nu=0.0032, re_tau=180.0,
                perturbation=0.05)
HIT_256 = dict(n=256, n_particles=2000, radius=4.0, density_ratio=5.0, tau=0.51,
               u_rms=0.03, k_peak=8.0, min_gap=1.0)
HIT_512 = dict(n=512, n_particles=16000, radius=4.0, density_ratio=5.0, tau=0.51,
               u_rms=0.03, k_peak=8.0, min_gap=1.0)


def pipe_parameters(radius: float = 73.0, nu: float = 0.0032, re_tau: float = 180.0):
    """Derived pipe-flow parameters (Sec. 2.1, Table 1): friction velocity
    from Re_tau = u_tau R / nu, body force from the stationary force balance
    2 pi R L tau_w = pi R^2 L rho g, i.e. g = 2 u_tau^2 / R, and the bulk
    velocity U_b = 14.7 u_tau of the reported turbulent state."""
    u_tau = re_tau * nu / radius
    g = 2.0 * u_tau * u_tau / radius
    tau = 3.0 * nu + 0.5
    return dict(u_tau=u_tau, g=g, tau=tau, u_bulk=14.7 * u_tau)
