"""Oracle of the pipe's radial profiles (test infrastructure).

TEST INFRASTRUCTURE ONLY: plain numpy statement of the binned profiles the
CUDA library computes. The paper reports pipe statistics against the radial
position (Sec. 2.2: mean streamwise velocity, velocity fluctuations,
dissipation rate). Reading, for the cells inside the pipe (not solid):

- r = sqrt(dx^2 + dy^2), dx = x - c_x, dy = y - c_y (axis along z), bin
  b = floor(r * nbins / R);
- cylindrical components u_r = (u_x dx + u_y dy) / r,
  u_theta = (u_y dx - u_x dy) / r (u_r = u_x, u_theta = u_y on the axis);
- per bin the mean over its cells of: 1 (the count is returned), u_r,
  u_theta, u_z, u_r^2, u_theta^2, u_z^2, u_r u_z, u_r u_theta,
  u_theta u_z, rho, and 2 nu s_ij s_ij with second-order central
  differences of the statistics velocity (the field of lbm_stats, periodic
  wrap).
Quantities in that order (NQ = 12); empty bins hold zeros.
"""
from __future__ import annotations

import numpy as np

NQ = 12


def cell_dissipation(u, nx, ny, nz, nu):
    """2 nu s_ij s_ij per cell, central differences, u shape (3, N)."""
    U = np.asarray(u, dtype=np.float64).reshape(3, nz, ny, nx)
    g = np.empty((3, 3, nz, ny, nx))
    for a in range(3):
        g[a, 0] = 0.5 * (np.roll(U[a], -1, axis=2) - np.roll(U[a], 1, axis=2))
        g[a, 1] = 0.5 * (np.roll(U[a], -1, axis=1) - np.roll(U[a], 1, axis=1))
        g[a, 2] = 0.5 * (np.roll(U[a], -1, axis=0) - np.roll(U[a], 1, axis=0))
    ss = np.zeros((nz, ny, nx))
    for a in range(3):
        for b in range(3):
            s = 0.5 * (g[a, b] + g[b, a])
            ss += s * s
    return (2.0 * nu * ss).reshape(-1)


def pipe_profiles(u, rho, solid, nx, ny, nz, cx, cy, R, nu, nbins):
    u = np.asarray(u, dtype=np.float64).reshape(3, -1)
    rho = np.asarray(rho, dtype=np.float64).reshape(-1)
    inside = np.asarray(solid).reshape(-1) == 0
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    dx = (x.reshape(-1) - cx).astype(np.float64)
    dy = (y.reshape(-1) - cy).astype(np.float64)
    r = np.sqrt(dx * dx + dy * dy)
    b = np.floor(r * nbins / R).astype(np.int64)
    keep = inside & (b < nbins)
    safe = np.where(r > 0, r, 1.0)
    ur = np.where(r > 0, (u[0] * dx + u[1] * dy) / safe, u[0])
    ut = np.where(r > 0, (u[1] * dx - u[0] * dy) / safe, u[1])
    uz = u[2]
    eps = cell_dissipation(u, nx, ny, nz, nu)
    qs = [np.ones_like(ur), ur, ut, uz, ur * ur, ut * ut, uz * uz, ur * uz, ur * ut, ut * uz, rho, eps]
    out = np.zeros((nbins, NQ))
    cnt = np.bincount(b[keep], minlength=nbins)[:nbins].astype(np.float64)
    for k, q in enumerate(qs):
        s = np.bincount(b[keep], weights=q[keep], minlength=nbins)[:nbins]
        out[:, k] = np.where(cnt > 0, s / np.where(cnt > 0, cnt, 1.0), 0.0)
    out[:, 0] = cnt
    return out
