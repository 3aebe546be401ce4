"""Oracle of the pipe's component-wise TKE budget (test infrastructure).

TEST INFRASTRUCTURE ONLY: a plain numpy statement of the budget terms of
Eq. 1a-c (Sec. 2.2): production E_O, turbulent transport E_T, pressure work
E_P, viscous diffusion E_V and viscous dissipation E_D of the streamwise (z),
radial (r) and azimuthal (theta) velocity fluctuations. The terms are taken
as printed. Readings, for the cells inside the pipe (not solid) with r > 0:

- Geometry: axis along z through (c_x, c_y); r = sqrt(dx^2 + dy^2),
  e_r = (dx, dy, 0) / r, e_theta = (-dy, dx, 0) / r, e_z; radial bin
  b = floor(r nbins / R) as for the radial profiles; the cells on the
  axis (r = 0) have no basis and are left out.
- Averages <.> are means over the cells of a bin (over theta and z at the
  bin's radius), and a fluctuation is the departure from its bin's mean:
  q' = q - <q>_b, taken cell by cell.
- Velocity gradients are second-order central differences of the Cartesian
  components (periodic wrap), G_ab = d u_a / d x_b. Their components in the
  local basis are T_ij = e_i . G . e_j; the strain is
  s_ij = (T_ij + T_ji) / 2 (the cylindrical components of the strain
  tensor). The derivatives of the component functions in Eq. 1 are
  du_i/dr = T_ir, du_i/dz = T_iz, (1/r) du_z/dtheta = T_ztheta,
  (1/r) du_r/dtheta = T_rtheta + u_theta / r,
  (1/r) du_theta/dtheta = T_thetatheta - u_r / r.
- Pressure fluctuation p' = c_s^2 rho' with c_s^2 = 1/3; the density in
  front of the pressure terms is the lattice reference density 1.
- d/dr of a binned profile F_b: central differences over the bin centres
  r_b = (b + 1/2) R / nbins, one-sided at the first and last bins
  (numpy.gradient); (1/r) d/dr (r F) uses the same derivative of r_b F_b.

Returned per bin (shape (nbins, NT)): the cell count, then
E_Oz, E_Tz, E_Pz, E_Vz, E_Dz, E_Tr, E_Pr, E_Vr, E_Dr,
E_Ttheta, E_Ptheta, E_Vtheta, E_Dtheta (NT = 14). Empty bins hold zeros and
their neighbours' radial derivatives treat them as zeros.
"""
from __future__ import annotations

import numpy as np

CS2 = 1.0 / 3.0
NAMES = ["count", "E_Oz", "E_Tz", "E_Pz", "E_Vz", "E_Dz", "E_Tr", "E_Pr", "E_Vr", "E_Dr",
         "E_Ttheta", "E_Ptheta", "E_Vtheta", "E_Dtheta"]
NT = len(NAMES)


def cartesian_gradient(u, nx, ny, nz):
    """G[a, b] = d u_a / d x_b per cell by central differences, shape (3, 3, N)."""
    U = np.asarray(u, dtype=np.float64).reshape(3, nz, ny, nx)
    G = np.empty((3, 3, nz, ny, nx))
    for a in range(3):
        G[a, 0] = 0.5 * (np.roll(U[a], -1, axis=2) - np.roll(U[a], 1, axis=2))
        G[a, 1] = 0.5 * (np.roll(U[a], -1, axis=1) - np.roll(U[a], 1, axis=1))
        G[a, 2] = 0.5 * (np.roll(U[a], -1, axis=0) - np.roll(U[a], 1, axis=0))
    return G.reshape(3, 3, -1)


def tke_budget(u, rho, solid, nx, ny, nz, cx, cy, R, nu, nbins):
    u = np.asarray(u, dtype=np.float64).reshape(3, -1)
    rho = np.asarray(rho, dtype=np.float64).reshape(-1)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    dx = (x.reshape(-1) - cx).astype(np.float64)
    dy = (y.reshape(-1) - cy).astype(np.float64)
    r = np.sqrt(dx * dx + dy * dy)
    b = np.floor(r * nbins / R).astype(np.int64)
    keep = (np.asarray(solid).reshape(-1) == 0) & (r > 0) & (b < nbins)

    G = cartesian_gradient(u, nx, ny, nz)[:, :, keep]
    u, rho, dx, dy, r, b = u[:, keep], rho[keep], dx[keep], dy[keep], r[keep], b[keep]
    zero = np.zeros_like(r)
    e = {"r": np.stack([dx / r, dy / r, zero]),
         "t": np.stack([-dy / r, dx / r, zero]),
         "z": np.stack([zero, zero, zero + 1.0])}
    vel = {i: np.einsum("an,an->n", e[i], u) for i in "rtz"}  # u_r, u_theta, u_z
    T = {(i, j): np.einsum("an,abn,bn->n", e[i], G, e[j]) for i in "rtz" for j in "rtz"}
    s = {(i, j): 0.5 * (T[(i, j)] + T[(j, i)]) for i in "rtz" for j in "rtz"}
    # derivatives of the component functions (Eq. 1): d/dr, (1/r) d/dtheta, d/dz
    dr = {i: T[(i, "r")] for i in "rtz"}
    dz = {i: T[(i, "z")] for i in "rtz"}
    dth = {"z": T[("z", "t")], "r": T[("r", "t")] + vel["t"] / r, "t": T[("t", "t")] - vel["r"] / r}
    p = CS2 * rho

    cnt = np.bincount(b, minlength=nbins)[:nbins].astype(np.float64)
    has = cnt > 0

    def mean(q):
        sm = np.bincount(b, weights=q, minlength=nbins)[:nbins]
        return np.where(has, sm / np.where(has, cnt, 1.0), 0.0)

    def fluct(q):
        return q - mean(q)[b]

    def avg(*qs):  # bin mean of a product of fluctuations
        prod = np.ones_like(r)
        for q in qs:
            prod = prod * fluct(q)
        return mean(prod)

    rb = (np.arange(nbins) + 0.5) * R / nbins
    h = R / nbins

    def ddr(F):
        return np.gradient(F, h) if nbins > 1 else np.zeros_like(F)

    def div_r(F):  # (1/r) d/dr (r F)
        return ddr(rb * F) / rb

    uz, ur, ut = vel["z"], vel["r"], vel["t"]
    out = np.zeros((nbins, NT))
    out[:, 0] = cnt
    # streamwise component (Eq. 1a)
    out[:, 1] = -avg(uz, ur) * ddr(mean(uz))
    out[:, 2] = -div_r(0.5 * avg(uz, uz, ur))
    out[:, 3] = avg(p, dz["z"])
    out[:, 4] = 2.0 * nu * div_r(avg(uz, s[("z", "r")]))
    out[:, 5] = -2.0 * nu * (avg(s[("z", "r")], dr["z"]) + avg(s[("z", "t")], dth["z"]) + avg(s[("z", "z")], dz["z"]))
    # radial component (Eq. 1b)
    out[:, 6] = -div_r(0.5 * avg(ur, ur, ur))
    out[:, 7] = -ddr(avg(ur, p)) + avg(p, dr["r"])
    out[:, 8] = 2.0 * nu * div_r(avg(ur, s[("r", "r")]))
    out[:, 9] = -2.0 * nu * (avg(s[("r", "r")], dr["r"]) + avg(s[("r", "t")], dth["r"]) + avg(s[("r", "z")], dz["r"]))
    # azimuthal component (Eq. 1c)
    out[:, 10] = -div_r(0.5 * avg(ut, ut, ur))
    out[:, 11] = avg(p, dth["t"])
    out[:, 12] = 2.0 * nu * div_r(avg(ut, s[("t", "r")]))
    out[:, 13] = -2.0 * nu * (avg(s[("t", "t")], dth["t"]) + avg(s[("t", "r")], dr["t"]) + avg(s[("t", "z")], dz["t"]))
    out[~has, 1:] = 0.0
    return out
