"""Pins of the TKE-budget oracle (oracle/tke_budget.py, Eq. 1a-c) against
closed forms and identities that do not go through its own routines:

- a harmonic streamwise field u_z = A dx + B dy + C dx dy: central
  differences are exact for it, the binned means of its cylindrical
  gradients vanish by symmetry, so E_Dz is minus the bin mean of the
  Cartesian dissipation 2 nu s_ij s_ij (computed by the profile oracle's
  own stencil); for a harmonic field the viscous diffusion of its energy
  balances its dissipation (E_Vz + E_Dz -> 0, up to the binning);
- z waves u_z = A cos kz, u_r = D (cos 2kz + cos 4kz), rho = 1 + d sin kz:
  the discrete z derivative of cos kz is -sin k sin kz exactly, which gives
  E_Tz = -A^2 D / (8 r), E_Tr = -3 D^3 / (8 r), E_Pz = -c_s^2 d A sin(k) / 2 and
  E_Dz = -nu A^2 sin^2 k, while the terms whose factors are orthogonal in
  z vanish (E_Dtheta, zero in the continuum, decays as the grid's
  O(r^-3) error of the radial field's curvature terms);
- a laminar profile plus a wave, u_z = U0 (1 - r^2/R^2) + A cos kz,
  u_r = A cos kz: E_Oz = A^2 U0 r / R^2;
- a z-modulated breathing and swirling field u = D r cos(2kz) e_r +
  Q r cos(kz) e_theta (linear in x and y, so the central differences are
  exact): E_Dr = -nu D^2 (1 + sin^2(2k) <r^2> / 2) and
  E_Dtheta = -nu Q^2 sin^2(k) <r^2> / 2 with <r^2> the bin's mean of r^2;
  the curvature terms of the theta derivatives cancel u_r / r and
  u_theta / r exactly (E_Ptheta = 0 with p' ~ cos 2kz), the pressure
  diffusion and pressure-strain parts of E_Pr cancel up to the binning,
  E_Vr -> 2 nu D^2, and E_Ttheta is the radial derivative of
  Q^2 D <r^3> / 8 (-> -Q^2 D r^2 / 2);
- a z-modulated differential swirl u_theta = W r^2 cos kz (u_r = u_z = 0):
  (1/r) du_r/dtheta = 0 while the strain s_rtheta = W r cos(kz) / 2 is not,
  so E_Dr vanishes up to the grid's error, and
  E_Dtheta = -2 nu (W^2 <r^2> / 2 + W^2 sin^2(k) <r^4> / 4);
- a rigid rotation: no strain and no fluctuation, every term vanishes.
"""
import numpy as np
import pytest

from oracle import profiles, tke_budget as tb

COL = {n: i for i, n in enumerate(tb.NAMES)}


def pipe_grid(n, nz, R):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(n), np.arange(n), indexing="ij")
    c = (n - 1) / 2
    dx, dy = x.reshape(-1) - c, y.reshape(-1) - c
    solid = (dx * dx + dy * dy >= R * R).astype(np.uint8)
    return dx, dy, z.reshape(-1).astype(np.float64), c, solid


def test_harmonic_streamwise_field_dissipation_and_diffusion():
    n, nz, R, nu, nb = 44, 2, 20.0, 0.02, 10
    A, B, C = 3e-3, -2e-3, 4e-5
    dx, dy, _, c, solid = pipe_grid(n, nz, R)
    u = np.zeros((3, dx.size))
    u[2] = A * dx + B * dy + C * dx * dy
    out = tb.tke_budget(u, np.ones(dx.size), solid, n, n, nz, c, c, R, nu, nb)
    # independent: the Cartesian dissipation per cell, averaged over each bin
    eps = profiles.cell_dissipation(u, n, n, nz, nu)
    r = np.sqrt(dx * dx + dy * dy)
    b = np.floor(r * nb / R).astype(int)
    scale = nu * (A * A + B * B)
    for k in range(nb):
        cells = (solid == 0) & (b == k) & (r > 0)
        assert out[k, 0] == cells.sum()
        assert out[k, COL["E_Dz"]] == pytest.approx(-eps[cells].mean(), rel=1e-9)
    for name in ("E_Oz", "E_Tz", "E_Pz", "E_Tr", "E_Pr", "E_Vr", "E_Dr", "E_Ttheta", "E_Ptheta", "E_Vtheta", "E_Dtheta"):
        assert np.max(np.abs(out[:, COL[name]])) < 1e-12 * scale, name
    # viscous diffusion balances dissipation for a harmonic field, away from
    # the first and last bins (one-sided radial derivatives there)
    bal = out[2:-2, COL["E_Vz"]] + out[2:-2, COL["E_Dz"]]
    assert np.max(np.abs(bal)) < 0.05 * np.max(np.abs(out[2:-2, COL["E_Dz"]]))
    assert np.all(out[:, COL["E_Dz"]] < 0) and np.all(out[2:-2, COL["E_Vz"]] > 0)


def test_z_waves_closed_forms():
    n, nz, R, nu, nb = 36, 16, 16.0, 0.01, 8
    A, D, d = 2e-3, 3e-3, 1e-3
    k = 2 * np.pi / nz
    dx, dy, z, c, solid = pipe_grid(n, nz, R)
    r = np.sqrt(dx * dx + dy * dy)
    safe = np.where(r > 0, r, 1.0)
    ur = D * (np.cos(2 * k * z) + np.cos(4 * k * z))
    u = np.zeros((3, dx.size))
    u[0] = ur * dx / safe
    u[1] = ur * dy / safe
    u[2] = A * np.cos(k * z)
    rho = 1.0 + d * np.sin(k * z)
    out = tb.tke_budget(u, rho, solid, n, n, nz, c, c, R, nu, nb)
    rb = (np.arange(nb) + 0.5) * R / nb
    # <cos^2 kz (cos 2kz + cos 4kz)> = 1/4, <(cos 2kz + cos 4kz)^3> = 3/4
    assert out[:, COL["E_Tz"]] == pytest.approx(-A * A * D / (8 * rb), rel=1e-9)
    assert out[:, COL["E_Tr"]] == pytest.approx(-3 * D ** 3 / (8 * rb), rel=1e-9)
    assert out[:, COL["E_Pz"]] == pytest.approx(np.full(nb, -d * A * np.sin(k) / 6), rel=1e-9)
    assert out[:, COL["E_Dz"]] == pytest.approx(np.full(nb, -nu * A * A * np.sin(k) ** 2), rel=1e-9)
    tiny = 1e-12 * A * D
    for name in ("E_Oz", "E_Pr", "E_Ttheta", "E_Ptheta", "E_Vtheta"):
        assert np.max(np.abs(out[:, COL[name]])) < tiny, name
    # E_Dtheta is zero in the continuum; on the grid the central differences
    # of u_r e_r miss u_r / r by O(r^-3), so it falls off steeply with r
    edt = np.abs(out[:, COL["E_Dtheta"]])
    assert np.all(np.diff(edt) < 0) and edt[-1] < 1e-4 * edt[0]


def test_production_of_a_laminar_profile_with_a_wave():
    n, nz, R, nu, nb = 48, 8, 22.0, 0.01, 11
    U0, A = 0.05, 1e-3
    k = 2 * np.pi / nz
    dx, dy, z, c, solid = pipe_grid(n, nz, R)
    r = np.sqrt(dx * dx + dy * dy)
    safe = np.where(r > 0, r, 1.0)
    w = A * np.cos(k * z)
    u = np.zeros((3, dx.size))
    u[0] = w * dx / safe
    u[1] = w * dy / safe
    u[2] = U0 * (1 - r * r / R ** 2) + w
    out = tb.tke_budget(u, np.ones(dx.size), solid, n, n, nz, c, c, R, nu, nb)
    rb = (np.arange(nb) + 0.5) * R / nb
    # dU/dr = -2 U0 r / R^2 and <u_z' u_r'> = A^2 / 2 (interior bins: the
    # binned mean of r^2 differs from r_b^2 by a near-constant offset)
    expect = A * A * U0 * rb / R ** 2
    assert out[1:-1, COL["E_Oz"]] == pytest.approx(expect[1:-1], rel=0.03)


def test_rigid_rotation_has_no_budget():
    n, nz, R, nu, nb = 40, 3, 18.0, 0.02, 9
    W = 2e-3
    dx, dy, _, c, solid = pipe_grid(n, nz, R)
    u = np.zeros((3, dx.size))
    u[0], u[1] = -W * dy, W * dx
    out = tb.tke_budget(u, np.ones(dx.size), solid, n, n, nz, c, c, R, nu, nb)
    assert np.max(np.abs(out[:, 1:])) < 1e-15 * max(nu, 1.0) * W * W * R
    assert out[:, 0].sum() == np.count_nonzero((solid == 0) & (np.floor(np.sqrt(dx * dx + dy * dy) * nb / R) < nb))


def test_breathing_and_swirling_field():
    n, nz, R, nu, nb = 48, 16, 22.0, 0.02, 11
    D, Q, d = 1e-4, 2e-4, 1e-3
    k = 2 * np.pi / nz
    dx, dy, z, c, solid = pipe_grid(n, nz, R)
    c1, c2 = np.cos(k * z), np.cos(2 * k * z)
    u = np.zeros((3, dx.size))
    u[0] = D * c2 * dx - Q * c1 * dy
    u[1] = D * c2 * dy + Q * c1 * dx
    rho = 1.0 + d * c2
    out = tb.tke_budget(u, rho, solid, n, n, nz, c, c, R, nu, nb)
    r = np.sqrt(dx * dx + dy * dy)
    b = np.floor(r * nb / R).astype(int)
    cells = [(solid == 0) & (b == j) & (r > 0) for j in range(nb)]
    r2 = np.array([np.mean(r[m] ** 2) for m in cells])
    assert out[:, COL["E_Dr"]] == pytest.approx(-nu * D * D * (1 + 0.5 * np.sin(2 * k) ** 2 * r2), rel=1e-9)
    assert out[:, COL["E_Dtheta"]] == pytest.approx(-0.5 * nu * Q * Q * np.sin(k) ** 2 * r2, rel=1e-9)
    scale = d * D / 3
    assert np.max(np.abs(out[:, COL["E_Ptheta"]])) < 1e-12 * scale
    # each part is c_s^2 d D / 2 in size; they cancel up to the binning
    # noise of d<r>/dr (a sign error in either would leave twice that)
    assert np.max(np.abs(out[1:-1, COL["E_Pr"]])) < 0.1 * scale / 2
    rb = (np.arange(nb) + 0.5) * R / nb
    assert out[1:-1, COL["E_Vr"]] == pytest.approx(np.full(nb - 2, 2 * nu * D * D), rel=0.03)
    # <u_theta'^2 u_r'> = Q^2 D <r^3> / 4 from the cells' radii alone; the
    # bin-centre derivative of r F is the one E_Tz and E_Tr pin exactly
    r3 = np.array([np.mean(r[m] ** 3) for m in cells])
    F = 0.5 * Q * Q * D * r3 / 4
    assert out[:, COL["E_Ttheta"]] == pytest.approx(-np.gradient(rb * F, R / nb) / rb, rel=1e-9)
    assert out[2:-1, COL["E_Ttheta"]] == pytest.approx(-0.5 * Q * Q * D * rb[2:-1] ** 2, rel=0.25)
    for name in ("E_Oz", "E_Tz", "E_Pz", "E_Vz", "E_Dz", "E_Tr", "E_Vtheta"):
        assert np.max(np.abs(out[:, COL[name]])) < 1e-12 * nu * D * D, name


def test_differential_swirl():
    n, nz, R, nu, nb = 56, 8, 26.0, 0.02, 13
    W = 1e-5
    k = 2 * np.pi / nz
    dx, dy, z, c, solid = pipe_grid(n, nz, R)
    r = np.sqrt(dx * dx + dy * dy)
    ck = np.cos(k * z)
    u = np.zeros((3, dx.size))
    u[0] = -W * ck * r * dy
    u[1] = W * ck * r * dx
    out = tb.tke_budget(u, np.ones(dx.size), solid, n, n, nz, c, c, R, nu, nb)
    b = np.floor(r * nb / R).astype(int)
    cells = [(solid == 0) & (b == j) & (r > 0) for j in range(nb)]
    r2 = np.array([np.mean(r[m] ** 2) for m in cells])
    r4 = np.array([np.mean(r[m] ** 4) for m in cells])
    rb = (np.arange(nb) + 0.5) * R / nb
    far = rb > 4  # the central differences of r dy, r dx are exact only far from the axis
    # a wrong sign of the u_theta / r term in (1/r) du_r/dtheta would make
    # E_Dr = nu W^2 <r^2>
    assert np.all(np.abs(out[far, COL["E_Dr"]]) < 0.05 * nu * W * W * r2[far])
    expect = -2 * nu * (W * W * r2 / 2 + W * W * np.sin(k) ** 2 * r4 / 4)
    assert out[far, COL["E_Dtheta"]] == pytest.approx(expect[far], rel=0.05)
