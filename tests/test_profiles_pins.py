"""Pins of the pipe-profile oracle (oracle/profiles.py): Poiseuille flow
(central differences are exact for a quadratic field, so the binned
dissipation is the closed form 4 nu U0^2 r^2 / R^4 averaged over the bin's
cells), a solid-body rotation (pure u_theta, no dissipation), and the cell
counts of the bins against the areas of the annuli."""
import numpy as np
import pytest

from oracle import profiles


def grid(n, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(n), np.arange(n), indexing="ij")
    c = (n - 1) / 2
    return x.reshape(-1) - c, y.reshape(-1) - c, c


def test_poiseuille_profile_and_dissipation():
    n, nz, R, U0, nu, nb = 40, 4, 17.0, 0.05, 0.01, 8
    dx, dy, c = grid(n, nz)
    r2 = dx * dx + dy * dy
    solid = (r2 >= R * R).astype(np.uint8)
    u = np.zeros((3, dx.size))
    # quadratic everywhere (also where the stencil of a wall cell reaches)
    u[2] = U0 * (1 - r2 / R ** 2)
    out = profiles.pipe_profiles(u, np.ones(dx.size), solid, n, n, nz, c, c, R, nu, nb)
    r = np.sqrt(r2)
    b = np.floor(r * nb / R).astype(int)
    for k in range(nb):
        cells = (solid == 0) & (b == k)
        assert out[k, 0] == cells.sum()
        assert out[k, 3] == pytest.approx(np.mean(U0 * (1 - r2[cells] / R ** 2)), rel=1e-12)
        assert abs(out[k, 1]) < 1e-15 and abs(out[k, 2]) < 1e-15
        assert out[k, 11] == pytest.approx(np.mean(4 * nu * U0 ** 2 * r2[cells] / R ** 4), rel=1e-10)
        assert out[k, 10] == pytest.approx(1.0)


def test_solid_body_rotation():
    n, nz, R, W, nb = 32, 2, 14.0, 1e-3, 7
    dx, dy, c = grid(n, nz)
    solid = (dx * dx + dy * dy >= R * R).astype(np.uint8)
    u = np.zeros((3, dx.size))
    u[0], u[1] = -W * dy, W * dx
    out = profiles.pipe_profiles(u, np.ones(dx.size), solid, n, n, nz, c, c, R, 0.02, nb)
    r = np.sqrt(dx * dx + dy * dy)
    b = np.floor(r * nb / R).astype(int)
    for k in range(nb):
        cells = (solid == 0) & (b == k)
        assert out[k, 2] == pytest.approx(W * np.mean(r[cells]), rel=1e-12)
        assert abs(out[k, 1]) < 1e-17
        assert out[k, 11] < 1e-25  # a rigid rotation has no strain


def test_bin_counts_follow_annulus_areas():
    n, nz, R, nb = 200, 1, 90.0, 9
    dx, dy, c = grid(n, nz)
    solid = (dx * dx + dy * dy >= R * R).astype(np.uint8)
    out = profiles.pipe_profiles(np.zeros((3, dx.size)), np.ones(dx.size), solid, n, n, nz, c, c, R, 0.01, nb)
    edges = np.arange(nb + 1) * R / nb
    area = np.pi * (edges[1:] ** 2 - edges[:-1] ** 2)
    assert np.allclose(out[:, 0], area, rtol=0.02)
    assert out[:, 0].sum() == (solid == 0).sum()
