"""Pins of the spectra oracle (oracle/spectra.py) against what the
mathematics fixes: Parseval, a single Fourier mode, the dissipation of a
single mode against its exact gradient, shell bookkeeping, and the
masked-velocity export of the C oracle."""
import numpy as np
import pytest

import oracle
from oracle import spectra


def test_parseval_random_field():
    n = 16
    rng = np.random.default_rng(0)
    u = rng.standard_normal((3, n ** 3))
    E, D = spectra.spectra(u, n, 0.01, 3 * n)
    assert E.sum() == pytest.approx(0.5 * np.mean(np.sum(u * u, axis=0)), rel=1e-12)


@pytest.mark.parametrize("m", [1, 3, 5])
def test_single_mode_energy_and_dissipation(m):
    """u_x = A sin(2 pi m y / n): all energy A^2/4 in shell m, dissipation
    nu <|grad u|^2> = nu A^2 (2 pi m / n)^2 / 2."""
    n, A, nu = 32, 0.03, 0.02
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    u = np.zeros((3, n, n, n))
    u[0] = A * np.sin(2 * np.pi * m * y / n)
    E, D = spectra.spectra(u, n, nu, n)
    assert E[m] == pytest.approx(A * A / 4, rel=1e-12)
    assert np.sum(np.delete(E, m)) < 1e-25
    kap = 2 * np.pi * m / n
    assert D[m] == pytest.approx(nu * A * A * kap * kap / 2, rel=1e-12)


def test_dissipation_equals_mean_squared_gradient():
    """Sum of D equals nu <|grad u|^2> with the exact (spectral) gradient of
    a band-limited field built from a few modes."""
    n, nu = 16, 0.015
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    modes = [(1, 2, 0, 0.02), (3, 0, 1, 0.01), (0, 2, 2, 0.015)]
    u = np.zeros((3, n, n, n))
    grad2 = 0.0
    for d, (a, b, c, A) in enumerate(modes):
        ph = 2 * np.pi * (a * x + b * y + c * z) / n
        u[d] += A * np.cos(ph)
        grad2 += A * A / 2 * (2 * np.pi / n) ** 2 * (a * a + b * b + c * c)
    E, D = spectra.spectra(u, n, nu, 2 * n)
    assert D.sum() == pytest.approx(nu * grad2, rel=1e-12)


def test_shells_match_brute_force_count():
    """Shell populations against a direct enumeration of the wave vectors
    (shell 1 holds the 6 axis vectors and the 12 with |k| = sqrt 2)."""
    n = 8
    shell, kappa2 = spectra.shells(n)
    ks = [k if k <= n // 2 - 1 else k - n for k in range(n)]  # numpy fftfreq order
    count = {}
    for a in ks:
        for b in ks:
            for c in ks:
                K = int(np.floor(np.sqrt(a * a + b * b + c * c) + 0.5))
                count[K] = count.get(K, 0) + 1
    for K, m in count.items():
        assert np.count_nonzero(shell == K) == m
    assert count[1] == 18 and count[0] == 1
    assert np.isclose(kappa2.max(), (2 * np.pi / n) ** 2 * 3 * (n // 2) ** 2)


def test_masked_velocity_replaces_solid_cells(orc):
    n = 16
    sim = orc.Sim(n, n, n, 0.6)
    u0 = np.full((3, n, n, n), 0.01)
    sim.init_velocity(u0)
    X = np.array([[7.5, 7.5, 7.5]])
    sim.add_spheres(X, 3.0, U=np.array([[0.02, 0.0, 0.0]]), W=np.zeros((1, 3)), fixed=True)
    sim.step(1, oracle.BC_IBB)
    u = sim.masked_velocity()
    solid = sim.solid()[0] == 1
    assert solid.any()
    assert np.allclose(u[0, solid], 0.02) and np.allclose(u[1:, solid], 0.0)
    rho, um = sim.macro()
    assert np.array_equal(u[:, ~solid], um[:, ~solid])
