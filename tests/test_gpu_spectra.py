"""3D spectra on the GPU (hand-written FP32 FFT) against the numpy oracle
of oracle/spectra.py on the oracle's own velocity field, bin by bin.

Tolerance per shell: |gpu - oracle| <= 1e-5 max(oracle) + 1e-4 |oracle|,
from the FP32 transform (relative rounding ~1e-7 per stage, 3 log2 n
stages) against FP64 numpy."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import spectra

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_05448_gb300 import build, lbm as L
    build.build()
    L.load()
    return L


def close(g, o):
    tol = 1e-5 * np.max(np.abs(o)) + 1e-4 * np.abs(o)
    return bool(np.all(np.abs(g - o) <= tol)), float(np.max(np.abs(g - o) / (np.max(np.abs(o)))))


def test_periodic_hit_spectrum_matches_oracle(lbm):
    n, tau, nb = 32, 0.6, 30
    u = workloads.hit_velocity(n, seed=2, k_peak=4.0, u_rms=0.03)
    g = lbm.Lattice(n, n, n, tau, storage=lbm.F64)
    o = oracle.Sim(n, n, n, tau)
    for s in (g, o):
        s.init_velocity(u)
    g.step(20)
    o.step(20)
    Eg, Dg = g.spectrum(nb)
    Eo, Do = spectra.spectra(o.masked_velocity(), n, (tau - 0.5) / 3, nb)
    okE, eE = close(Eg, Eo)
    okD, eD = close(Dg, Do)
    assert okE and okD, (eE, eD)
    # the two sums: mean kinetic energy and the spectral dissipation
    assert Eg.sum() == pytest.approx(o.stats()["kinetic_energy"], rel=1e-5)


def test_masked_sphere_spectrum_matches_oracle(lbm):
    p = workloads.SPHERE_32
    n = p["n"]
    u = workloads.noise_velocity((n, n, n), 1e-3, seed=1)
    g = lbm.Lattice(n, n, n, p["tau"], force=p["force"], storage=lbm.F64, max_particles=1)
    o = oracle.Sim(n, n, n, p["tau"], force=p["force"])
    X = np.array([p["centre"]])
    for s in (g, o):
        s.init_velocity(u)
        s.add_spheres(X, p["radius"], U=np.array([[0.01, 0.0, 0.0]]), W=np.zeros((1, 3)), fixed=True)
    g.step(10, lbm.BC_IBB)
    o.step(10, oracle.BC_IBB)
    Eg, Dg = g.spectrum(28)
    Eo, Do = spectra.spectra(o.masked_velocity(), n, (p["tau"] - 0.5) / 3, 28)
    okE, eE = close(Eg, Eo)
    okD, eD = close(Dg, Do)
    assert okE and okD, (eE, eD)


@pytest.mark.parametrize("n,m", [(16, 3), (64, 7)])
def test_single_mode_lands_in_its_shell(lbm, n, m):
    A = 0.02
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    u = np.zeros((3, n, n, n))
    u[2] = A * np.sin(2 * np.pi * m * x / n)
    g = lbm.Lattice(n, n, n, 0.6, storage=lbm.F32)
    g.init_velocity(u)
    E, D = g.spectrum(n)
    assert E[m] == pytest.approx(A * A / 4, rel=1e-5)
    assert np.sum(np.delete(E, m)) < 1e-9 * E[m]
    nu = 0.1 / 3
    assert D[m] == pytest.approx(2 * nu * (2 * np.pi * m / n) ** 2 * A * A / 4, rel=1e-5)
    g.close()


def test_non_cube_is_rejected(lbm):
    g = lbm.Lattice(32, 32, 16, 0.6, storage=lbm.F32)
    g.init_velocity(np.zeros((3, 16, 32, 32)))
    with pytest.raises(lbm.LbmError):
        g.spectrum(8)
    g.close()
