"""D3Q27 on the GPU (lbm_grid.lattice = 27): the periodic box and the pipe
with its linear IBB wall, vs the D3Q27 oracle (oracle/d3q27.py), element by
element on seeded inputs.

Tolerances as for D3Q19: FP64 storage 1e-12 and FP32 1e-5, relative to the
field's largest magnitude.
"""
import numpy as np
import pytest

import workloads
from oracle import d3q27 as q27

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


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_random_populations_f64_step_by_step(lbm):
    nz, ny, nx = 6, 10, 37  # ragged rows
    N = nx * ny * nz
    rng = np.random.default_rng(7)
    f = q27.W.reshape(27, 1) * (1 + 0.1 * (rng.random((27, N)) - 0.5))
    F = (2e-4, -1e-4, 5e-5)
    g = lbm.Lattice(nx, ny, nz, 0.62, force=F, storage=lbm.F64, lattice=27)
    g.set_populations(f)
    assert rel(g.populations(), f) < 1e-15
    o = f.reshape(27, nz, ny, nx)
    for _ in range(3):
        g.step(1)
        o = q27.step(o, 0.62, F)
        assert rel(g.populations(), o.reshape(27, N)) < 1e-12
    rg, ug = g.macro()
    ro, uo = q27.macro(o, F)
    assert rel(rg, ro.reshape(-1)) < 1e-12
    assert rel(ug, uo.reshape(3, -1)) < 1e-12
    g.close()


def test_shear_wave_f32_100_steps(lbm):
    nz, ny, nx = 4, 6, 48
    k = 2 * np.pi / nx
    x = np.arange(nx)
    u = np.zeros((3, nz, ny, nx))
    u[0] = 0.03
    u[1] = 0.01 * np.sin(k * x)
    u[2] = 0.005 * np.cos(2 * k * x)
    F = (1e-6, 0, 0)
    g = lbm.Lattice(nx, ny, nz, 0.7, force=F, storage=lbm.F32, lattice=27)
    g.init_velocity(u)
    g.step(100)
    o = q27.step(q27.feq(np.ones((nz, ny, nx)), u), 0.7, F, n=100)
    rg, ug = g.macro()
    ro, uo = q27.macro(o, F)
    assert rel(ug, uo.reshape(3, -1)) < 1e-5
    # transverse waves leave rho - 1 at round-off size, below FP32's
    # resolution of 1: compare rho itself
    assert rel(rg, ro.reshape(-1)) < 1e-6
    g.close()


def _pipe_pair(lbm, nx, ny, nz, R, tau, F, storage, seed):
    u = workloads.pipe_velocity(nx, ny, nz, R, 0.02, perturbation=0.1, seed=seed)
    g = lbm.Lattice(nx, ny, nz, tau, force=F, storage=storage, lattice=27)
    g.init_velocity(u)
    g.set_pipe(R)
    solid = q27.pipe_solid(nx, ny, nz, R)
    links = q27.pipe_links(solid, R)
    o = q27.feq(np.ones((nz, ny, nx)), u)
    return g, o, solid, links


@pytest.mark.parametrize("R", [10.3, 6.4, 7.4])
def test_pipe_wall_f64_step_by_step(lbm, R):
    """The D3Q27 pipe with the linear interpolated bounce-back on its wall
    (and the halfway fallback, which the 6.4 radius in a 16 x 15 section
    reaches), a body force along z: every fluid cell's populations after
    each step against the oracle's pipe step. The 7.4 radius in a 16 x 15
    section puts fluid cells on the y faces, whose pulls wrap
    periodically; the other two keep the faces solid, where the sweep
    addresses pulls by per-direction plane pointers."""
    n = 24 if R > 8 else 16
    nz, F, tau = 5, (0.0, 0.0, 3e-6), 0.62
    g, o, solid, links = _pipe_pair(lbm, n, n - 1, nz, R, tau, F, lbm.F64, seed=3)
    fl = ~solid.reshape(-1)
    for _ in range(4):
        g.step(1, lbm.BC_IBB)
        o = q27.step_pipe(o, solid, links, tau, F)
        assert rel(g.populations()[:, fl], o.reshape(27, -1)[:, fl]) < 1e-12
    rg, ug = g.macro()
    ro, uo = q27.macro(o, F)
    assert rel(ug[:, fl], uo.reshape(3, -1)[:, fl]) < 1e-12
    g.close()


def test_pipe_wall_f32_200_steps(lbm):
    nx, ny, nz, R, tau, F = 26, 26, 8, 11.6, 0.6, (0.0, 0.0, 2e-6)
    g, o, solid, links = _pipe_pair(lbm, nx, ny, nz, R, tau, F, lbm.F32, seed=4)
    g.step(200, lbm.BC_IBB)
    for _ in range(200):
        o = q27.step_pipe(o, solid, links, tau, F)
    fl = ~solid.reshape(-1)
    rg, ug = g.macro()
    ro, uo = q27.macro(o, F)
    assert rel(ug[:, fl], uo.reshape(3, -1)[:, fl]) < 1e-5
    assert rel(rg[fl], ro.reshape(-1)[fl]) < 1e-6
    g.close()


def test_d3q27_refuses_what_it_does_not_build(lbm):
    g = lbm.Lattice(16, 16, 16, 0.6, storage=lbm.F32, lattice=27)
    g.init_velocity(workloads.noise_velocity((16, 16, 16), 0.01, seed=2))
    with pytest.raises(lbm.LbmError):
        g.step(1, lbm.BC_IBB)  # IBB without a pipe
    with pytest.raises(lbm.LbmError):
        g.add_spheres(np.array([[8.0, 8.0, 8.0]]), 3.0)
    with pytest.raises(lbm.LbmError):
        g.set_mrt_rates(1.2, 1.3, 1.1, 1.5, 1.9)
    g.step(2)
    s = g.stats()
    assert np.isfinite(s["kinetic_energy"]) and s["kinetic_energy"] > 0
    g.close()
    with pytest.raises(ValueError):
        lbm.Lattice(16, 16, 16, 0.6, storage=lbm.F16S, lattice=27)
