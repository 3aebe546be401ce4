"""The benchmark configuration itself: the 148x148x438 pipe with the IBB
wall in FP32, swept exactly as bench.py times it (fluid-run work items,
persistent grid, compact ghost values). The oracle runs the same 4 steps
in FP64 at full size; every fluid cell's velocity and density are compared
(FP32 bar 1e-5 of the field maximum), and the wall links bit-exactly; the
16-bit storages against the same oracle run, at their own bars."""
import numpy as np
import pytest

import oracle
import workloads

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


def _setup():
    p = workloads.PIPE_148
    nx, ny, nz, R = p["nx"], p["ny"], p["nz"], p["radius"]
    pp = workloads.pipe_parameters(R, p["nu"], p["re_tau"])
    force = (0.0, 0.0, pp["g"])
    u = workloads.pipe_velocity(nx, ny, nz, R, pp["u_bulk"], p["perturbation"], seed=0)
    return nx, ny, nz, R, pp["tau"], force, u


@pytest.fixture(scope="module")
def reference():
    """The oracle's links before the first step and its fields after 4 steps."""
    nx, ny, nz, R, tau, force, u = _setup()
    o = oracle.Sim(nx, ny, nz, tau, force=force)
    o.init_velocity(u)
    o.set_pipe(R)
    links = o.links()
    o.step(4, oracle.BC_IBB)
    fluid = o.solid()[0] == 0
    ro, uo = o.macro()
    return links, fluid, ro, uo


def test_benchmark_pipe_full_size(lbm, reference):
    nx, ny, nz, R, tau, force, u = _setup()
    lo, fluid, ro, uo = reference
    g = lbm.Lattice(nx, ny, nz, tau, force=force, storage=lbm.F32)
    g.init_velocity(u)
    g.set_pipe(R)
    la = g.links()
    assert len(la["cell"]) == len(lo["cell"]) == 1130040
    ka, ko = np.lexsort((la["dir"], la["cell"])), np.lexsort((lo["dir"], lo["cell"]))
    for key in ("cell", "dir", "scheme"):
        assert np.array_equal(np.asarray(la[key])[ka], np.asarray(lo[key])[ko]), key
    assert np.array_equal(np.asarray(la["q"])[ka].view(np.int64), np.asarray(lo["q"])[ko].view(np.int64))
    g.step(4, lbm.BC_IBB)
    rg, ug = g.macro()
    assert rel(ug[:, fluid], uo[:, fluid]) < 1e-5
    assert rel(rg[fluid], ro[fluid]) < 1e-5
    assert np.max(np.abs(rg[fluid] - ro[fluid])) < 1e-6
    g.close()


@pytest.mark.parametrize("storage,tol", [("f16s", 2e-3), ("bf16s", 3e-2)])
def test_benchmark_pipe_full_size_16bit(lbm, reference, storage, tol):
    """The benchmark pipe on 16-bit storage, swept as the bench's 16-bit
    lines time it (two cells per lane, the wall in the sweep): velocity
    within the 16-bit bars of the smaller parity tests, relative to the
    field maximum, after the same 4 steps."""
    nx, ny, nz, R, tau, force, u = _setup()
    _, fluid, ro, uo = reference
    g = lbm.Lattice(nx, ny, nz, tau, force=force, storage=lbm.STORAGE[storage])
    g.init_velocity(u)
    g.set_pipe(R)
    g.step(4, lbm.BC_IBB)
    rg, ug = g.macro()
    assert np.all(np.isfinite(ug[:, fluid]))
    assert rel(ug[:, fluid], uo[:, fluid]) < tol
    g.close()


@pytest.mark.parametrize("bc,steps", [("ibb", 3), ("ibm_b", 2)])
def test_particle_laden_box_full_size(lbm, bc, steps):
    """The particle-laden benchmark box itself: 256^3 HIT (seeded Fourier
    modes, u_rms 0.03), 2000 moving spheres of radius 4 at density ratio 5,
    d'Humieres rates, tau 0.51, FP32 storage, set up as bench.py does. IBB:
    the wall links at set-up (lists exact, q of the FP32 path within 1e-6).
    After a few steps every fluid cell's velocity and density and every
    particle's motion against the FP64 oracle at the FP32 bar."""
    n, npart = 256, 2000
    u = workloads.hit_velocity(n, seed=0, k_peak=8.0, u_rms=0.03, dtype=np.float64)
    X = workloads.place_spheres((n, n, n), npart, 4.0, 1.0, seed=0)
    g = lbm.Lattice(n, n, n, 0.51, storage=lbm.F32, rates=lbm.RATES_DHUMIERES, max_particles=npart)
    o = oracle.Sim(n, n, n, 0.51, rates=oracle.RATES_DHUMIERES)
    for s in (g, o):
        s.init_velocity(u)
        s.add_spheres(X, 4.0, density_ratio=5.0)
    if bc == "ibb":
        la, lo = g.links(), o.links()
        ka, ko = np.lexsort((la["dir"], la["cell"])), np.lexsort((lo["dir"], lo["cell"]))
        for key in ("cell", "dir", "scheme", "pid"):
            assert np.array_equal(np.asarray(la[key])[ka], np.asarray(lo[key])[ko]), key
        assert np.max(np.abs(np.asarray(la["q"])[ka] - np.asarray(lo["q"])[ko])) < 1e-6
    g.step(steps, lbm.BC_IBB if bc == "ibb" else lbm.BC_IBM_B)
    o.step(steps, oracle.BC_IBB if bc == "ibb" else oracle.BC_IBM_B)
    fluid = (o.solid()[0] == 0) & ((g.flags() & 1) == 0) if bc == "ibb" else np.ones(n ** 3, dtype=bool)
    rg, ug = g.macro()
    ro, uo = o.macro()
    assert rel(ug[:, fluid], uo[:, fluid]) < 1e-5
    assert rel(rg[fluid], ro[fluid]) < 1e-5
    Pg, Po = g.particles(), o.particles()
    for k in ("U", "W"):
        assert rel(Pg[k], Po[k]) < 1e-5, k
    assert np.max(np.abs(Pg["X"] - Po["X"])) < 1e-6
    g.close()
