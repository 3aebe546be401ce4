"""GPU path vs the oracle, element by element, on seeded inputs.

Tolerances: FP64 storage 1e-12 relative to the field maximum; FP32 1e-5
(max |gpu - oracle| / max |oracle| per field over the horizon); link lists
bit-exact (cell, direction, scheme, owner, and the FP64 bits of q).
"""
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


def pair(lbm, shape, tau, force=(0, 0, 0), storage=None, rates=oracle.RATES_SRT, max_particles=0):
    nz, ny, nx = shape
    g = lbm.Lattice(nx, ny, nz, tau, force=force, storage=lbm.F64 if storage is None else storage,
                    rates=rates, max_particles=max_particles)
    o = oracle.Sim(nx, ny, nz, tau, force=force, rates=rates)
    return g, o


@pytest.mark.parametrize("rates", [oracle.RATES_SRT, oracle.RATES_DHUMIERES])
def test_periodic_random_populations_f64(lbm, rates):
    shape = (7, 18, 37)  # ragged: x not a multiple of the warp
    # departures of +-10 % around 1/19 keep |u| below the watchdog limit
    f = workloads.random_populations(int(np.prod(shape)), seed=3, lo=0.05, hi=0.061)
    g, o = pair(lbm, shape, 0.57, force=(2e-4, -1e-4, 3e-5), rates=rates)
    g.set_populations(f)
    o.set_populations(f)
    assert rel(g.populations(), f) < 1e-15
    for k in range(3):
        g.step(1)
        o.step(1)
        assert rel(g.populations(), o.populations()) < 1e-12
    rg, ug = g.macro()
    ro, uo = o.macro()
    assert rel(rg, ro) < 1e-12 and rel(ug, uo) < 1e-12


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_custom_mrt_rates(lbm, storage, tol):
    """Non-shear MRT rates set on a running context (the bulk-viscosity knob,
    lbm_set_mrt_rates): an SRT context switches to the MRT collision with
    the new energy, energy-square, flux, pi and m rates. Random departures
    plus a standing density wave on ragged rows, with a body force."""
    shape = (6, 10, 37)
    nz, ny, nx = shape
    N = nz * ny * nx
    f = workloads.random_populations(N, seed=5, lo=0.052, hi=0.0575)
    wave = 1.0 + 1e-3 * np.cos(2 * np.pi * np.arange(nx) / nx)
    f = f * np.broadcast_to(wave, shape).reshape(1, N)
    g, o = pair(lbm, shape, 0.7, force=(1e-5, -2e-6, 0),
                storage=lbm.F64 if storage == "f64" else lbm.F32)
    g.set_populations(f)
    o.set_populations(f)
    g.step(5)
    o.step(5)
    rates = (0.5, 1.3, 1.1, 1.5, 1.9)
    g.set_mrt_rates(*rates)
    o.set_group_rates(*rates)
    g.step(40)
    o.step(40)
    rg, ug = g.macro()
    ro, uo = o.macro()
    assert rel(ug, uo) < tol
    assert rel(rg - 1.0, ro - 1.0) < 10 * tol
    if storage == "f64":
        assert rel(g.populations(), o.populations()) < tol
    with pytest.raises(lbm.LbmError):
        g.set_mrt_rates(2.5, 1.3, 1.1, 1.5, 1.9)
    with pytest.raises(lbm.LbmError):
        g.set_mrt_rates(0.5, 1.3, 0.0, 1.5, 1.9)


@pytest.mark.parametrize("rates,tau", [(oracle.RATES_SRT, 0.6), (oracle.RATES_DHUMIERES, 0.51)])
def test_periodic_hit_f32_200_steps(lbm, rates, tau):
    n = 32
    u = workloads.hit_velocity(n, seed=0, k_peak=4.0, u_rms=0.03)
    g, o = pair(lbm, (n, n, n), tau, storage=lbm.F32, rates=rates)
    g.init_velocity(u)
    o.init_velocity(u)
    g.step(200)
    o.step(200)
    rg, ug = g.macro()
    ro, uo = o.macro()
    assert rel(rg, ro) < 1e-5
    assert rel(ug, uo) < 1e-5
    assert rel(g.populations(), o.populations()) < 1e-5


def _links_equal(a, b, q_exact=True, q_tol=1e-12):
    ka = np.lexsort((a["dir"], a["cell"]))
    kb = np.lexsort((b["dir"], b["cell"]))
    for k in ("cell", "dir", "scheme", "pid"):
        assert np.array_equal(np.asarray(a[k])[ka], np.asarray(b[k])[kb]), k
    if q_exact:
        assert np.array_equal(a["q"][ka].view(np.uint64), b["q"][kb].view(np.uint64))
    else:
        assert np.max(np.abs(a["q"][ka] - b["q"][kb])) < q_tol


def test_pipe_links_bit_exact(lbm):
    g, o = pair(lbm, (5, 40, 41), 0.6)
    g.set_pipe(18.3)
    o.set_pipe(18.3)
    _links_equal(g.links(), o.links())
    assert np.array_equal(g.flags() & 1, o.solid()[0])


def test_sphere_links_bit_exact(lbm):
    n = 40
    X = workloads.place_spheres((n, n, n), 12, 4.0, 0.5, seed=5)
    g, o = pair(lbm, (n, n, n), 0.6, max_particles=12)
    z = np.zeros((12, 3))
    g.add_spheres(X, 4.0, U=z, W=z, fixed=True)
    o.add_spheres(X, 4.0, U=z, W=z, fixed=True)
    _links_equal(g.links(), o.links())
    s, own = o.solid()
    assert np.array_equal(g.flags() & 1, s)
    L = g.links()
    assert set(np.unique(L["scheme"]).tolist()) <= {0, 1, 2}


@pytest.mark.parametrize("storage", ["f32", "bf16s"])
def test_sphere_links_reduced_storage(lbm, storage):
    """32/16-bit storage forms q as c0/(s - b) with an FP32 square root
    (error below 3e-7); the lists (cell, direction, scheme, particle) stay
    those of the exact FP64 q, which decides the scheme within 1e-5 of
    q = 1/2."""
    n = 40
    X = workloads.place_spheres((n, n, n), 12, 4.0, 0.5, seed=5)
    g, o = pair(lbm, (n, n, n), 0.6, storage=lbm.STORAGE[storage], max_particles=12)
    z = np.zeros((12, 3))
    g.add_spheres(X, 4.0, U=z, W=z, fixed=True)
    o.add_spheres(X, 4.0, U=z, W=z, fixed=True)
    a, b = g.links(), o.links()
    ka = np.lexsort((a["dir"], a["cell"]))
    kb = np.lexsort((b["dir"], b["cell"]))
    for k in ("cell", "dir", "scheme", "pid"):
        assert np.array_equal(np.asarray(a[k])[ka], np.asarray(b[k])[kb]), k
    assert np.max(np.abs(a["q"][ka] - b["q"][kb])) < 1e-6


def test_fixed_sphere_ibb_f64_drag_and_fields(lbm):
    """32^3 box, sphere R=4 at the centre, IBB, body force 1e-6, tau=0.6,
    +-1e-4 noise (the small FP64 sphere workload), 100 steps."""
    p = workloads.SPHERE_32
    n = p["n"]
    u = workloads.noise_velocity((n, n, n), p["noise"], seed=0)
    g, o = pair(lbm, (n, n, n), p["tau"], force=p["force"], max_particles=1)
    X = np.array([p["centre"]])
    z = np.zeros((1, 3))
    for s in (g, o):
        s.init_velocity(u)
        s.add_spheres(X, p["radius"], U=z, W=z, fixed=True)
    g.step(100, lbm.BC_IBB)
    o.step(100, oracle.BC_IBB)
    fluid = o.solid()[0] == 0
    assert rel(g.populations()[:, fluid], o.populations()[:, fluid]) < 1e-12
    Fg, Fo = g.particles()["F"][0], o.particles()["F"][0]
    assert np.max(np.abs(Fg - Fo)) < 1e-12 * max(1.0, np.max(np.abs(Fo)))
    sg, so = g.stats(), o.stats()
    for k in ("kinetic_energy", "dissipation", "mass"):
        assert sg[k] == pytest.approx(so[k], rel=1e-11, abs=1e-300), k


def test_moving_spheres_ibb_f64(lbm):
    n = 28
    X = workloads.place_spheres((n, n, n), 3, 3.5, 1.5, seed=2)
    u = workloads.hit_velocity(n, seed=4, k_peak=3.0, u_rms=0.02)
    g, o = pair(lbm, (n, n, n), 0.6, rates=oracle.RATES_DHUMIERES, max_particles=3)
    for s in (g, o):
        s.init_velocity(u)
        s.add_spheres(X, 3.5, density_ratio=1.5)
    Pg, Po = g.particles(), o.particles()
    assert rel(Pg["U"], Po["U"]) < 1e-12  # release velocity
    refilled = 0
    for _ in range(3):
        g.step(10, lbm.BC_IBB)
        for _ in range(10):  # the oracle one step at a time, counting uncovered nodes
            before = o.solid()[0]
            o.step(1, oracle.BC_IBB)
            refilled += int(((before == 1) & (o.solid()[0] == 0)).sum())
        Pg, Po = g.particles(), o.particles()
        for k in ("X", "U", "W"):
            assert np.max(np.abs(Pg[k] - Po[k])) < 1e-11 * max(1.0, np.max(np.abs(Po[k]))), k
        assert rel(Pg["F"], Po["F"]) < 1e-9
        fluid = o.solid()[0] == 0
        assert np.array_equal(g.flags() & 1, o.solid()[0])
        assert rel(g.populations()[:, fluid], o.populations()[:, fluid]) < 1e-11
    assert refilled > 0
    # positions now differ in the last bits (forces summed in another order),
    # so q can differ in the last bits too; the list itself must agree
    _links_equal(g.links(), o.links(), q_exact=False)
    # bit-exact for identical positions: rebuild both from the GPU's positions
    X = g.particles()["X"]
    g2, o2 = pair(lbm, (n, n, n), 0.6, max_particles=3)
    z = np.zeros((3, 3))
    g2.add_spheres(X, 3.5, U=z, W=z, fixed=True)
    o2.add_spheres(X, 3.5, U=z, W=z, fixed=True)
    _links_equal(g2.links(), o2.links())


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_pipe_ibb_200_steps(lbm, storage, tol):
    """Pipe wall by interpolated bounce-back: rows of up to 43 fluid cells,
    i.e. two ragged sweep segments per row, plus the z-periodic ends."""
    nx, ny, nz, R = 47, 46, 12, 21.5
    g, o = pair(lbm, (nz, ny, nx), 0.6, force=(0, 0, 2e-6),
                storage=lbm.F64 if storage == "f64" else lbm.F32)
    u = workloads.pipe_velocity(nx, ny, nz, R, 0.02, perturbation=0.1, seed=4)
    for s in (g, o):
        s.init_velocity(u)
        s.set_pipe(R)
    g.step(200, lbm.BC_IBB)
    o.step(200, oracle.BC_IBB)
    fluid = o.solid()[0] == 0  # solid cells hold ghost values on the GPU
    assert rel(g.populations()[:, fluid], o.populations()[:, fluid]) < tol
    rg, ug = g.macro()
    ro, uo = o.macro()
    assert rel(ug[:, fluid], uo[:, fluid]) < tol
    assert rel(rg[fluid], ro[fluid]) < tol
    # rho - 1 is O(1e-6) here: FP64 resolves it to 1e-8 of itself. In FP32
    # every step rounds the 19 stored values (|g| <= 0.02, half an ulp
    # 1e-9), so rho = 1 + sum g random-walks by about
    # sqrt(19 x 200) x 1e-9 = 6e-8; the bar is three times that.
    if storage == "f64":
        assert rel(rg[fluid] - 1.0, ro[fluid] - 1.0) < 1e-8
    else:
        assert np.max(np.abs(rg[fluid] - ro[fluid])) < 2e-7


@pytest.mark.parametrize("bc,nz", [("ibm_u", 4), ("ibm_b", 4), ("ibm_b", 31)])
def test_pipe_ibm_f64(lbm, bc, nz):
    # nz = 31: the pipe's interpolation and spreading run on six z tiles of
    # 6 planes (the last one ragged) whose halo planes wrap at both ends
    shape = (nz, 26, 27)
    gpar = (0, 0, 2e-6)
    g, o = pair(lbm, shape, 0.7, force=gpar)
    u = workloads.pipe_velocity(27, 26, nz, 10.0, 0.01, perturbation=0.05, seed=1)
    for s in (g, o):
        s.init_velocity(u)
        s.set_pipe(10.0)
    g.step(40, lbm.BC[bc])
    o.step(40, oracle.BC_IBM_U if bc == "ibm_u" else oracle.BC_IBM_B)
    assert rel(g.populations(), o.populations()) < 1e-11
    assert rel(g.ibm_force(), o.ibm_force()) < 1e-10
    mg, mo = g.markers(), o.markers()
    assert len(mg["dV"]) == len(mo["dV"])
    assert rel(mg["F"], mo["F"]) < 1e-10


@pytest.mark.parametrize("bc", ["ibm_u", "ibm_b"])
def test_pipe_ibm_f32_200_steps(lbm, bc):
    """Pipe wall by IBM in FP32 storage: an odd row length (warps of the box
    sweep cross row ends), support cells collided in place after the three
    passes, and the pipe's interpolation and spreading on five z tiles."""
    nx, ny, nz, R = 47, 46, 30, 21.5
    g, o = pair(lbm, (nz, ny, nx), 0.6, force=(0, 0, 2e-6), storage=lbm.F32)
    u = workloads.pipe_velocity(nx, ny, nz, R, 0.02, perturbation=0.1, seed=4)
    for s in (g, o):
        s.init_velocity(u)
        s.set_pipe(R)
    g.step(200, lbm.BC[bc])
    o.step(200, oracle.BC_IBM_U if bc == "ibm_u" else oracle.BC_IBM_B)
    rg, ug = g.macro()
    ro, uo = o.macro()
    assert rel(ug, uo) < 1e-5
    assert rel(rg, ro) < 1e-5
    # F = 2 rho (U_d - U*) is about 600 times smaller than u here, and its
    # error is that of the interpolated velocity U*: the same 1e-5 bar holds
    # for U* = -F / (2 rho) on the velocity's scale
    dF = np.max(np.abs(g.ibm_force() - o.ibm_force()))
    assert dF / (2 * np.max(np.abs(uo))) < 1e-5


@pytest.mark.parametrize("bc", ["ibm_u", "ibm_b"])
def test_moving_spheres_ibm_f64(lbm, bc):
    n = 26
    X = workloads.place_spheres((n, n, n), 2, 4.0, 2.0, seed=9)
    u = workloads.hit_velocity(n, seed=6, k_peak=3.0, u_rms=0.02)
    g, o = pair(lbm, (n, n, n), 0.65, rates=oracle.RATES_DHUMIERES, max_particles=2)
    for s in (g, o):
        s.init_velocity(u)
        s.add_spheres(X, 4.0, density_ratio=5.0)
    obc = oracle.BC_IBM_U if bc == "ibm_u" else oracle.BC_IBM_B
    for _ in range(2):
        g.step(10, lbm.BC[bc])
        o.step(10, obc)
        Pg, Po = g.particles(), o.particles()
        # the inner-fluid term is a difference of nearly equal sums and the
        # spreading adds in another order: particle quantities agree to ~1e-9
        for k in ("X", "U", "W"):
            assert np.max(np.abs(Pg[k] - Po[k])) < 1e-10 * max(1.0, np.max(np.abs(Po[k]))), k
        assert rel(Pg["F"], Po["F"]) < 1e-8
        assert rel(g.populations(), o.populations()) < 1e-10
    sg, so = g.stats(oracle.STATS_BINS), o.stats(oracle.STATS_BINS)
    assert sg["particle_ke"] == pytest.approx(so["particle_ke"], rel=1e-7)
    assert sg["dissipation"] == pytest.approx(so["dissipation"], rel=1e-9)
    assert np.array_equal(sg["bin_count"], so["bin_count"])
    assert np.allclose(sg["bin_eps"], so["bin_eps"], rtol=1e-8)


def test_moving_spheres_ibb_f32_within_tolerance(lbm):
    n = 32
    X = workloads.place_spheres((n, n, n), 4, 4.0, 1.5, seed=12)
    u = workloads.hit_velocity(n, seed=8, k_peak=3.0, u_rms=0.03)
    g, o = pair(lbm, (n, n, n), 0.55, storage=lbm.F32, rates=oracle.RATES_DHUMIERES, max_particles=4)
    for s in (g, o):
        s.init_velocity(u)
        s.add_spheres(X, 4.0, density_ratio=5.0)
    g.step(200, lbm.BC_IBB)
    o.step(200, oracle.BC_IBB)
    fluid = (o.solid()[0] == 0) & ((g.flags() & 1) == 0)
    rg, ug = g.macro()
    ro, uo = o.macro()
    assert rel(ug[:, fluid], uo[:, fluid]) < 1e-5
    assert rel(rg[fluid], ro[fluid]) < 1e-5
    Pg, Po = g.particles(), o.particles()
    assert rel(Pg["U"], Po["U"]) < 1e-5
    assert rel(Pg["W"], Po["W"]) < 1e-5


@pytest.mark.parametrize("storage,tol", [("f16s", 2e-3), ("bf16s", 3e-2)])
def test_16bit_storage_error_bounded(lbm, storage, tol):
    n = 32
    u = workloads.hit_velocity(n, seed=0, k_peak=4.0, u_rms=0.03)
    g, o = pair(lbm, (n, n, n), 0.6, storage=lbm.STORAGE[storage])
    g.init_velocity(u)
    o.init_velocity(u)
    g.step(100)
    o.step(100)
    ug, uo = g.macro()[1], o.macro()[1]
    assert rel(ug, uo) < tol


@pytest.mark.parametrize("storage,tol", [("f16s", 2e-3), ("bf16s", 3e-2)])
def test_16bit_storage_ragged_rows_and_pipe(lbm, storage, tol):
    """16-bit storage on a 70-wide periodic box (rows of two and a ragged
    piece, periodic x ends) and on a pipe swept by fluid-run segments."""
    nx, ny, nz = 70, 18, 10
    u = workloads.noise_velocity((nz, ny, nx), 0.02, seed=5)
    g, o = pair(lbm, (nz, ny, nx), 0.6, force=(1e-5, 0, 0), storage=lbm.STORAGE[storage])
    g.init_velocity(u)
    o.init_velocity(u)
    g.step(100)
    o.step(100)
    assert rel(g.macro()[1], o.macro()[1]) < tol
    nx, ny, nz, R = 46, 46, 8, 21.5
    g, o = pair(lbm, (nz, ny, nx), 0.6, force=(0, 0, 2e-6), storage=lbm.STORAGE[storage])
    u = workloads.pipe_velocity(nx, ny, nz, R, 0.02, perturbation=0.1, seed=4)
    for s in (g, o):
        s.init_velocity(u)
        s.set_pipe(R)
    g.step(100, lbm.BC_IBB)
    o.step(100, oracle.BC_IBB)
    fluid = o.solid()[0] == 0
    assert rel(g.macro()[1][:, fluid], o.macro()[1][:, fluid]) < tol


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("f16s", 2e-3), ("bf16s", 3e-2)])
def test_pipe_ibb_without_body_force(lbm, storage, tol):
    """The pipe sweeps' variants without a body force (a perturbed flow
    decaying against the wall): the one-cell FP32 sweep and the 16-bit pair
    sweep, each with the wall inside the sweep, over 150 steps."""
    nx, ny, nz, R = 46, 44, 10, 20.5
    g, o = pair(lbm, (nz, ny, nx), 0.62, storage=lbm.STORAGE[storage])
    u = workloads.pipe_velocity(nx, ny, nz, R, 0.03, perturbation=0.2, seed=9)
    for s in (g, o):
        s.init_velocity(u)
        s.set_pipe(R)
    g.step(150, lbm.BC_IBB)
    o.step(150, oracle.BC_IBB)
    fluid = o.solid()[0] == 0
    assert rel(g.macro()[1][:, fluid], o.macro()[1][:, fluid]) < tol
    if storage == "f32":
        assert rel(g.populations()[:, fluid], o.populations()[:, fluid]) < tol


@pytest.mark.parametrize("storage,tol", [("f16s", 2e-3), ("bf16s", 3e-2)])
def test_16bit_pipe_odd_width_one_cell_sweep(lbm, storage, tol):
    """A pipe of odd width on 16-bit storage: pairs of cells do not share
    aligned words, so the one-cell sweep of the inline wall form runs
    (even widths take the two-cells-per-lane sweep)."""
    nx, ny, nz, R = 47, 46, 8, 21.5
    g, o = pair(lbm, (nz, ny, nx), 0.6, force=(0, 0, 2e-6), storage=lbm.STORAGE[storage])
    u = workloads.pipe_velocity(nx, ny, nz, R, 0.02, perturbation=0.1, seed=6)
    for s in (g, o):
        s.init_velocity(u)
        s.set_pipe(R)
    g.step(100, lbm.BC_IBB)
    o.step(100, oracle.BC_IBB)
    fluid = o.solid()[0] == 0
    assert rel(g.macro()[1][:, fluid], o.macro()[1][:, fluid]) < tol


def test_moving_spheres_ibm_b_f32_200_steps(lbm):
    """The particle-laden IBM-B step in FP32 storage (the benchmark's HIT
    path) over 200 steps: velocity, density and the particles' motion."""
    n = 32
    X = workloads.place_spheres((n, n, n), 3, 4.0, 2.0, seed=21)
    u = workloads.hit_velocity(n, seed=8, k_peak=3.0, u_rms=0.03)
    g, o = pair(lbm, (n, n, n), 0.55, storage=lbm.F32, rates=oracle.RATES_DHUMIERES, max_particles=3)
    for s in (g, o):
        s.init_velocity(u)
        s.add_spheres(X, 4.0, density_ratio=5.0)
    g.step(200, lbm.BC_IBM_B)
    o.step(200, oracle.BC_IBM_B)
    rg, ug = g.macro()
    ro, uo = o.macro()
    assert rel(ug, uo) < 1e-5
    assert rel(rg, ro) < 1e-5
    Pg, Po = g.particles(), o.particles()
    for k in ("U", "W"):
        assert rel(Pg[k], Po[k]) < 1e-5, k
    assert np.max(np.abs(Pg["X"] - Po["X"])) < 1e-5


@pytest.mark.parametrize("bc", ["ibb", "ibm_b"])
def test_soft_sphere_contact(lbm, bc):
    """Two spheres of density ratio 5, 0.5 lu apart and closing: the normal
    spring-dashpot contact (margin 1 lu) acts from the first step and turns
    them back; positions and velocities match the oracle through the
    collision."""
    n = 32
    X = np.array([[11.25, 16.0, 15.7], [19.75, 16.3, 16.1]])  # centres 8.5 + apart, radii 4: gap ~0.5
    U = np.array([[0.02, 0.0, 0.0], [-0.02, 0.0, 0.0]])
    u = workloads.noise_velocity((n, n, n), 1e-3, seed=1)
    g, o = pair(lbm, (n, n, n), 0.6, rates=oracle.RATES_DHUMIERES, max_particles=2)
    for s in (g, o):
        s.init_velocity(u)
        s.add_spheres(X, 4.0, density_ratio=5.0, U=U, W=np.zeros((2, 3)))
    d0 = np.linalg.norm(X[1] - X[0]) - 8.0
    assert d0 < 1.0  # inside the contact margin at the start
    obc = oracle.BC_IBB if bc == "ibb" else oracle.BC_IBM_B
    vrel = [U[1, 0] - U[0, 0]]
    for _ in range(6):
        g.step(5, lbm.BC[bc])
        o.step(5, obc)
        Pg, Po = g.particles(), o.particles()
        for k in ("X", "U", "W"):
            assert np.max(np.abs(Pg[k] - Po[k])) < 1e-10 * max(1.0, np.max(np.abs(Po[k]))), k
        vrel.append(Po["U"][1, 0] - Po["U"][0, 0])
    assert vrel[0] < 0 and vrel[-1] > 0  # closing at first, separating after the contact
    assert max(vrel) > 0.05  # turned back by the spring (the fluid alone could not do it)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_single_node_fallback_between_close_spheres(lbm, storage, tol):
    """Two fixed spheres 0.6 lu apart: links in the gap whose upstream node
    is solid take the single-node scheme; with a body force and a random
    flow the GPU matches the oracle."""
    n = 20
    X = np.array([[6.3, 10.1, 9.7], [12.1, 10.4, 9.9]])
    g, o = pair(lbm, (n, n, n), 0.6, force=(1e-5, 2e-6, 0), storage=lbm.STORAGE[storage],
                rates=oracle.RATES_DHUMIERES, max_particles=2)
    u = workloads.hit_velocity(n, seed=3, k_peak=2.0, u_rms=0.01)
    z = np.zeros((2, 3))
    for s in (g, o):
        s.init_velocity(u)
        s.add_spheres(X, 2.6, U=z, W=np.array([[0, 0, 0.01], [0.005, 0, 0]]), fixed=True)
    L = o.links()
    assert (L["scheme"] == oracle.SCHEME_SINGLE).sum() >= 10
    # sphere links of 32/16-bit storage carry q to FP32 accuracy (3e-7)
    _links_equal(g.links(), o.links(), q_exact=storage == "f64", q_tol=1e-6)
    g.step(60, lbm.BC_IBB)
    o.step(60, oracle.BC_IBB)
    fluid = o.solid()[0] == 0
    assert rel(g.populations()[:, fluid], o.populations()[:, fluid]) < tol
    Fg, Fo = g.particles(), o.particles()
    assert rel(Fg["F"], Fo["F"]) < (1e-10 if storage == "f64" else 1e-4)
    assert rel(Fg["T"], Fo["T"]) < (1e-10 if storage == "f64" else 1e-4)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5), ("bf16s", 3e-2)])
def test_single_node_fallback_on_pipe_wall(lbm, storage, tol):
    """A pipe of radius 6.4 in a 16 x 16 section has wall links whose
    upstream node is outside the pipe (8 per plane): the static wall's ghost
    pass evaluates the single-node scheme from the wall cell's kept
    values."""
    nx, ny, nz, R = 16, 16, 6, 6.4
    g, o = pair(lbm, (nz, ny, nx), 0.6, force=(0, 0, 5e-6), storage=lbm.STORAGE[storage])
    u = workloads.pipe_velocity(nx, ny, nz, R, 0.01, perturbation=0.1, seed=2)
    for s in (g, o):
        s.init_velocity(u)
        s.set_pipe(R)
    assert (o.links()["scheme"] == oracle.SCHEME_SINGLE).sum() == 8 * nz
    g.step(200, lbm.BC_IBB)
    o.step(200, oracle.BC_IBB)
    fluid = o.solid()[0] == 0
    rg, ug = g.macro()
    ro, uo = o.macro()
    assert rel(ug[:, fluid], uo[:, fluid]) < tol
