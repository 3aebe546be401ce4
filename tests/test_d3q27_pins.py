"""Pins of the D3Q27 oracle (oracle/d3q27.py), the velocity set of the
paper's pipe solver (Sec. 2.1), against mathematics that its code does not
compute:

- the lattice: 1 + 6 + 12 + 8 velocities whose weights make the moment
  tensors isotropic up to fourth order (sum w = 1, sum w c c = I/3,
  sum w c c c c = (dd + dd + dd)/9, odd moments zero, brute force over
  all index tuples) and sum w c_x^2 c_y^2 c_z^2 = 1/27;
- the equilibrium's moments: rho, rho u and rho (u u + I/3), exactly;
- a step conserves mass exactly and adds F to the momentum of every cell
  (Guo forcing: the half-force shift and the source add up to F), and a
  fluid at rest pushed for n steps moves at (n - 1/2) F;
- a Taylor-Green vortex decays at 2 nu k^2 with nu = (tau - 1/2)/3, within
  1 % at N = 32, and the error falls about 4x from N = 16 to N = 32;
- a step commutes with a cubic rotation of the box (x -> y -> z -> x);
- streaming moves a population along its own velocity (pull:
  f(x, t+1) = f*(x - c, t)), and a shear wave u_y = e sin(kx) on a uniform
  flow U along x is carried downstream at U while it decays at nu k^2
  (u_y = e exp(-nu k^2 t) sin(k (x - U t)));
- the pipe wall: every fluid cell with a solid neighbour is a link, and
  its q is the root of the cylinder equation found by bisection; a fluid
  at rest stays at rest (the interpolation weights sum to one); the
  steady flow driven by a body force is the Hagen-Poiseuille profile
  g (R^2 - r^2) / (4 nu) within 0.4 % at R = 8 (the D3Q19 oracle, with the
  same wall, reaches 0.19 %).
"""
import itertools

import numpy as np
import pytest

from oracle import d3q27 as q27


def test_lattice_groups_and_isotropy():
    c, w = q27.lattice()
    n2 = np.sum(c * c, axis=1)
    assert [int(np.sum(n2 == k)) for k in range(4)] == [1, 6, 12, 8]
    assert len({tuple(v) for v in c}) == 27
    assert np.sum(w) == pytest.approx(1.0, abs=1e-15)
    d = np.eye(3)
    for a in range(3):
        assert abs(np.sum(w * c[:, a])) < 1e-16
        for b in range(3):
            assert np.sum(w * c[:, a] * c[:, b]) == pytest.approx(d[a, b] / 3, abs=1e-15)
            for e in range(3):
                assert abs(np.sum(w * c[:, a] * c[:, b] * c[:, e])) < 1e-16
    for a, b, e, g in itertools.product(range(3), repeat=4):
        expect = (d[a, b] * d[e, g] + d[a, e] * d[b, g] + d[a, g] * d[b, e]) / 9
        assert np.sum(w * c[:, a] * c[:, b] * c[:, e] * c[:, g]) == pytest.approx(expect, abs=1e-15)
    assert np.sum(w * c[:, 0] ** 2 * c[:, 1] ** 2 * c[:, 2] ** 2) == pytest.approx(1 / 27, abs=1e-16)


def test_equilibrium_moments():
    rng = np.random.default_rng(1)
    rho = 1 + 0.05 * rng.standard_normal((3, 4, 5))
    u = 0.05 * rng.standard_normal((3, 3, 4, 5))
    f = q27.feq(rho, u)
    c = q27.C.astype(np.float64)
    assert np.max(np.abs(np.sum(f, axis=0) - rho)) < 1e-15
    j = np.einsum("ia,i...->a...", c, f)
    assert np.max(np.abs(j - rho * u)) < 1e-15
    P = np.einsum("ia,ib,i...->ab...", c, c, f)
    expect = rho * (np.einsum("a...,b...->ab...", u, u) + np.eye(3)[:, :, None, None, None] / 3)
    assert np.max(np.abs(P - expect)) < 1e-15


def test_step_conserves_mass_and_adds_the_force():
    rng = np.random.default_rng(2)
    shape = (5, 6, 7)
    f = q27.W.reshape(27, 1, 1, 1) * (1 + 0.1 * rng.random((27,) + shape))
    F = np.array([2e-4, -1e-4, 5e-5])
    c = q27.C.astype(np.float64)
    m0, p0 = np.sum(f), np.einsum("ia,izyx->a", c, f)
    g = q27.step(f, 0.7, F, n=3)
    m1, p1 = np.sum(g), np.einsum("ia,izyx->a", c, g)
    assert m1 == pytest.approx(m0, rel=1e-14)
    N = np.prod(shape)
    assert p1 == pytest.approx(p0 + 3 * N * F, abs=1e-12)
    # a uniform fluid at rest pushed for n steps: the stored (post-collision)
    # momentum is n F and the velocity of the last collision (n - 1/2) F
    h = q27.feq(np.ones((2, 2, 2)), np.zeros((3, 2, 2, 2)))
    rho, u = q27.macro(q27.step(h, 0.7, F, n=4), F)
    assert np.max(np.abs(u - 3.5 * F.reshape(3, 1, 1, 1))) < 1e-15
    assert np.max(np.abs(rho - 1.0)) < 1e-15


def tgv_rate(n, tau=0.8, u0=1e-3, steps=120, skip=20):
    k = 2 * np.pi / n
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    u = np.zeros((3, 2, n, n))
    u[0] = -u0 * np.cos(k * x) * np.sin(k * y)
    u[1] = u0 * np.sin(k * x) * np.cos(k * y)
    f = q27.feq(np.ones((2, n, n)), u)
    E = []
    for _ in range(steps):
        f = q27.step(f, tau)
        _, v = q27.macro(f)
        E.append(np.sum(v * v))
    t = np.arange(1, steps + 1)
    slope = np.polyfit(t[skip:], np.log(E[skip:]), 1)[0]
    nu = (tau - 0.5) / 3
    return -0.5 * slope, 2 * nu * k * k


def test_taylor_green_decay_and_convergence():
    g32, t32 = tgv_rate(32)
    g16, t16 = tgv_rate(16)
    e32, e16 = abs(g32 / t32 - 1), abs(g16 / t16 - 1)
    assert e32 < 0.01
    assert e16 / e32 == pytest.approx(4.0, rel=0.3)


def test_step_commutes_with_a_cubic_rotation():
    rng = np.random.default_rng(3)
    n = 6
    f = q27.W.reshape(27, 1, 1, 1) * (1 + 0.05 * rng.random((27, n, n, n)))
    F = np.array([1e-4, 2e-4, -3e-4])
    # rotation R: x -> y -> z -> x, i.e. velocity (a, b, e) -> (e, a, b);
    # a field g(x, y, z) = f(z, x, y) on axes (z, y, x)
    c = q27.C
    perm = [int(np.flatnonzero((c == np.array([v[2], v[0], v[1]])).all(axis=1))[0]) for v in c]

    def rotate(h):
        out = np.empty_like(h)
        for i in range(27):
            # new[z', y', x'] = old[y', x', z'] for new coordinates (x', y', z') = (z, x, y)
            out[perm[i]] = np.transpose(h[i], (1, 2, 0))
        return out

    Fr = np.array([F[2], F[0], F[1]])
    a = rotate(q27.step(f, 0.65, F, n=2))
    b = q27.step(rotate(f), 0.65, Fr, n=2)
    assert np.max(np.abs(a - b)) < 1e-15


def test_streaming_moves_along_the_velocity():
    n = 5
    for i, ci in enumerate(q27.C):
        f = np.zeros((27, n, n, n))
        f[i, 2, 2, 2] = 1.0
        g = q27.stream(f)
        z, y, x = (int(v[0]) for v in np.nonzero(g[i]))
        assert (x, y, z) == (2 + ci[0], 2 + ci[1], 2 + ci[2])
        assert np.count_nonzero(g) == 1


def test_shear_wave_is_carried_by_the_flow():
    n, tau, U, e, T = 32, 0.8, 0.05, 1e-4, 50
    k = 2 * np.pi / n
    x = np.arange(n)
    u = np.zeros((3, 2, 2, n))
    u[0] = U
    u[1] = e * np.sin(k * x)
    f = q27.feq(np.ones((2, 2, n)), u)
    f = q27.step(f, tau, n=T)
    _, v = q27.macro(f)
    uy = v[1].mean(axis=(0, 1))
    a, b = np.sum(uy * np.sin(k * x)), np.sum(uy * np.cos(k * x))
    phase = np.arctan2(-b, a)          # k U T for a wave carried downstream
    assert phase == pytest.approx(k * U * T, rel=0.02)
    nu = (tau - 0.5) / 3
    amp = 2 * np.hypot(a, b) / n
    assert amp == pytest.approx(e * np.exp(-nu * k * k * T), rel=0.02)


@pytest.mark.parametrize("R", [7.3, 6.0])  # 6.0: cells at r^2 = 36.5 lie just outside the wall
def test_pipe_links_q_by_bisection(R):
    n, nz = 20, 3
    solid = q27.pipe_solid(n, n, nz, R)
    links = q27.pipe_links(solid, R)
    c0 = 0.5 * (n - 1)
    nlinks = 0
    for i, (m, q, up) in enumerate(links):
        ci = q27.C[i]
        # every fluid cell with a solid neighbour along c_i is a link
        nb = np.roll(solid, shift=(-ci[2], -ci[1], -ci[0]), axis=(0, 1, 2))
        assert np.array_equal(m, ~solid & nb)
        for z, y, x in zip(*np.nonzero(m)):
            nlinks += 1
            dx, dy = x - c0, y - c0
            h = lambda t: (dx + t * ci[0]) ** 2 + (dy + t * ci[1]) ** 2 - R * R
            lo, hi = 0.0, 1.0
            assert h(lo) < 0 <= h(hi)
            for _ in range(80):
                mid = 0.5 * (lo + hi)
                lo, hi = (mid, hi) if h(mid) < 0 else (lo, mid)
            assert 0 < q[z, y, x] <= 1
            assert abs(q[z, y, x] - 0.5 * (lo + hi)) < 1e-12
    assert nlinks > 100


def test_pipe_keeps_a_fluid_at_rest():
    R, n = 6.4, 16
    solid = q27.pipe_solid(n, n, 2, R)
    links = q27.pipe_links(solid, R)
    f = np.broadcast_to(q27.W.reshape(27, 1, 1, 1), (27, 2, n, n)).copy()
    g = f
    for _ in range(3):
        g = q27.step_pipe(g, solid, links, 0.7)
    assert np.max(np.abs(g - f)) < 1e-16


def test_pipe_hagen_poiseuille():
    R, tau, grav = 8.0, 0.8, 1e-6
    n = int(2 * np.ceil(R) + 4)
    solid = q27.pipe_solid(n, n, 1, R)
    links = q27.pipe_links(solid, R)
    nu = (tau - 0.5) / 3
    _, y, x = np.meshgrid(np.arange(1), np.arange(n), np.arange(n), indexing="ij")
    r2 = (x - 0.5 * (n - 1)) ** 2 + (y - 0.5 * (n - 1)) ** 2
    exact = np.where(solid, 0.0, grav * (R * R - r2) / (4 * nu))
    u = np.zeros((3,) + solid.shape)
    u[2] = exact
    F = (0.0, 0.0, grav)
    f = q27.feq(np.ones(solid.shape), u)
    for _ in range(int(3 * R * R / nu)):
        f = q27.step_pipe(f, solid, links, tau, F)
    _, v = q27.macro(f, F)
    fl = ~solid
    err = np.sqrt(np.sum((v[2][fl] - exact[fl]) ** 2) / np.sum(exact[fl] ** 2))
    assert err < 0.004
    assert np.max(np.abs(v[0][fl])) < 1e-6 * np.max(exact) and np.max(np.abs(v[1][fl])) < 1e-6 * np.max(exact)
