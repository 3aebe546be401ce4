"""Pin of the oracle's energy-mode rate, the bulk-viscosity knob of the MRT
solver (Sec. 2.2: present in the paper's code but left off).

A standing sound wave rho = 1 + A cos(kx) released from rest in a periodic
box decays as exp(-Gamma t) with, for the linearised isothermal
Navier-Stokes equations, Gamma = k^2 (4 nu / 3 + nu_b) / 2. For the D3Q19
MRT of d'Humieres et al. (2002), nu = (1/s_nu - 1/2) / 3 and
nu_b = (2/9) (1/s_e - 1/2), so with s_e = 1/tau the bulk viscosity is the
BGK value 2 nu / 3. The rate is measured from the wave's acoustic energy
a^2 + (b / c_s)^2, where a and b are the cos(kx) and sin(kx) projections of
rho - 1 and u_x, fitted over whole half periods.
"""
import numpy as np
import pytest

import oracle

NX, NY, NZ, TAU, AMP = 64, 4, 4, 0.8, 1e-4


def decay_rate(s_e, steps=560):
    o = oracle.Sim(NX, NY, NZ, TAU)
    if s_e is not None:
        o.set_group_rates(s_e, 1.4, 1.2, 1.4, 1.98)
    _, w, _ = oracle.lattice()
    k = 2 * np.pi / NX
    x = np.arange(NX)
    rho = np.broadcast_to(1.0 + AMP * np.cos(k * x), (NZ, NY, NX)).reshape(-1)
    o.set_populations(np.asarray(w)[:, None] * rho[None, :])
    cs = 1 / np.sqrt(3)
    E = []
    for _ in range(steps):
        o.step(1)
        r, u = o.macro()
        rb = r.reshape(NZ, NY, NX).mean(axis=(0, 1)) - 1.0
        ub = u[0].reshape(NZ, NY, NX).mean(axis=(0, 1))
        a = 2.0 / NX * np.sum(rb * np.cos(k * x))
        b = 2.0 / NX * np.sum(ub * np.sin(k * x))
        E.append(a * a + (b / cs) ** 2)
    o.close()
    t = np.arange(1, steps + 1)
    slope = np.polyfit(t, np.log(np.array(E)), 1)[0]
    return -0.5 * slope


def theory(s_e):
    k = 2 * np.pi / NX
    nu = (TAU - 0.5) / 3
    nu_b = 2.0 / 9.0 * (1.0 / s_e - 0.5)
    return 0.5 * k * k * (4 * nu / 3 + nu_b)


def test_sound_attenuation_gives_the_bulk_viscosity():
    g_bgk = decay_rate(None)             # all rates 1/tau: nu_b = 2 nu / 3
    g_low = decay_rate(0.5)              # nu_b = (2/9)(2 - 1/2) = 1/3
    assert g_bgk == pytest.approx(theory(1 / TAU), rel=0.01)
    assert g_low == pytest.approx(theory(0.5), rel=0.01)
    # the difference isolates the bulk viscosity: (k^2 / 2) delta nu_b
    k = 2 * np.pi / NX
    d_nu_b = 2.0 / 9.0 * (1 / 0.5 - TAU)
    assert (g_low - g_bgk) == pytest.approx(0.5 * k * k * d_nu_b, rel=0.01)
