"""D3Q27 oracle: the velocity set of the paper's pipe solver (test infrastructure).

TEST INFRASTRUCTURE ONLY: a plain numpy statement of one D3Q27 lattice
Boltzmann step on a periodic box. The paper's pipe runs used a D3Q27 MRT
model with a single relaxation parameter (Sec. 2.1), which is BGK when the
equilibrium moments are those of the equilibrium distribution. Readings
(the paper gives no formulas):

- velocities: all c in {-1, 0, 1}^3, ordered rest, the 6 faces, the 12
  edges, the 8 corners (each group in the order of itertools.product over
  (-1, 0, 1)); weights 8/27, 2/27, 1/54, 1/216 (the product of the 1D
  weights 2/3 and 1/6);
- equilibrium: the same second-order polynomial as for D3Q19,
  f_eq = w rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u);
- body force by Guo et al. (2002): u = (sum f c + F/2) / rho and the source
  (1 - 1/(2 tau)) w [3 (c - u) + 9 (c.u) c] . F;
- a step is pull streaming f(x) <- f*(x - c) with periodic wrap, then the
  collision f* = f - (f - f_eq) / tau + source; the stored state is the
  post-collision one (as for D3Q19), whose velocity is
  u = (sum f* c - F/2) / rho.

Populations have shape (27, nz, ny, nx), x fastest.
"""
from __future__ import annotations

import itertools

import numpy as np

Q = 27


def lattice():
    """(c, w): c of shape (27, 3) integers, w of shape (27,)."""
    cs = list(itertools.product((-1, 0, 1), repeat=3))
    groups = {k: [c for c in cs if sum(abs(v) for v in c) == k] for k in range(4)}
    c = np.array(groups[0] + groups[1] + groups[2] + groups[3], dtype=np.int64)
    w1 = {0: 2.0 / 3.0, 1: 1.0 / 6.0}
    w = np.array([w1[abs(a)] * w1[abs(b)] * w1[abs(d)] for a, b, d in c])
    return c, w


C, W = lattice()


def feq(rho, u):
    """Equilibrium populations for rho of shape S and u of shape (3,) + S."""
    cu = np.tensordot(C.astype(np.float64), u, axes=(1, 0))
    uu = np.sum(u * u, axis=0)
    return W.reshape((Q,) + (1,) * np.ndim(rho)) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu)


def moments(f, F):
    """rho and the forced velocity u = (sum f c + F/2) / rho."""
    rho = np.sum(f, axis=0)
    j = np.tensordot(C.T.astype(np.float64), f, axes=(1, 0))
    u = (j + 0.5 * np.asarray(F, dtype=np.float64).reshape((3,) + (1,) * np.ndim(rho))) / rho
    return rho, u


def collide(f, tau, F=(0.0, 0.0, 0.0)):
    """BGK collision with the Guo source, cell by cell (any trailing shape)."""
    Fv = np.asarray(F, dtype=np.float64)
    rho, u = moments(f, Fv)
    cu = np.tensordot(C.astype(np.float64), u, axes=(1, 0))
    shape = (Q,) + (1,) * np.ndim(rho)
    cF = (C.astype(np.float64) @ Fv).reshape(shape)
    uF = np.tensordot(Fv, u, axes=(0, 0))
    src = W.reshape(shape) * (3.0 * (cF - uF) + 9.0 * cu * cF)
    return f - (f - feq(rho, u)) / tau + (1.0 - 0.5 / tau) * src


def stream(f):
    """Pull streaming with periodic wrap: f_i(x) <- f_i(x - c_i)."""
    out = np.empty_like(f)
    for i in range(Q):
        cx, cy, cz = (int(v) for v in C[i])
        out[i] = np.roll(f[i], shift=(cz, cy, cx), axis=(0, 1, 2))
    return out


def step(f, tau, F=(0.0, 0.0, 0.0), n=1):
    """n steps of the post-collision state: stream, then collide."""
    for _ in range(n):
        f = collide(stream(f), tau, F)
    return f


def macro(f, F=(0.0, 0.0, 0.0)):
    """rho and u of a post-collision state: the collision added F to the
    momentum rho u - F/2 of its input, so u = (sum f c - F/2) / rho."""
    rho = np.sum(f, axis=0)
    j = np.tensordot(C.T.astype(np.float64), f, axes=(1, 0))
    u = (j - 0.5 * np.asarray(F, dtype=np.float64).reshape((3,) + (1,) * np.ndim(rho))) / rho
    return rho, u


# ---------------------------------------------------------------- pipe wall --
# The pipe of the paper's runs (Sec. 2.1) with the linear interpolated
# bounce-back, read as for D3Q19: a cell is solid iff
# (x - c_x)^2 + (y - c_y)^2 >= R^2 with the axis at ((nx-1)/2, (ny-1)/2)
# along z; a link (x_f, i) joins a fluid cell to a solid x_f + c_i, and the
# wall sits at x_f + q c_i with q the root in (0, 1] of
# |d + q c_perp|^2 = R^2 (d = (x - c_x, y - c_y), c_perp = (c_x, c_y)).
# The unknown f_ibar(x_f) after streaming is, with post-collision values f*
# and a wall at rest (Bouzidi et al. 2001, linear):
#   q < 1/2: 2q f*_i(x_f) + (1 - 2q) f*_i(x_f - c_i), if x_f - c_i is fluid,
#            else f*_i(x_f) (halfway bounce-back);
#   q >= 1/2: f*_i(x_f) / (2q) + (2q - 1) / (2q) f*_ibar(x_f).

OPP = np.array([int(np.flatnonzero((C == -C[i]).all(axis=1))[0]) for i in range(Q)])


def pipe_solid(nx, ny, nz, R):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    dx, dy = x - 0.5 * (nx - 1), y - 0.5 * (ny - 1)
    return dx * dx + dy * dy >= R * R


def pipe_links(solid, R):
    """Per direction i: (mask of fluid cells whose neighbour x + c_i is solid,
    q at those cells, mask of those whose x - c_i is fluid)."""
    nz, ny, nx = solid.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    dx, dy = x - 0.5 * (nx - 1), y - 0.5 * (ny - 1)
    out = []
    for i in range(Q):
        cx, cy, cz = (int(v) for v in C[i])
        nb_solid = np.roll(solid, shift=(-cz, -cy, -cx), axis=(0, 1, 2))   # solid[x + c_i]
        up_fluid = ~np.roll(solid, shift=(cz, cy, cx), axis=(0, 1, 2))     # fluid at x - c_i
        m = ~solid & nb_solid
        a = float(cx * cx + cy * cy)
        q = np.zeros(solid.shape)
        if a > 0 and np.any(m):
            b = cx * dx[m] + cy * dy[m]
            c0 = dx[m] ** 2 + dy[m] ** 2 - R * R
            q[m] = (-b + np.sqrt(b * b - a * c0)) / a
        out.append((m, q, up_fluid))
    return out


def step_pipe(f, solid, links, tau, F=(0.0, 0.0, 0.0)):
    """One step of the post-collision state with the pipe wall: pull
    streaming, the bounced populations at the wall links, then the collision
    of the fluid cells (the body force acts on fluid cells; solid cells keep
    their values and are never read)."""
    g = stream(f)
    for i, (m, q, up) in enumerate(links):
        if not np.any(m):
            continue
        j = OPP[i]
        lo = m & (q < 0.5)
        hi = m & (q >= 0.5)
        v = g[j].copy()
        lin = lo & up
        v[lin] = 2 * q[lin] * f[i][lin] + (1 - 2 * q[lin]) * g[i][lin]
        half = lo & ~up
        v[half] = f[i][half]
        v[hi] = f[i][hi] / (2 * q[hi]) + (2 * q[hi] - 1) / (2 * q[hi]) * f[j][hi]
        g[j] = v
    fluid = ~solid
    out = f.copy()
    out[:, fluid] = collide(g[:, fluid], tau, F)
    return out
