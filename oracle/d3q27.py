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
