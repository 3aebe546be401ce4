"""Oracle: plain FP64 CPU implementation of the D3Q19 lattice Boltzmann method
with IBB and IBM no-slip walls (arXiv:1906.05448, Secs. 2.1 and 3.1).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package. It shares no
code with the CUDA library in ``paper_1906_05448_gb300``; it is the slow,
obviously-correct statement the GPU path is checked against. The C source is
``lbm_oracle.c`` (FP64, dense moment matrices, brute-force geometry,
``-ffp-contract=off``); the MLP closure oracle is ``mlp_oracle.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblbm_oracle.so")
_SRC = [os.path.join(_HERE, "lbm_oracle.c")]
_lock = threading.Lock()
_lib = None

BC_NONE, BC_IBB, BC_IBM_U, BC_IBM_B = 0, 1, 2, 3
RATES_SRT, RATES_DHUMIERES = 0, 1
SCHEME_QUAD, SCHEME_LINEAR, SCHEME_SINGLE, SCHEME_HALFWAY = 0, 1, 2, 3
CHAIN_SPHERE, CHAIN_PIPE, CHAIN_SINGLE, CHAIN_HALFWAY = 0, 1, 2, 3
STATS_UNMASK, STATS_BINS = 1, 4
NBINS = 40


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build (gcc, FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRC + [os.path.join(_HERE, "lbm_oracle.h")])
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", "-o", tmp] + _SRC + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class Stats(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double), ("momentum", ctypes.c_double * 3),
        ("kinetic_energy", ctypes.c_double), ("dissipation", ctypes.c_double),
        ("kinetic_energy_fluid", ctypes.c_double), ("dissipation_fluid", ctypes.c_double),
        ("particle_ke", ctypes.c_double), ("particle_ake", ctypes.c_double),
        ("force", ctypes.c_double * 3), ("torque", ctypes.c_double * 3),
        ("bulk_velocity", ctypes.c_double),
        ("nbins", ctypes.c_int),
        ("bin_r", ctypes.c_double * NBINS), ("bin_tke", ctypes.c_double * NBINS),
        ("bin_eps", ctypes.c_double * NBINS), ("bin_count", ctypes.c_longlong * NBINS),
        ("nfluid", ctypes.c_longlong), ("nlinks", ctypes.c_longlong),
        ("nmarkers", ctypes.c_longlong), ("step", ctypes.c_longlong),
    ]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_L = ctypes.POINTER(ctypes.c_longlong)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_P = ctypes.c_void_p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            so = build()
            L = ctypes.CDLL(so)
            sig = {
                "orc_lattice": (None, [_I, _D, _I]),
                "orc_moment_matrix": (None, [_D]),
                "orc_rates": (None, [ctypes.c_int, ctypes.c_double, _D]),
                "orc_feq": (None, [ctypes.c_double, _D, _D]),
                "orc_collide_mrt": (None, [_D, _D, ctypes.c_int, ctypes.c_double, _D]),
                "orc_collide_bgk": (None, [_D, _D, ctypes.c_double, _D]),
                "orc_peskin_phi": (ctypes.c_double, [ctypes.c_double]),
                "orc_solid_fraction": (ctypes.c_double, [_D, _D, ctypes.c_double]),
                "orc_marker_count": (ctypes.c_int, [ctypes.c_double]),
                "orc_sphere_markers": (None, [ctypes.c_double, ctypes.c_int, _D]),
                "orc_create": (_P, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, ctypes.c_int]),
                "orc_destroy": (None, [_P]),
                "orc_set_group_rates": (None, [_P] + [ctypes.c_double] * 5),
                "orc_set_threads": (None, [ctypes.c_int]),
                "orc_get_threads": (ctypes.c_int, []),
                "orc_init_velocity": (None, [_P, _D, ctypes.c_double]),
                "orc_set_populations": (None, [_P, _D]),
                "orc_get_populations": (None, [_P, _D]),
                "orc_set_pipe": (None, [_P, ctypes.c_double]),
                "orc_set_channel": (None, [_P] + [ctypes.c_double] * 4 + [ctypes.c_int]),
                "orc_add_spheres": (ctypes.c_int, [_P, ctypes.c_int, _D, _D, ctypes.c_double, _D, _D, ctypes.c_int]),
                "orc_step": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
                "orc_macro": (None, [_P, _D, _D]),
                "orc_get_solid": (None, [_P, _U8, _I]),
                "orc_num_links": (ctypes.c_longlong, [_P]),
                "orc_get_links": (None, [_P, _L, _I, _I, _D, _I]),
                "orc_num_particles": (ctypes.c_int, [_P]),
                "orc_get_particles": (None, [_P, _D, _D, _D, _D, _D]),
                "orc_num_markers": (ctypes.c_longlong, [_P]),
                "orc_get_markers": (None, [_P, _D, _D, _D, _I]),
                "orc_get_ibm_force": (None, [_P, _D]),
                "orc_stats": (None, [_P, ctypes.c_int, ctypes.POINTER(Stats)]),
                "orc_masked_velocity": (None, [_P, ctypes.c_int, _D]),
                "orc_marker_residual": (ctypes.c_double, [_P, ctypes.c_int]),
                "orc_particles_advance": (None, [_P, ctypes.c_int]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def lattice():
    c = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, dtype=np.int32)
    lib().orc_lattice(c.ctypes.data_as(_I), _dp(w), opp.ctypes.data_as(_I))
    return c, w, opp


def moment_matrix():
    M = np.zeros((19, 19))
    lib().orc_moment_matrix(_dp(M))
    return M


def rates(rate_set: int, tau: float):
    s = np.zeros(19)
    lib().orc_rates(rate_set, tau, _dp(s))
    return s


def feq(rho: float, u) -> np.ndarray:
    out = np.zeros(19)
    lib().orc_feq(rho, _dp(_c64(u)), _dp(out))
    return out


def collide_mrt(f, F, rate_set: int, tau: float) -> np.ndarray:
    out = np.zeros(19)
    lib().orc_collide_mrt(_dp(_c64(f)), _dp(_c64(F)), rate_set, tau, _dp(out))
    return out


def collide_bgk(f, F, tau: float) -> np.ndarray:
    out = np.zeros(19)
    lib().orc_collide_bgk(_dp(_c64(f)), _dp(_c64(F)), tau, _dp(out))
    return out


def peskin_phi(r: float) -> float:
    return lib().orc_peskin_phi(float(r))


def solid_fraction(x, X, R: float) -> float:
    return lib().orc_solid_fraction(_dp(_c64(x)), _dp(_c64(X)), float(R))


def marker_count(RL: float) -> int:
    return lib().orc_marker_count(float(RL))


def sphere_markers(RL: float, n: int) -> np.ndarray:
    out = np.zeros((n, 3))
    lib().orc_sphere_markers(float(RL), n, _dp(out))
    return out


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return lib().orc_get_threads()


class Sim:
    """One oracle simulation (FP64, host memory)."""

    def __init__(self, nx, ny, nz, tau, force=(0.0, 0.0, 0.0), rates=RATES_SRT):
        self.L = lib()
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        F = _c64(force)
        self.h = self.L.orc_create(nx, ny, nz, float(tau), _dp(F), int(rates))
        if not self.h:
            raise MemoryError("oracle allocation failed")

    def close(self):
        if self.h:
            self.L.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_velocity(self, u, rho0=1.0):
        u = _c64(u).reshape(3, self.N)
        self.L.orc_init_velocity(self.h, _dp(u), float(rho0))

    def set_group_rates(self, s_e, s_eps, s_q, s_pi, s_m):
        """Non-shear MRT rates by group (e, eps, q, pi, m); shear stays 1/tau."""
        self.L.orc_set_group_rates(self.h, float(s_e), float(s_eps), float(s_q), float(s_pi), float(s_m))

    def set_populations(self, f):
        f = _c64(f).reshape(19, self.N)
        self.L.orc_set_populations(self.h, _dp(f))

    def populations(self) -> np.ndarray:
        f = np.zeros((19, self.N))
        self.L.orc_get_populations(self.h, _dp(f))
        return f

    def set_pipe(self, radius):
        self.L.orc_set_pipe(self.h, float(radius))

    def set_channel(self, y_lo, y_hi, u_lo=0.0, u_hi=0.0, chain=CHAIN_SPHERE):
        """Plane walls at y = y_lo and y = y_hi moving along x (test geometry
        of the bounce-back schemes; chain selects the schemes of the links)."""
        self.L.orc_set_channel(self.h, float(y_lo), float(y_hi), float(u_lo), float(u_hi), int(chain))

    def add_spheres(self, X, R, density_ratio=1.0, U=None, W=None, fixed=False):
        X = _c64(X).reshape(-1, 3)
        n = X.shape[0]
        R = _c64(np.broadcast_to(np.asarray(R, dtype=np.float64), (n,)))
        Ua = None if U is None else _c64(U).reshape(n, 3)
        Wa = None if W is None else _c64(W).reshape(n, 3)
        rc = self.L.orc_add_spheres(self.h, n, _dp(X), _dp(R), float(density_ratio), _dp(Ua), _dp(Wa), int(bool(fixed)))
        if rc != 0:
            raise ValueError("oracle rejected add_spheres")

    def step(self, n, bc=BC_NONE):
        rc = self.L.orc_step(self.h, int(n), int(bc))
        if rc != 0:
            raise ValueError("oracle: boundary treatment changed after the first step")

    def macro(self):
        rho = np.zeros(self.N)
        u = np.zeros((3, self.N))
        self.L.orc_macro(self.h, _dp(rho), _dp(u))
        return rho, u

    def solid(self):
        s = np.zeros(self.N, dtype=np.uint8)
        o = np.zeros(self.N, dtype=np.int32)
        self.L.orc_get_solid(self.h, s.ctypes.data_as(_U8), o.ctypes.data_as(_I))
        return s, o

    def links(self) -> dict:
        n = self.L.orc_num_links(self.h)
        cell = np.zeros(n, dtype=np.int64)
        d = np.zeros(n, dtype=np.int32)
        sc = np.zeros(n, dtype=np.int32)
        q = np.zeros(n)
        pid = np.zeros(n, dtype=np.int32)
        if n:
            self.L.orc_get_links(self.h, cell.ctypes.data_as(_L), d.ctypes.data_as(_I), sc.ctypes.data_as(_I),
                                 _dp(q), pid.ctypes.data_as(_I))
        return dict(cell=cell, dir=d, scheme=sc, q=q, pid=pid)

    def particles(self) -> dict:
        n = self.L.orc_num_particles(self.h)
        arr = {k: np.zeros((n, 3)) for k in ("X", "U", "W", "F", "T")}
        if n:
            self.L.orc_get_particles(self.h, *[_dp(arr[k]) for k in ("X", "U", "W", "F", "T")])
        return arr

    def markers(self) -> dict:
        n = self.L.orc_num_markers(self.h)
        X = np.zeros((n, 3))
        F = np.zeros((n, 3))
        dV = np.zeros(n)
        pid = np.zeros(n, dtype=np.int32)
        if n:
            self.L.orc_get_markers(self.h, _dp(X), _dp(F), _dp(dV), pid.ctypes.data_as(_I))
        return dict(X=X, F=F, dV=dV, pid=pid)

    def ibm_force(self) -> np.ndarray:
        F = np.zeros((3, self.N))
        self.L.orc_get_ibm_force(self.h, _dp(F))
        return F

    def particles_advance(self, n: int) -> None:
        self.L.orc_particles_advance(self.h, int(n))

    def marker_residual(self, p: int) -> float:
        return self.L.orc_marker_residual(self.h, int(p))

    def masked_velocity(self, flags=0):
        """Velocity field of the statistics, shape (3, N)."""
        u = np.zeros((3, self.N))
        self.L.orc_masked_velocity(self.h, int(flags), _dp(u))
        return u

    def stats(self, flags=0) -> dict:
        s = Stats()
        self.L.orc_stats(self.h, int(flags), ctypes.byref(s))
        return s.as_dict()
