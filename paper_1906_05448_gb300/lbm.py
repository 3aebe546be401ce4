"""Thin ctypes binding of the C ABI in include/lbm.h (argument marshalling only).

Every step of the method runs in the CUDA library liblbm_gb300.so; this
module only converts numpy arrays to pointers, allocates the device
workspace as a torch uint8 tensor and passes torch's current CUDA stream.
There is no CPU fallback: importing without the built library, or creating a
context without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ESTATE, LBM_EUNSUPPORTED, LBM_EIO = range(9)
BC_NONE, BC_IBB, BC_IBM_U, BC_IBM_B = 0, 1, 2, 3
F64, F32, F16S, BF16S = 0, 1, 2, 3
RATES_SRT, RATES_DHUMIERES = 0, 1
STATS_UNMASK, STATS_BINS, STATS_CLOSURE = 1, 4, 8
FIELD_RHO, FIELD_U, FIELD_POPS, FIELD_FLAGS, FIELD_IBM_FORCE = 0, 1, 2, 3, 4
NBINS = 40

STORAGE = {"f64": F64, "f32": F32, "f16s": F16S, "bf16s": BF16S}
BC = {"none": BC_NONE, "ibb": BC_IBB, "ibm_u": BC_IBM_U, "ibm_b": BC_IBM_B}

# every entry point declared in include/lbm.h
EXPORTS = [
    "lbm_workspace_bytes", "lbm_create", "lbm_init_velocity", "lbm_set_populations", "lbm_set_pipe",
    "lbm_add_spheres", "lbm_step", "lbm_set_wait_limit", "lbm_checkpoint", "lbm_restore", "lbm_stats", "lbm_spectrum", "lbm_pipe_profiles", "lbm_tke_budget", "lbm_set_mrt_rates", "lbm_get_field", "lbm_num_links", "lbm_get_links",
    "lbm_get_particles", "lbm_num_particles", "lbm_num_markers", "lbm_get_markers", "lbm_profile",
    "lbm_mlp_workspace_bytes", "lbm_mlp_num_params", "lbm_mlp_forward", "lbm_mlp_loss_grad", "lbm_mlp_train",
    "lbm_closure_samples", "lbm_closure_targets", "lbm_closure_set_weights",
    "lbm_field_energy_noalloc", "lbm_field_energy_noalloc_max_cells", "lbm_last_error",
    "lbm_status_string", "lbm_destroy",
]
NGROUPS = 9
GROUPS = ["bulk", "ibb_boundary", "ibm_passes", "ibm_collide", "particles", "geometry", "stats", "other", "closure"]


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("storage", ctypes.c_int),
                ("rates", ctypes.c_int), ("max_particles", ctypes.c_int), ("max_links", ctypes.c_longlong),
                ("max_markers", ctypes.c_longlong), ("max_sites", ctypes.c_longlong), ("lattice", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double), ("momentum", ctypes.c_double * 3),
        ("kinetic_energy", ctypes.c_double), ("dissipation", ctypes.c_double),
        ("kinetic_energy_fluid", ctypes.c_double), ("dissipation_fluid", ctypes.c_double),
        ("particle_ke", ctypes.c_double), ("particle_ake", ctypes.c_double),
        ("force", ctypes.c_double * 3), ("torque", ctypes.c_double * 3),
        ("bulk_velocity", ctypes.c_double), ("nbins", ctypes.c_int),
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


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * NGROUPS), ("spans", ctypes.c_longlong * NGROUPS),
                ("launches", ctypes.c_longlong * NGROUPS), ("total_launches", ctypes.c_longlong)]


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_L = ctypes.POINTER(ctypes.c_longlong)
_P = ctypes.c_void_p
_lib = None


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lbm status {status}: {msg}")
        self.status = status


def library_path() -> str:
    return _build.SO


def load(build_if_missing: bool = False):
    """Load liblbm_gb300.so. Raises if it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.SO
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
        _build.build()
    L = ctypes.CDLL(path)
    sig = {
        "lbm_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(Grid)]),
        "lbm_create": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_double, _D, _P, ctypes.c_size_t, _P,
                                      ctypes.POINTER(_P)]),
        "lbm_init_velocity": (ctypes.c_int, [_P, _D, ctypes.c_double]),
        "lbm_set_populations": (ctypes.c_int, [_P, _D]),
        "lbm_set_pipe": (ctypes.c_int, [_P, ctypes.c_double]),
        "lbm_add_spheres": (ctypes.c_int, [_P, ctypes.c_int, _D, _D, ctypes.c_double, _D, _D, ctypes.c_int]),
        "lbm_step": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
        "lbm_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_double]),
        "lbm_checkpoint": (ctypes.c_int, [_P, ctypes.c_char_p]),
        "lbm_restore": (ctypes.c_int, [_P, ctypes.c_char_p]),
        "lbm_stats": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(Stats)]),
        "lbm_spectrum": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _D, _D]),
        "lbm_pipe_profiles": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _D]),
        "lbm_tke_budget": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _D]),
        "lbm_set_mrt_rates": (ctypes.c_int, [_P] + [ctypes.c_double] * 5),
        "lbm_get_field": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t]),
        "lbm_num_links": (ctypes.c_int, [_P, _L]),
        "lbm_get_links": (ctypes.c_int, [_P, ctypes.c_longlong, _L, _I, _I, _D, _I]),
        "lbm_get_particles": (ctypes.c_int, [_P, _D, _D, _D, _D, _D]),
        "lbm_num_particles": (ctypes.c_int, [_P, _I]),
        "lbm_num_markers": (ctypes.c_int, [_P, _L]),
        "lbm_get_markers": (ctypes.c_int, [_P, ctypes.c_longlong, _D, _D, _D, _I]),
        "lbm_profile": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(Profile)]),
        "lbm_mlp_workspace_bytes": (ctypes.c_size_t, []),
        "lbm_mlp_num_params": (ctypes.c_int, []),
        "lbm_mlp_forward": (ctypes.c_int, [_P, ctypes.c_longlong, _P, _P, _P, ctypes.c_size_t, _P]),
        "lbm_mlp_loss_grad": (ctypes.c_int, [_P, _P, ctypes.c_longlong, _P, _P, _D, _P, ctypes.c_size_t, _P]),
        "lbm_mlp_train": (ctypes.c_int, [_P, _P, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_double, _P,
                                         _P, ctypes.c_size_t, _P, _D]),
        "lbm_closure_samples": (ctypes.c_int, [_P, ctypes.c_double, _P, _P, ctypes.c_longlong, _L]),
        "lbm_closure_targets": (ctypes.c_int, [_P, _P, ctypes.c_longlong, ctypes.c_double, _P]),
        "lbm_closure_set_weights": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
        "lbm_field_energy_noalloc": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                    _P, _P]),
        "lbm_field_energy_noalloc_max_cells": (ctypes.c_longlong, []),
        "lbm_last_error": (ctypes.c_char_p, [_P]),
        "lbm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "lbm_destroy": (None, [_P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_grid(nx, ny, nz, storage=F32, rates=RATES_SRT, max_particles=0, max_links=0, max_markers=0,
              max_sites=0, lattice=19) -> Grid:
    if isinstance(storage, str):
        storage = STORAGE[storage]
    return Grid(nx, ny, nz, storage, rates, max_particles, max_links, max_markers, max_sites, lattice)


def workspace_bytes(grid: Grid) -> int:
    return int(load().lbm_workspace_bytes(ctypes.byref(grid)))


class Lattice:
    """One simulation context (lbm_create ... lbm_destroy)."""

    def __init__(self, nx, ny, nz, tau, force=(0.0, 0.0, 0.0), storage=F32, rates=RATES_SRT,
                 max_particles=0, max_links=0, max_markers=0, max_sites=0, device=None, stream=None, lattice=19):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the library has no CPU path")
        self.L = load()
        self.grid = make_grid(nx, ny, nz, storage, rates, max_particles, max_links, max_markers, max_sites, lattice)
        self.q = 27 if lattice == 27 else 19
        self.N = nx * ny * nz
        self.shape = (nz, ny, nx)
        nbytes = workspace_bytes(self.grid)
        if nbytes == 0:
            raise ValueError("invalid grid")
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        F = _c64(force)
        h = _P()
        rc = self.L.lbm_create(ctypes.byref(self.grid), float(tau), _dp(F), ctypes.c_void_p(self.workspace.data_ptr()),
                               nbytes, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != LBM_OK:
            raise LbmError(rc, self.L.lbm_status_string(rc).decode())
        self.h = h

    # -- helpers
    def _check(self, rc, allow=()):
        if rc != LBM_OK and rc not in allow:
            raise LbmError(rc, self.L.lbm_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.L.lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- API
    def init_velocity(self, u, rho0=1.0):
        u = _c64(u).reshape(3 * self.N)
        self._check(self.L.lbm_init_velocity(self.h, _dp(u), float(rho0)))

    def set_populations(self, f):
        f = _c64(f).reshape(self.q * self.N)
        self._check(self.L.lbm_set_populations(self.h, _dp(f)))

    def set_pipe(self, radius):
        self._check(self.L.lbm_set_pipe(self.h, float(radius)))

    def add_spheres(self, X, R, density_ratio=1.0, U=None, W=None, fixed=False):
        X = _c64(X).reshape(-1, 3)
        n = X.shape[0]
        R = _c64(np.broadcast_to(np.asarray(R, dtype=np.float64), (n,)))
        Ua = None if U is None else _c64(U).reshape(n, 3)
        Wa = None if W is None else _c64(W).reshape(n, 3)
        self._check(self.L.lbm_add_spheres(self.h, n, _dp(X), _dp(R), float(density_ratio), _dp(Ua), _dp(Wa),
                                           int(bool(fixed))))
        self.np = n

    def step(self, n, bc=BC_NONE):
        if isinstance(bc, str):
            bc = BC[bc]
        return self._check(self.L.lbm_step(self.h, int(n), int(bc)))

    def set_wait_limit(self, seconds):
        """Bound of the host waits on the stream (LBM_ETIMEOUT when it runs out)."""
        self._check(self.L.lbm_set_wait_limit(self.h, float(seconds)))

    def checkpoint(self, path):
        self._check(self.L.lbm_checkpoint(self.h, os.fsencode(path)))

    def restore(self, path):
        """Load a checkpoint into this freshly created context (same grid, tau, force)."""
        self._check(self.L.lbm_restore(self.h, os.fsencode(path)))
        n = ctypes.c_int()
        self._check(self.L.lbm_num_particles(self.h, ctypes.byref(n)))
        self.np = n.value

    def spectrum(self, nbins, flags=0):
        """3D kinetic-energy and dissipation spectra E[K], D[K], K < nbins."""
        E = np.zeros(int(nbins))
        D = np.zeros(int(nbins))
        self._check(self.L.lbm_spectrum(self.h, int(flags), int(nbins), _dp(E), _dp(D)))
        return E, D

    def pipe_profiles(self, nbins, flags=0):
        """Radial profiles of the pipe, shape (nbins, 12): count, then the means
        of u_r, u_t, u_z, u_r^2, u_t^2, u_z^2, u_r u_z, u_r u_t, u_t u_z, rho, eps."""
        out = np.zeros((int(nbins), 12))
        self._check(self.L.lbm_pipe_profiles(self.h, int(flags), int(nbins), _dp(out)))
        return out

    def set_mrt_rates(self, s_e, s_eps, s_q, s_pi, s_m):
        """Non-shear MRT rates by group (e, eps, q, pi, m); shear stays 1/tau."""
        self._check(self.L.lbm_set_mrt_rates(self.h, float(s_e), float(s_eps), float(s_q), float(s_pi), float(s_m)))

    def tke_budget(self, nbins, flags=0):
        """Component-wise TKE budget of the pipe, shape (nbins, 14): count, then
        E_Oz, E_Tz, E_Pz, E_Vz, E_Dz, E_Tr, E_Pr, E_Vr, E_Dr, E_Tt, E_Pt, E_Vt, E_Dt."""
        out = np.zeros((int(nbins), 14))
        self._check(self.L.lbm_tke_budget(self.h, int(flags), int(nbins), _dp(out)))
        return out

    def stats(self, flags=0) -> dict:
        s = Stats()
        self._check(self.L.lbm_stats(self.h, int(flags), ctypes.byref(s)))
        return s.as_dict()

    def _field(self, which, n, dtype):
        out = np.empty(n, dtype=dtype)
        self._check(self.L.lbm_get_field(self.h, which, out.ctypes.data_as(_P), out.nbytes))
        return out

    def macro(self):
        rho = self._field(FIELD_RHO, self.N, np.float64)
        u = self._field(FIELD_U, 3 * self.N, np.float64).reshape(3, self.N)
        return rho, u

    def populations(self):
        return self._field(FIELD_POPS, self.q * self.N, np.float64).reshape(self.q, self.N)

    def flags(self):
        return self._field(FIELD_FLAGS, self.N, np.uint8)

    def ibm_force(self):
        return self._field(FIELD_IBM_FORCE, 3 * self.N, np.float64).reshape(3, self.N)

    def links(self) -> dict:
        n = ctypes.c_longlong()
        self._check(self.L.lbm_num_links(self.h, ctypes.byref(n)))
        n = n.value
        cell = np.zeros(n, dtype=np.int64)
        d = np.zeros(n, dtype=np.int32)
        sc = np.zeros(n, dtype=np.int32)
        q = np.zeros(n)
        pid = np.zeros(n, dtype=np.int32)
        if n:
            self._check(self.L.lbm_get_links(self.h, n, cell.ctypes.data_as(_L), d.ctypes.data_as(_I),
                                             sc.ctypes.data_as(_I), _dp(q), pid.ctypes.data_as(_I)))
        return dict(cell=cell, dir=d, scheme=sc, q=q, pid=pid)

    def particles(self) -> dict:
        n = getattr(self, "np", 0)
        arr = {k: np.zeros((n, 3)) for k in ("X", "U", "W", "F", "T")}
        if n:
            self._check(self.L.lbm_get_particles(self.h, *[_dp(arr[k]) for k in ("X", "U", "W", "F", "T")]))
        return arr

    def profile(self, enable=-1) -> dict:
        """Totals per kernel group since profiling was enabled; enable=1/0 switches it."""
        p = Profile()
        self._check(self.L.lbm_profile(self.h, int(enable), ctypes.byref(p)))
        return dict(ms={g: p.ms[i] for i, g in enumerate(GROUPS)},
                    spans={g: p.spans[i] for i, g in enumerate(GROUPS)},
                    launches={g: p.launches[i] for i, g in enumerate(GROUPS)},
                    total_launches=p.total_launches)

    def profile_enable(self, on=True):
        self._check(self.L.lbm_profile(self.h, 1 if on else 0, None))

    # -- learned closure
    def closure_samples(self, u_scale, capacity):
        """Features (n, 85) and cells (n,) of the near-surface nodes, as torch
        CUDA tensors (rows in no fixed order)."""
        import torch
        X = torch.empty((capacity, 85), dtype=torch.float32, device=self.workspace.device)
        cells = torch.empty(capacity, dtype=torch.int32, device=self.workspace.device)
        n = ctypes.c_longlong()
        self._check(self.L.lbm_closure_samples(self.h, float(u_scale), ctypes.c_void_p(X.data_ptr()),
                                               ctypes.c_void_p(cells.data_ptr()), capacity, ctypes.byref(n)))
        return X[: n.value], cells[: n.value]

    def closure_targets(self, cells, g_scale):
        import torch
        cells = cells.contiguous()
        T = torch.empty((cells.numel(), 9), dtype=torch.float32, device=self.workspace.device)
        self._check(self.L.lbm_closure_targets(self.h, ctypes.c_void_p(cells.data_ptr()), cells.numel(),
                                               float(g_scale), ctypes.c_void_p(T.data_ptr())))
        return T

    def closure_set_weights(self, w, u_scale, g_scale):
        w = np.ascontiguousarray(w, dtype=np.float32)
        self._check(self.L.lbm_closure_set_weights(self.h, w.ctypes.data_as(_P), w.size, float(u_scale),
                                                   float(g_scale)))

    def markers(self) -> dict:
        n = ctypes.c_longlong()
        self._check(self.L.lbm_num_markers(self.h, ctypes.byref(n)))
        n = n.value
        X = np.zeros((n, 3))
        F = np.zeros((n, 3))
        dV = np.zeros(n)
        pid = np.zeros(n, dtype=np.int32)
        if n:
            self._check(self.L.lbm_get_markers(self.h, n, _dp(X), _dp(F), _dp(dV), pid.ctypes.data_as(_I)))
        return dict(X=X, F=F, dV=dV, pid=pid)


# ------------------------------------------------------------- perceptron ---
class MLP:
    """Device workspace for the lbm_mlp_* entry points (torch CUDA tensors in,
    torch CUDA tensors out)."""

    def __init__(self, device=None):
        import torch
        self.L = load()
        self.dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.nbytes = int(self.L.lbm_mlp_workspace_bytes())
        self.ws = torch.empty(self.nbytes, dtype=torch.uint8, device=self.dev)
        self.nparam = int(self.L.lbm_mlp_num_params())

    def _s(self):
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream(self.dev).cuda_stream)

    def _w(self, w):
        import torch
        if not isinstance(w, torch.Tensor):
            w = torch.as_tensor(np.asarray(w, dtype=np.float32))
        return w.to(self.dev, torch.float32).contiguous()

    def forward(self, X, w):
        import torch
        X = X.to(self.dev, torch.float32).contiguous()
        w = self._w(w)
        Y = torch.empty((X.shape[0], 9), dtype=torch.float32, device=self.dev)
        rc = self.L.lbm_mlp_forward(ctypes.c_void_p(X.data_ptr()), X.shape[0], ctypes.c_void_p(w.data_ptr()),
                                    ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(self.ws.data_ptr()), self.nbytes,
                                    self._s())
        if rc != LBM_OK:
            raise LbmError(rc, "lbm_mlp_forward")
        return Y

    def loss_grad(self, X, T, w):
        import torch
        X = X.to(self.dev, torch.float32).contiguous()
        T = T.to(self.dev, torch.float32).contiguous()
        w = self._w(w)
        g = torch.empty(self.nparam, dtype=torch.float32, device=self.dev)
        loss = ctypes.c_double()
        rc = self.L.lbm_mlp_loss_grad(ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()), X.shape[0],
                                      ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                      ctypes.byref(loss), ctypes.c_void_p(self.ws.data_ptr()), self.nbytes, self._s())
        if rc != LBM_OK:
            raise LbmError(rc, "lbm_mlp_loss_grad")
        return loss.value, g

    def train(self, X, T, w, epochs, batch=4096, lr=1e-3):
        """Returns (trained weights tensor, mean loss of the last epoch)."""
        import torch
        X = X.to(self.dev, torch.float32).contiguous()
        T = T.to(self.dev, torch.float32).contiguous()
        w = self._w(w).clone()
        last = ctypes.c_double()
        rc = self.L.lbm_mlp_train(ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()), X.shape[0],
                                  int(epochs), int(batch), float(lr), ctypes.c_void_p(w.data_ptr()),
                                  ctypes.c_void_p(self.ws.data_ptr()), self.nbytes, self._s(), ctypes.byref(last))
        if rc != LBM_OK:
            raise LbmError(rc, "lbm_mlp_train")
        return w, last.value
