"""The allocation-free energy/dissipation entry point, for callers that
cannot call cudaMalloc (solvers whose device memory all belongs to another
framework's pool, loops that must not pay cudaMalloc's implicit
synchronisation). On two consecutive calls, which share its fixed scratch
array, it must give what the existing statistics entry point (lbm_stats)
gives for the same unmasked field, and what the oracle's statistics give for
the oracle's own field."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _call(L, lbm, torch, u, n3, nu, stream):
    nx, ny, nz = n3
    u_dev = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float64)).cuda()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    res = []
    for _ in range(2):
        rc = L.lbm_field_energy_noalloc(ctypes.c_void_p(u_dev.data_ptr()), nx, ny, nz, nu,
                                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == lbm.LBM_OK
        torch.cuda.synchronize()
        res.append(out.cpu().numpy().copy())
        out.fill_(float("nan"))
    return res, u_dev, out


def test_noalloc_energy_matches_stats_and_oracle_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_05448_gb300 import build, lbm
    build.build()
    L = lbm.load()
    assert L.lbm_field_energy_noalloc_max_cells() == 512 ** 3
    tau = 0.6
    nu = (tau - 0.5) / 3.0
    stream = torch.cuda.current_stream()
    for n, seed in ((40, 1), (24, 2)):
        n3 = (n, n + 3, n - 5)
        u0 = np.ascontiguousarray(workloads.hit_velocity(48, seed=seed, k_peak=4.0, u_rms=0.02)[:, : n - 5, : n + 3, :n])
        # against the existing entry point, on the GPU context's own field
        lat = lbm.Lattice(*n3, tau, storage=lbm.F64)
        lat.init_velocity(u0)
        lat.step(5)
        ref = lat.stats(0)
        _, u = lat.macro()
        res, u_dev, out = _call(L, lbm, torch, u, n3, nu, stream)
        for k, e in res:
            assert k == pytest.approx(ref["kinetic_energy"], rel=1e-12)
            assert e == pytest.approx(ref["dissipation"], rel=1e-12)
        lat.close()
        # against the oracle, on the oracle's field
        o = oracle.Sim(*n3, tau)
        o.init_velocity(u0)
        o.step(5)
        so = o.stats(0)
        _, uo = o.macro()
        res, _, _ = _call(L, lbm, torch, uo.reshape(3, -1), n3, nu, stream)
        for k, e in res:
            assert k == pytest.approx(so["kinetic_energy"], rel=1e-12)
            assert e == pytest.approx(so["dissipation"], rel=1e-12)
    too_big = L.lbm_field_energy_noalloc(ctypes.c_void_p(u_dev.data_ptr()), 1024, 1024, 1024, nu,
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert too_big == lbm.LBM_ENOMEM
