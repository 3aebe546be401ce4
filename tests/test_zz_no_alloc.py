"""The allocation-free energy/dissipation entry point, for callers that
cannot call cudaMalloc (stream capture, externally owned device memory,
loops that must not synchronise): it must give what lbm_stats gives for the
same unmasked field, on consecutive calls that share its fixed scratch."""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_noalloc_energy_matches_stats_twice():
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
        lat = lbm.Lattice(n, n + 3, n - 5, tau, storage=lbm.F64)
        u0 = workloads.hit_velocity(48, seed=seed, k_peak=4.0, u_rms=0.02)[:, : n - 5, : n + 3, :n]
        lat.init_velocity(np.ascontiguousarray(u0))
        lat.step(5)
        ref = lat.stats(0)
        _, u = lat.macro()
        u_dev = torch.from_numpy(np.ascontiguousarray(u)).cuda()
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        for _ in range(2):
            rc = L.lbm_field_energy_noalloc(ctypes.c_void_p(u_dev.data_ptr()), n, n + 3, n - 5, nu,
                                            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
            assert rc == lbm.LBM_OK
            torch.cuda.synchronize()
            k, e = out.cpu().numpy()
            assert k == pytest.approx(ref["kinetic_energy"], rel=1e-12)
            assert e == pytest.approx(ref["dissipation"], rel=1e-12)
            out.fill_(float("nan"))
        lat.close()
    too_big = L.lbm_field_energy_noalloc(ctypes.c_void_p(u_dev.data_ptr()), 1024, 1024, 1024, nu,
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert too_big == lbm.LBM_ENOMEM
