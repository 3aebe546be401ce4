"""C-ABI behaviour on the GPU: error statuses, watchdog, capacities,
profiling counters. Failures are made on the host (a NaN written into the
uploaded populations, a too-small capacity); nothing faults the GPU."""
import numpy as np
import pytest

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


def test_watchdog_reports_nan(lbm):
    n = 12
    L = lbm.Lattice(n, n, n, 0.6, storage=lbm.F32)
    f = np.tile(np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)[:, None], (1, n ** 3))
    f[5, 100] = np.nan
    L.set_populations(f)
    L.step(3)
    with pytest.raises(lbm.LbmError) as e:
        L.stats()
    assert e.value.status == lbm.LBM_EUNSTABLE
    with pytest.raises(lbm.LbmError) as e:
        L.step(1)
    assert e.value.status == lbm.LBM_ESTATE
    L.close()


def test_bc_fixed_by_first_step(lbm):
    L = lbm.Lattice(16, 16, 8, 0.6)
    L.set_pipe(6.0)
    L.step(2, lbm.BC_IBB)
    with pytest.raises(lbm.LbmError) as e:
        L.step(1, lbm.BC_IBM_B)
    assert e.value.status == lbm.LBM_ESTATE
    with pytest.raises(lbm.LbmError) as e:
        L.set_pipe(5.0)
    assert e.value.status == lbm.LBM_ESTATE
    L.close()


def test_link_capacity_overflow_is_reported(lbm):
    L = lbm.Lattice(24, 24, 4, 0.6, max_links=100)
    with pytest.raises(lbm.LbmError) as e:
        L.set_pipe(10.0)
    assert e.value.status == lbm.LBM_ENOMEM
    L.close()


def test_invalid_arguments(lbm):
    L = lbm.Lattice(16, 16, 16, 0.6, max_particles=1)
    with pytest.raises(lbm.LbmError) as e:
        L.add_spheres(np.array([[3.0, 3.0, 3.0], [8.0, 8, 8]]), 2.0)
    assert e.value.status == lbm.LBM_ENOMEM
    with pytest.raises(lbm.LbmError) as e:
        L.add_spheres(np.array([[30.0, 3.0, 3.0]]), 2.0)
    assert e.value.status == lbm.LBM_EINVAL
    L.close()


def test_profile_counts_launches_and_times(lbm):
    L = lbm.Lattice(40, 40, 16, 0.6, storage=lbm.F32)
    L.init_velocity(workloads.pipe_velocity(40, 40, 16, 17.0, 0.02, 0.05, seed=0))
    L.set_pipe(17.0)
    L.profile_enable(True)
    L.step(2, lbm.BC_IBB)
    p = L.profile(0)
    # a static wall without single-node links runs its interpolated
    # bounce-back inside the sweep: one pass forms the wall's partial values
    # from the initial populations, later sweeps leave them for the next step
    assert p["launches"]["bulk"] == 2 and p["launches"]["ibb_boundary"] == 1
    L.profile_enable(True)
    L.step(10, lbm.BC_IBB)
    p = L.profile(0)
    assert p["launches"]["bulk"] == 10 and p["launches"]["ibb_boundary"] == 0
    assert p["spans"]["bulk"] == 10 and p["ms"]["bulk"] > 0
    # profile again after re-enabling: events are reused, destroy frees each once
    L.profile_enable(True)
    L.step(5, lbm.BC_IBB)
    p = L.profile(0)
    assert p["spans"]["bulk"] == 5
    L.close()
    # moving spheres: link pass with momentum exchange
    S = lbm.Lattice(24, 24, 24, 0.6, storage=lbm.F32, max_particles=1)
    S.init_velocity(np.zeros((3, 24, 24, 24)))
    S.add_spheres(np.array([[11.5, 12.0, 12.5]]), 4.0)
    S.step(1, lbm.BC_IBB)
    S.profile_enable(True)
    S.step(4, lbm.BC_IBB)
    p = S.profile(0)
    # moving walls: the link pass and the single-node pass each step
    assert p["launches"]["bulk"] == 4 and p["launches"]["ibb_boundary"] == 8
    S.close()


def test_wait_limit_runs_out_and_context_stays_usable(lbm):
    """LBM_ETIMEOUT from the bounded host wait: a host function that sleeps
    1.5 s is enqueued on the library's stream ahead of the status check, and
    the wait limit is set to 0.2 s. Nothing waits on the GPU: the stream is
    held on the host. A later call with a longer limit succeeds."""
    import ctypes
    import time

    n = 16
    L = lbm.Lattice(n, n, n, 0.6, storage=lbm.F32)
    L.step(2)
    L.stats()  # nothing pending
    # the CUDA runtime the library itself loaded (matched by soname)
    cudart = ctypes.CDLL("libcudart.so.13")
    HOSTFN = ctypes.CFUNCTYPE(None, ctypes.c_void_p)
    slept = []

    def hold(_):
        time.sleep(1.5)
        slept.append(1)

    cb = HOSTFN(hold)
    cudart.cudaLaunchHostFunc.argtypes = [ctypes.c_void_p, HOSTFN, ctypes.c_void_p]
    cudart.cudaLaunchHostFunc.restype = ctypes.c_int
    assert cudart.cudaLaunchHostFunc(ctypes.c_void_p(L.stream.cuda_stream), cb, None) == 0
    L.step(1)
    with pytest.raises(lbm.LbmError):
        L.set_wait_limit(0.0)
    L.set_wait_limit(0.2)
    t0 = time.time()
    with pytest.raises(lbm.LbmError) as e:
        L.stats()
    assert e.value.status == lbm.LBM_ETIMEOUT
    assert time.time() - t0 < 1.4 and not slept
    L.set_wait_limit(30.0)
    s = L.stats()
    assert slept and s["step"] == 3
    L.step(1)
    assert L.stats()["step"] == 4
    L.close()
