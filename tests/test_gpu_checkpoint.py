"""Checkpoint and restart through the C ABI (lbm_checkpoint / lbm_restore;
the paper restarts its IBM-U pipe run from the IBM-B field, Sec. 2.2).

N steps in one context must equal N/2 steps, a checkpoint, a restore into a
fresh context and N/2 more steps: bit for bit where the step is
deterministic (every path but the sphere IBM spreading, which sums with FP64
atomics in no fixed order; there the bar is the run-to-run round-off)."""
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


def _pipe(lbm, storage, bc):
    nx, ny, nz, R = 28, 28, 12, 12.5
    u = workloads.pipe_velocity(nx, ny, nz, R, 0.03, perturbation=0.05, seed=4)

    def make():
        return lbm.Lattice(nx, ny, nz, 0.56, force=(0, 0, 2e-6), storage=storage)

    def setup(L):
        L.init_velocity(u)
        L.set_pipe(R)
    return make, setup, bc


def _spheres(lbm, storage, bc):
    n = 32
    X = workloads.place_spheres((n, n, n), 3, 4.0, 1.5, seed=9)
    u = workloads.hit_velocity(n, seed=5, k_peak=3.0, u_rms=0.01)

    def make():
        return lbm.Lattice(n, n, n, 0.6, storage=storage, rates=lbm.RATES_DHUMIERES, max_particles=3)

    def setup(L):
        L.init_velocity(u)
        L.add_spheres(X, 4.0, density_ratio=2.0)
    return make, setup, bc


CASES = {
    "pipe_ibb_f32": (_pipe, "f32", 1, 0.0),
    "pipe_ibb_bf16s": (_pipe, "bf16s", 1, 0.0),
    "pipe_ibm_b_f32": (_pipe, "f32", 3, 0.0),
    "spheres_ibb_f32": (_spheres, "f32", 1, 0.0),
    "spheres_ibb_f64": (_spheres, "f64", 1, 0.0),
    "spheres_ibm_b_f64": (_spheres, "f64", 3, 1e-11),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_restart_continues_bit_for_bit(lbm, case, tmp_path):
    fn, storage, bc, tol = CASES[case]
    make, setup, bc = fn(lbm, lbm.STORAGE[storage], bc)
    nsteps = 16
    A = make()
    setup(A)
    A.step(nsteps // 2, bc)
    sA_half = A.stats()
    path = str(tmp_path / "state.ckpt")
    A.checkpoint(path)
    A.step(nsteps // 2, bc)
    fA, pA, sA = A.populations(), A.particles(), A.stats()
    A.close()

    B = make()
    B.restore(path)
    sB_half = B.stats()
    for k in ("kinetic_energy", "dissipation", "mass", "step", "nlinks", "nmarkers"):
        assert sB_half[k] == sA_half[k], k
    B.step(nsteps // 2, bc)
    fB, pB, sB = B.populations(), B.particles(), B.stats()
    B.close()
    assert sB["step"] == nsteps
    if tol == 0.0:
        assert np.array_equal(fA, fB, equal_nan=True)
        for k in pA:
            assert np.array_equal(pA[k], pB[k]), k
        assert sA["kinetic_energy"] == sB["kinetic_energy"]
    else:
        fl = np.isfinite(fA)
        assert np.max(np.abs(fA[fl] - fB[fl])) <= tol * np.max(np.abs(fA[fl]))
        for k in pA:
            assert np.allclose(pA[k], pB[k], rtol=0, atol=tol * max(1e-30, np.abs(pA[k]).max())), k


def test_restore_refuses_other_configurations(lbm, tmp_path):
    path = str(tmp_path / "s.ckpt")
    A = lbm.Lattice(16, 16, 8, 0.6, storage=lbm.F32)
    A.set_pipe(6.0)
    A.step(3, lbm.BC_IBB)
    A.checkpoint(path)
    A.close()
    for kw in (dict(nx=16, ny=16, nz=9, tau=0.6, storage=lbm.F32), dict(nx=16, ny=16, nz=8, tau=0.61, storage=lbm.F32),
               dict(nx=16, ny=16, nz=8, tau=0.6, storage=lbm.F64)):
        B = lbm.Lattice(kw["nx"], kw["ny"], kw["nz"], kw["tau"], storage=kw["storage"])
        with pytest.raises(lbm.LbmError) as e:
            B.restore(path)
        assert e.value.status == lbm.LBM_EINVAL
        B.close()
    B = lbm.Lattice(16, 16, 8, 0.6, storage=lbm.F32)
    B.step(1)
    with pytest.raises(lbm.LbmError) as e:
        B.restore(path)
    assert e.value.status == lbm.LBM_ESTATE
    B.close()
    C = lbm.Lattice(16, 16, 8, 0.6, storage=lbm.F32)
    with pytest.raises(lbm.LbmError) as e:
        C.restore(str(tmp_path / "missing.ckpt"))
    assert e.value.status == lbm.LBM_EIO
    with open(path, "r+b") as f:  # truncated file
        f.truncate(200)
    with pytest.raises(lbm.LbmError) as e:
        C.restore(path)
    assert e.value.status == lbm.LBM_EIO
    C.close()
