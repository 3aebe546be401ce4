"""Pipe radial profiles on the GPU against the numpy oracle of
oracle/profiles.py applied to the oracle's own state (statistics velocity,
density, solid flags), bin by bin: bit-equal cell counts, and means within
1e-10 of the largest mean of each quantity (FP64 storage)."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import profiles

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


def compare(g, o):
    assert np.array_equal(g[:, 0], o[:, 0])
    for k in range(1, profiles.NQ):
        scale = max(np.max(np.abs(o[:, k])), 1e-300)
        assert np.max(np.abs(g[:, k] - o[:, k])) <= 1e-10 * scale, k


@pytest.mark.parametrize("bc,flags", [("ibb", 0), ("ibm_b", 0), ("ibm_b", 1)])
def test_pipe_profiles_match_oracle(lbm, bc, flags):
    nx, ny, nz, R, nb, tau = 40, 40, 6, 17.0, 12, 0.6
    force = (0, 0, 2e-6)
    g = lbm.Lattice(nx, ny, nz, tau, force=force, storage=lbm.F64)
    o = oracle.Sim(nx, ny, nz, tau, force=force)
    u = workloads.pipe_velocity(nx, ny, nz, R, 0.02, perturbation=0.1, seed=3)
    for s in (g, o):
        s.init_velocity(u)
        s.set_pipe(R)
    obc = {"ibb": oracle.BC_IBB, "ibm_b": oracle.BC_IBM_B}[bc]
    g.step(30, lbm.BC[bc])
    o.step(30, obc)
    prof_g = g.pipe_profiles(nb, flags)
    rho, _ = o.macro()
    prof_o = profiles.pipe_profiles(o.masked_velocity(flags), rho, o.solid()[0], nx, ny, nz,
                                    0.5 * (nx - 1), 0.5 * (ny - 1), R, (tau - 0.5) / 3, nb)
    compare(prof_g, prof_o)
    assert prof_g[:, 3][prof_g[:, 0] > 0].max() > 0  # a flow along the axis


def test_profiles_need_a_pipe(lbm):
    g = lbm.Lattice(16, 16, 16, 0.6, storage=lbm.F32)
    g.init_velocity(np.zeros((3, 16, 16, 16)))
    with pytest.raises(lbm.LbmError):
        g.pipe_profiles(4)
    g.close()
