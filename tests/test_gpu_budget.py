"""GPU component-wise TKE budget of the pipe (lbm_tke_budget, Eq. 1a-c) vs
the oracle (oracle/tke_budget.py) on the same FP64 state after 30 steps.

The state itself agrees to about 1e-12; the budget takes fluctuations about
bin means and their products, with the bin sums added in another order, so
each term is held to 1e-7 of its largest magnitude over the bins (the
pressure fluctuation c_s^2 rho' loses about five digits to the cancellation
rho - <rho>); the cell counts agree exactly.
"""
import numpy as np
import pytest

import oracle
import workloads
from oracle import tke_budget as tb

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


@pytest.mark.parametrize("bc,flags", [("ibb", 0), ("ibm_b", 0), ("ibm_b", 1)])
def test_tke_budget_matches_oracle(lbm, bc, flags):
    nx, ny, nz, R, nb, tau = 40, 40, 12, 17.0, 12, 0.6
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
    bud_g = g.tke_budget(nb, flags)
    rho, _ = o.macro()
    bud_o = tb.tke_budget(o.masked_velocity(flags), rho, o.solid()[0], nx, ny, nz,
                          0.5 * (nx - 1), 0.5 * (ny - 1), R, (tau - 0.5) / 3, nb)
    assert np.array_equal(bud_g[:, 0], bud_o[:, 0])
    for k in range(1, tb.NT):
        scale = max(np.max(np.abs(bud_o[:, k])), 1e-300)
        assert np.max(np.abs(bud_g[:, k] - bud_o[:, k])) <= 1e-7 * scale, tb.NAMES[k]
    # a developing flow: production, transport and dissipation are present
    assert np.max(np.abs(bud_o[:, tb.NAMES.index("E_Dz")])) > 0
    assert np.max(np.abs(bud_o[:, tb.NAMES.index("E_Oz")])) > 0
    g.close()


def test_tke_budget_arguments(lbm):
    g = lbm.Lattice(16, 16, 8, 0.6, storage=lbm.F32)
    g.init_velocity(np.zeros((3, 8, 16, 16)))
    with pytest.raises(lbm.LbmError):
        g.tke_budget(4)  # no pipe
    g.close()
    g = lbm.Lattice(16, 16, 8, 0.6, storage=lbm.F32)
    g.init_velocity(np.zeros((3, 8, 16, 16)))
    g.set_pipe(6.0)
    with pytest.raises(lbm.LbmError):
        g.tke_budget(0)
    with pytest.raises(lbm.LbmError):
        g.tke_budget(257)
    out = g.tke_budget(3)
    assert out.shape == (3, tb.NT) and np.all(np.isfinite(out)) and out[:, 0].sum() > 0
    g.close()
