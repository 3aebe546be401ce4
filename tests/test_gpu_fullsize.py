"""The benchmark configuration itself: the 148x148x438 pipe with the IBB
wall in FP32, swept exactly as bench.py times it (fluid-run work items,
persistent grid, compact ghost values). The oracle runs the same 4 steps
in FP64 at full size; every fluid cell's velocity and density are compared
(FP32 bar 1e-5 of the field maximum), and the wall links bit-exactly."""
import numpy as np
import pytest

import oracle
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


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_benchmark_pipe_full_size(lbm):
    p = workloads.PIPE_148
    nx, ny, nz, R = p["nx"], p["ny"], p["nz"], p["radius"]
    pp = workloads.pipe_parameters(R, p["nu"], p["re_tau"])
    force = (0.0, 0.0, pp["g"])
    u = workloads.pipe_velocity(nx, ny, nz, R, pp["u_bulk"], p["perturbation"], seed=0)
    g = lbm.Lattice(nx, ny, nz, pp["tau"], force=force, storage=lbm.F32)
    o = oracle.Sim(nx, ny, nz, pp["tau"], force=force)
    for s in (g, o):
        s.init_velocity(u)
        s.set_pipe(R)
    la, lo = g.links(), o.links()
    assert len(la["cell"]) == len(lo["cell"]) == 1130040
    ka, ko = np.lexsort((la["dir"], la["cell"])), np.lexsort((lo["dir"], lo["cell"]))
    for key in ("cell", "dir", "scheme"):
        assert np.array_equal(np.asarray(la[key])[ka], np.asarray(lo[key])[ko]), key
    assert np.array_equal(np.asarray(la["q"])[ka].view(np.int64), np.asarray(lo["q"])[ko].view(np.int64))
    g.step(4, lbm.BC_IBB)
    o.step(4, oracle.BC_IBB)
    fluid = o.solid()[0] == 0
    rg, ug = g.macro()
    ro, uo = o.macro()
    assert rel(ug[:, fluid], uo[:, fluid]) < 1e-5
    assert rel(rg[fluid], ro[fluid]) < 1e-5
    assert np.max(np.abs(rg[fluid] - ro[fluid])) < 1e-6
