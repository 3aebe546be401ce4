"""Host-side checks of the C ABI library: it builds for sm_103a, loads, and
exports every entry point include/lbm.h declares. No GPU calls."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1906_05448_gb300 import build, lbm
    build.build()
    return lbm.load()


def declared_entry_points():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    from paper_1906_05448_gb300 import lbm
    names = declared_entry_points()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(lbm.EXPORTS) == names


def test_workspace_bytes_host_only(lib):
    from paper_1906_05448_gb300 import lbm
    g = lbm.make_grid(148, 148, 438, storage="f32")
    b32 = lbm.workspace_bytes(g)
    g16 = lbm.make_grid(148, 148, 438, storage="f16s")
    b16 = lbm.workspace_bytes(g16)
    N = 148 * 148 * 438
    assert b32 >= 2 * 19 * 4 * N
    # storage-dependent parts: two population buffers, the wall cells'
    # values (19 per possible site, default N/4 + 65536 sites) and the
    # compact ghost values (one per possible link, default N/4 + 65536)
    ms = N // 4 + 65536
    assert b32 - b16 == pytest.approx(2 * 19 * 2 * N + 19 * 2 * ms + 2 * ms, rel=0.01)
    assert lbm.workspace_bytes(lbm.make_grid(2, 2, 2)) == 0
    assert lbm.workspace_bytes(lbm.make_grid(16, 16, 16, storage=9)) == 0


def test_d3q27_workspace_rules(lib):
    from paper_1906_05448_gb300 import lbm
    n = (40, 24, 16)
    N = n[0] * n[1] * n[2]
    b19 = lbm.workspace_bytes(lbm.make_grid(*n, storage="f32"))
    b27 = lbm.workspace_bytes(lbm.make_grid(*n, storage="f32", lattice=27))
    # two buffers of 8 more FP32 planes, and per (x, y) column the pipe wall's
    # direction masks (2 x 4 B) and two FP32 weights per direction
    cols = n[0] * n[1]
    assert b27 - b19 == pytest.approx(2 * 8 * 4 * N + cols * (8 + 2 * 4 * 27), abs=4096)
    assert lbm.workspace_bytes(lbm.make_grid(*n, storage="f64", lattice=27)) > 0
    # D3Q27 runs BGK on FP64 or FP32 storage only; other velocity sets are refused
    assert lbm.workspace_bytes(lbm.make_grid(*n, storage="f16s", lattice=27)) == 0
    assert lbm.workspace_bytes(lbm.make_grid(*n, storage="f32", rates=lbm.RATES_DHUMIERES, lattice=27)) == 0
    assert lbm.workspace_bytes(lbm.make_grid(*n, storage="f32", lattice=15)) == 0
    assert lbm.workspace_bytes(lbm.make_grid(*n, storage="f32", lattice=0)) == b19


def test_create_rejects_bad_arguments_without_gpu(lib):
    from paper_1906_05448_gb300 import lbm
    g = lbm.make_grid(16, 16, 16)
    h = ctypes.c_void_p()
    F = (ctypes.c_double * 3)(0, 0, 0)
    # null workspace and tau <= 1/2 are refused before any CUDA call
    assert lib.lbm_create(ctypes.byref(g), 0.6, F, None, 1 << 30, None, ctypes.byref(h)) == lbm.LBM_EINVAL
    assert lib.lbm_create(ctypes.byref(g), 0.5, F, ctypes.c_void_p(256), 1 << 30, None, ctypes.byref(h)) == lbm.LBM_EINVAL
    assert lib.lbm_create(ctypes.byref(g), 0.6, F, ctypes.c_void_p(256), 16, None, ctypes.byref(h)) == lbm.LBM_ENOMEM
    assert lib.lbm_status_string(lbm.LBM_EUNSTABLE) == b"numerical instability detected"


def test_kernels_built_for_sm103a():
    from paper_1906_05448_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    src = open(os.path.join(ROOT, "paper_1906_05448_gb300", "lbm.py")).read()
    assert "oracle" not in src.replace("oracle.", "")  # the binding never reaches the oracle
