"""Host logic of the IBB sweep work list (segments.h), compiled with g++.

Checks on seeded solid patterns: every fluid cell is swept by exactly one
fluid lane, zero lanes sit on solid cells only, nothing leaves the grid,
every 32-byte sector holding a fluid cell is written whole, and two pieces
per warp keep the warps nearly full.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1906_05448_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <vector>
#include "segments.h"
int main(int argc, char **argv) {
    int nx, ny, nz; long long sec;
    if (std::sscanf(argv[1], "%d", &nx) != 1 || std::sscanf(argv[2], "%d", &ny) != 1 ||
        std::sscanf(argv[3], "%d", &nz) != 1 || std::sscanf(argv[4], "%lld", &sec) != 1) return 2;
    const long long N = (long long)nx * ny * nz;
    std::vector<uint8_t> fl(N);
    FILE *f = std::fopen(argv[5], "rb");
    if (!f || std::fread(fl.data(), 1, N, f) != (size_t)N) return 3;
    std::fclose(f);
    std::vector<unsigned long long> segs;
    if (!lbmgb::build_sweep_segments(fl.data(), nx, ny, nz, 1, sec, segs)) return 4;
    std::vector<lbmgb::SweepItem> items;
    lbmgb::pack_sweep_items(segs, items);
    FILE *o = std::fopen(argv[6], "wb");
    std::fwrite(items.data(), sizeof(lbmgb::SweepItem), items.size(), o);
    std::fclose(o);
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("segments")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return d, exe


def run(harness, flags, sec):
    d, exe = harness
    nz, ny, nx = flags.shape
    fin, fout = d / "fl.bin", d / "seg.bin"
    flags.astype(np.uint8).tofile(fin)
    subprocess.run([str(exe), str(nx), str(ny), str(nz), str(sec), str(fin), str(fout)], check=True)
    return np.fromfile(fout, dtype=np.uint32).reshape(-1, 4)


def decode(items, nx):
    """Per lane of every warp item: global cell index and whether it is a
    zero lane."""
    cells, zero = [], []
    for k, (row_a, wa, row_b, wb) in enumerate(items.tolist()):
        used = parts = 0
        for row, w in ((row_a, wa), (row_b, wb)):
            n = (w >> 16) & 0xff
            if n == 0:
                continue
            x0, lead, trail = w & 0xffff, (w >> 24) & 15, w >> 28
            assert lead + trail <= n
            for lp in range(n):
                cells.append(row * nx + x0 - lead + lp)
                zero.append(lp < lead or lp >= n - trail)
            used += n
            parts += 1
        assert 1 <= used <= 32
        # the packer closes a warp only when it is full or holds two pieces
        assert used == 32 or parts == 2 or k == len(items) - 1
    return np.array(cells, dtype=np.int64), np.array(zero, dtype=bool)


def pipe_flags(nx, ny, nz, R):
    y, x = np.mgrid[0:ny, 0:nx]
    cy, cx = (ny - 1) / 2, (nx - 1) / 2
    solid = (x - cx) ** 2 + (y - cy) ** 2 >= R * R
    return np.broadcast_to(solid, (nz, ny, nx)).astype(np.uint8)


CASES = [
    ("pipe148", lambda: pipe_flags(148, 148, 3, 73.0)),
    ("pipe47", lambda: pipe_flags(47, 46, 4, 21.5)),
    ("random", lambda: (np.random.default_rng(7).random((5, 13, 77)) < 0.3).astype(np.uint8)),
    ("long_runs", lambda: (np.random.default_rng(8).random((3, 9, 301)) < 0.02).astype(np.uint8)),
    ("all_fluid", lambda: np.zeros((2, 3, 40), np.uint8)),
    ("all_solid", lambda: np.ones((2, 3, 40), np.uint8)),
]


@pytest.mark.parametrize("sec", [1, 4, 8, 16])
@pytest.mark.parametrize("name,make", CASES)
def test_segments_cover_fluid_once(harness, name, make, sec):
    fl = make()
    nz, ny, nx = fl.shape
    N = fl.size
    flat = fl.reshape(-1)
    items = run(harness, np.ascontiguousarray(fl), sec)
    cells, zero = decode(items, nx)
    assert np.all((cells >= 0) & (cells < N))
    fluid_lanes = cells[~zero]
    # every fluid cell exactly once, no solid cell as a fluid lane
    assert np.array_equal(np.sort(fluid_lanes), np.flatnonzero(flat == 0))
    # zero lanes only on solid cells, each at most once
    assert np.all(flat[cells[zero]] == 1)
    assert len(np.unique(cells[zero])) == zero.sum()
    if sec == 1:
        assert zero.sum() == 0
        return
    # every 32-byte sector that holds a fluid cell and lies inside the grid
    # is written whole
    written = np.zeros(N, bool)
    written[cells] = True
    for s0 in np.unique(fluid_lanes // sec) * sec:
        seg = np.arange(s0, min(s0 + sec, N))
        if len(seg) == sec:
            assert written[seg].all(), (name, s0)


