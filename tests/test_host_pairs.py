"""Host logic of the two-cells-per-lane pipe sweep's work list and wall
tables (pairs.h), compiled with g++.

Checks on seeded solid patterns with seeded wall records: every fluid cell
is swept by exactly one pair half, pairs start on even cells, the added
zero cells are solid, items hold at most 32 pairs in at most two pieces;
per item, the wall-cell mask marks exactly its wall cells, its slot range
starts at its first wall cell's first slot and counts their links; every
ghost slot names its wall cell's place in the item and its direction.
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
#include "pairs.h"
struct Rec { unsigned x, y; };
int main(int argc, char **argv) {
    int nx, ny, nz; long long nw;
    if (std::sscanf(argv[1], "%d", &nx) != 1 || std::sscanf(argv[2], "%d", &ny) != 1 ||
        std::sscanf(argv[3], "%d", &nz) != 1 || std::sscanf(argv[4], "%lld", &nw) != 1) return 2;
    const long long N = (long long)nx * ny * nz;
    std::vector<uint8_t> fl(N);
    std::vector<int> bcells(nw);
    std::vector<Rec> wr(nw);
    FILE *f = std::fopen(argv[5], "rb");
    if (!f || std::fread(fl.data(), 1, N, f) != (size_t)N) return 3;
    if (nw && std::fread(bcells.data(), 4, nw, f) != (size_t)nw) return 3;
    if (nw && std::fread(wr.data(), 8, nw, f) != (size_t)nw) return 3;
    std::fclose(f);
    std::vector<lbmgb::SweepItem> items;
    std::vector<lbmgb::PairItemWall> iw;
    std::vector<unsigned short> ws;
    if (!lbmgb::build_pair_tables(fl.data(), nx, ny, nz, 1, bcells, wr, items, iw, ws)) return 4;
    FILE *o = std::fopen(argv[6], "wb");
    const long long ni = (long long)items.size(), ns = (long long)ws.size();
    std::fwrite(&ni, 8, 1, o);
    std::fwrite(&ns, 8, 1, o);
    std::fwrite(items.data(), 16, items.size(), o);
    std::fwrite(iw.data(), 16, iw.size(), o);
    std::fwrite(ws.data(), 2, ws.size(), o);
    std::fclose(o);
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("pairs")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return d, exe


def run(harness, solid, bcells, masks):
    d, exe = harness
    nz, ny, nx = solid.shape
    first = np.concatenate([[0], np.cumsum([bin(int(m)).count("1") for m in masks])[:-1]]).astype(np.uint32)
    wr = np.stack([first, np.asarray(masks, dtype=np.uint32)], axis=1).astype(np.uint32)
    fin, fout = d / "in.bin", d / "out.bin"
    with open(fin, "wb") as f:
        solid.astype(np.uint8).tofile(f)
        np.asarray(bcells, dtype=np.int32).tofile(f)
        wr.tofile(f)
    subprocess.run([str(exe), str(nx), str(ny), str(nz), str(len(bcells)), str(fin), str(fout)], check=True)
    raw = fout.read_bytes()
    ni, ns = np.frombuffer(raw[:16], dtype=np.int64)
    items = np.frombuffer(raw[16:16 + 16 * ni], dtype=np.uint32).reshape(-1, 4)
    iw = np.frombuffer(raw[16 + 16 * ni:16 + 32 * ni], dtype=np.uint32).reshape(-1, 4)
    ws = np.frombuffer(raw[16 + 32 * ni:16 + 32 * ni + 2 * ns], dtype=np.uint16)
    return items, iw, ws, wr


def lanes(item, nx):
    """(lane, pair's first cell, zero0, zero1) of every lane that holds a pair."""
    row_a, word_a, row_b, word_b = (int(v) for v in item)
    la = (word_a >> 16) & 0xff
    out = []
    for lane in range(32):
        pa = lane < la
        wd, row = (word_a, row_a) if pa else (word_b, row_b)
        lp = lane if pa else lane - la
        ln, lead, trail = (wd >> 16) & 0xff, (wd >> 24) & 15, wd >> 28
        if lp >= ln:
            continue
        c0 = row * nx + 2 * ((wd & 0xffff) - lead + lp)
        out.append((lane, c0, bool(lead and lp == 0), bool(trail and lp == ln - 1)))
    return out


def check(harness, solid, seed):
    nz, ny, nx = solid.shape
    flat = solid.reshape(-1).astype(bool)
    rng = np.random.default_rng(seed)
    # wall cells: fluid cells with a solid x or y neighbour (any set of fluid
    # cells would do); each replaces a seeded nonempty subset of directions 1..18
    s = solid.astype(bool)
    nb = np.zeros_like(s)
    for ax, sh in ((2, 1), (2, -1), (1, 1), (1, -1)):
        nb |= np.roll(s, sh, axis=ax)
    bcells = np.flatnonzero((~s & nb).reshape(-1))
    masks = [int(rng.integers(1, 1 << 18)) << 1 for _ in bcells]
    items, iw, ws, wr = run(harness, solid, bcells, masks)
    rank = {int(c): r for r, c in enumerate(bcells)}
    seen = np.zeros(flat.size, dtype=np.int32)
    for it, item in enumerate(items):
        lanes_ = lanes(item, nx)
        assert 0 < len(lanes_) <= 32
        assert int(item[1]) >> 16 & 0xff <= 32
        mask, links, first = 0, 0, None
        for lane, c0, z0, z1 in lanes_:
            assert c0 % 2 == 0
            for h, zero in ((0, z0), (1, z1)):
                c = c0 + h
                if zero:
                    assert flat[c], "a zero cell must be solid"
                    continue
                assert not flat[c], "a swept cell must be fluid"
                seen[c] += 1
                if c in rank:
                    r = rank[c]
                    first = r if first is None else first
                    mask |= 1 << (2 * lane + h)
                    m = int(wr[r, 1])
                    links += bin(m).count("1")
                    k = int(wr[r, 0])
                    for i in range(1, 19):
                        if m >> i & 1:
                            assert int(ws[k]) == (2 * lane + h) | (i << 6)
                            k += 1
        assert int(iw[it, 2]) | (int(iw[it, 3]) << 32) == mask
        assert int(iw[it, 1]) == links
        if first is not None:
            assert int(iw[it, 0]) == int(wr[first, 0])
    assert np.array_equal(seen[~flat], np.ones(int((~flat).sum()), dtype=np.int32))
    assert np.all(seen[flat] == 0)
    assert len(ws) == sum(bin(m).count("1") for m in masks)


def test_pipe_cross_sections(harness):
    for (nx, ny, nz, R) in ((46, 46, 3, 21.5), (148, 148, 2, 73.0), (40, 38, 4, 17.2)):
        y, x = np.mgrid[0:ny, 0:nx]
        sec = (x - 0.5 * (nx - 1)) ** 2 + (y - 0.5 * (ny - 1)) ** 2 >= R * R
        check(harness, np.broadcast_to(sec, (nz, ny, nx)).copy(), seed=nx)


def test_random_patterns(harness):
    rng = np.random.default_rng(7)
    for n, p in ((24, 0.3), (50, 0.6), (64, 0.1)):
        solid = rng.random((3, 9, n)) < p
        check(harness, solid, seed=n)


def test_odd_width_is_refused(harness):
    d, exe = harness
    solid = np.zeros((2, 4, 7), dtype=np.uint8)
    fin = d / "odd.bin"
    solid.tofile(fin)
    r = subprocess.run([str(exe), "7", "4", "2", "0", str(fin), str(d / "o.bin")])
    assert r.returncode == 4
