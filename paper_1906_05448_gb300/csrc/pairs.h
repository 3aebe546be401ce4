// Work list and wall tables of the pipe sweep with two cells per lane
// (sweep_pair16.cu; host code, no CUDA).
//
// Each run of fluid cells of an x-row is taken from an even cell to an odd
// one: an odd first cell adds its (solid) left neighbour, an even last cell
// its (solid) right neighbour; those zero cells are stored as zeros. The
// run is cut into pieces of up to 32 pairs, encoded as the sweep segments of
// segments.h in pair units (x of the first pair, pairs; bit 56: the first
// pair's first cell is a zero cell; bit 60: the last pair's second cell
// is), and packed two pieces per warp item (pack_sweep_items).
//
// Wall tables, per item: the first ghost slot and the number of links of
// its wall cells (one contiguous range of slots, in the order of the item's
// cells), and the 64-bit mask of its wall cells (bit 2 lane + h for cell h
// of the lane's pair); per ghost slot: the item cell of its wall cell and
// the direction it replaces (cell | direction << 6).
#pragma once

#include <stdint.h>

#include <algorithm>
#include <vector>

#include "segments.h"

namespace lbmgb {

struct PairItemWall {
    unsigned first, links, mask_lo, mask_hi;
};

// fl: one byte per cell, bit `solid_bit` on solid cells; bcells: the wall
// cells in cell order (their rank is the index); wr[r]: .x the first ghost
// slot of wall cell r, .y the mask of the directions it replaces (slots in
// rank order, then direction order). Returns false (tables undefined) when
// nx is odd or too large, or an item's wall cells are not consecutive ranks.
template <typename Rec>
inline bool build_pair_tables(const uint8_t *fl, int nx, int ny, int nz, int solid_bit, const std::vector<int> &bcells,
                              const std::vector<Rec> &wr, std::vector<SweepItem> &items,
                              std::vector<PairItemWall> &iwall, std::vector<unsigned short> &wslot) {
    items.clear();
    iwall.clear();
    wslot.clear();
    if (nx % 2 != 0 || nx >= 65536 || nx < 2) return false;
    std::vector<unsigned long long> segs;
    for (long long row = 0; row < (long long)ny * nz; row++) {
        const long long base = row * nx;
        for (int x = 0; x < nx;) {
            if (fl[base + x] & solid_bit) {
                x++;
                continue;
            }
            int xe = x;
            while (xe + 1 < nx && !(fl[base + xe + 1] & solid_bit)) xe++;
            const int lead = x & 1, trail = (xe & 1) ? 0 : 1;
            const int xs = x - lead, np = (xe + trail - xs + 1) / 2;
            for (int off = 0; off < np; off += 32) {
                const int len = np - off < 32 ? np - off : 32;
                const int fa = off == 0 ? lead : 0, zt = off + len == np ? trail : 0;
                segs.push_back((unsigned long long)row | ((unsigned long long)(xs / 2 + off + fa) << 32) |
                               ((unsigned long long)len << 48) | ((unsigned long long)fa << 56) |
                               ((unsigned long long)zt << 60));
            }
            x = xe + 1;
        }
    }
    pack_sweep_items(segs, items);
    auto rank_of = [&](long long cell) -> long long {
        auto it = std::lower_bound(bcells.begin(), bcells.end(), (int)cell);
        return (it != bcells.end() && *it == (int)cell) ? (long long)(it - bcells.begin()) : -1;
    };
    size_t nl = 0;
    for (size_t r = 0; r < bcells.size(); r++) nl += (size_t)__builtin_popcount(wr[r].y);
    wslot.assign(nl, 0);
    iwall.resize(items.size());
    for (size_t it = 0; it < items.size(); it++) {
        const SweepItem &w = items[it];
        const int la = (int)((w.word_a >> 16) & 0xff);
        long long first = -1, count = 0;
        unsigned links = 0;
        unsigned long long mask = 0;
        for (int lane = 0; lane < 32; lane++) {
            const bool pa = lane < la;
            const unsigned wd = pa ? w.word_a : w.word_b, row = pa ? w.row_a : w.row_b;
            const int lp = pa ? lane : lane - la;
            const int len = (int)((wd >> 16) & 0xff), lead = (int)((wd >> 24) & 15), trail = (int)(wd >> 28);
            if (lp >= len) continue;
            const long long c0 = (long long)row * nx + 2LL * ((long long)(wd & 0xffff) - lead + lp);
            for (int h = 0; h < 2; h++) {
                if ((h == 0 && lead && lp == 0) || (h == 1 && trail && lp == len - 1)) continue;  // zero cell
                const long long r = rank_of(c0 + h);
                if (r < 0) continue;
                if (first < 0) first = r;
                if (r != first + count) return false;  // the item's links must be one range of slots
                count++;
                const int slot = 2 * lane + h;
                mask |= 1ULL << slot;
                const unsigned m = wr[(size_t)r].y;
                for (int i = 1; i < 19; i++)
                    if ((m >> i) & 1u)
                        wslot[wr[(size_t)r].x + (unsigned)__builtin_popcount(m & ((1u << i) - 1u))] =
                            (unsigned short)(slot | (i << 6));
                links += (unsigned)__builtin_popcount(m);
            }
        }
        iwall[it] = PairItemWall{first < 0 ? 0u : wr[(size_t)first].x, links, (unsigned)mask, (unsigned)(mask >> 32)};
    }
    return true;
}

}  // namespace lbmgb
