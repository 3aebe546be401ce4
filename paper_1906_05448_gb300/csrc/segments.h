// Work list of the IBB sweep for a static wall (host code, no CUDA).
//
// Each run of fluid cells of an x-row is cut into segments of at most 32
// lanes; one warp sweeps one segment, so solid cells are never pulled and
// the sweep needs no flag byte. A run is widened over the solid cells that
// share its first and last 32-byte sector in memory (possibly cells of the
// neighbouring rows); those lanes only store zeros, so that no sector of
// the destination array is left partly written.
//
// Segment encoding (64 bits): row y + ny z (bits 0-31); x of lane 0 plus
// the leading zero lanes (32-47); lanes (48-55); leading (56-59) and
// trailing (60-63) zero lanes. Lane l < lanes sweeps cell row * nx + x0 -
// lead + l; it stores zeros when l < lead or l >= lanes - trail.
#pragma once

#include <stdint.h>

#include <vector>

namespace lbmgb {

// flags: one byte per cell, bit `solid_bit` set on solid cells; sec = cells
// per 32-byte sector (32 / bytes per population), 1 to disable widening.
// Returns false when the grid cannot be encoded (nx >= 65536).
inline bool build_sweep_segments(const uint8_t *flags, int nx, int ny, int nz, int solid_bit, long long sec,
                                 std::vector<unsigned long long> &segs) {
    segs.clear();
    if (nx >= 65536 || nx < 1 || sec < 1 || sec > 16) return false;
    const long long N = (long long)nx * ny * nz;
    auto solid = [&](long long g) { return (flags[g] & solid_bit) != 0; };
    for (long long row = 0; row < (long long)ny * nz; row++) {
        const long long base = row * nx;
        for (int x = 0; x < nx;) {
            if (solid(base + x)) {
                x++;
                continue;
            }
            int xe = x;
            while (xe + 1 < nx && !solid(base + xe + 1)) xe++;
            // zero lanes: solid cells of the run's end sectors. The tail runs
            // to the sector end, the grid end or the next run's first cell; a
            // lead that meets a fluid cell is left to the previous run's tail.
            const long long g0 = base + x, g1 = base + xe;
            int lead = 0, tail = 0;
            while ((g1 + tail + 1) % sec != 0 && g1 + tail + 1 < N && solid(g1 + tail + 1)) tail++;
            while ((g0 - lead) % sec != 0 && g0 - lead - 1 >= 0 && solid(g0 - lead - 1)) lead++;
            if ((g0 - lead) % sec != 0) lead = 0;
            const int total = lead + (xe - x + 1) + tail;
            for (int off = 0; off < total; off += 32) {
                const int len = total - off < 32 ? total - off : 32;
                // zero lanes of this piece: its share of [0, lead) and of [total - tail, total)
                int fa = lead - off, zt = off + len - (total - tail);
                fa = fa < 0 ? 0 : (fa > len ? len : fa);
                zt = zt < 0 ? 0 : (zt > len ? len : zt);
                const int x0 = x - lead + off + fa;
                segs.push_back((unsigned long long)row | ((unsigned long long)x0 << 32) |
                               ((unsigned long long)len << 48) | ((unsigned long long)fa << 56) |
                               ((unsigned long long)zt << 60));
            }
            x = xe + 1;
        }
    }
    return true;
}

// Warp items of the sweep: up to two pieces of fluid runs (possibly of two
// rows) share one warp, so that few lanes idle on short runs. A piece is
// (row, word) with word = x of its lane 0 plus its leading zero lanes
// (bits 0-15) | lanes (16-23) | leading zero lanes (24-27) | trailing zero
// lanes (28-31); lanes 0 means no piece. Lanes [0, lanes_a) take piece a,
// the next lanes_b lanes piece b. Pieces longer than the lanes left in a
// warp are split; the zero lanes follow their cells.
struct SweepItem {
    unsigned row_a, word_a, row_b, word_b;
};

inline unsigned sweep_word(int x_lane0, int lanes, int lead, int trail) {
    return (unsigned)(x_lane0 + lead) | ((unsigned)lanes << 16) | ((unsigned)lead << 24) | ((unsigned)trail << 28);
}

inline void pack_sweep_items(const std::vector<unsigned long long> &segs, std::vector<SweepItem> &items) {
    items.clear();
    SweepItem cur{0u, 0u, 0u, 0u};
    int used = 0, parts = 0;
    auto flush = [&]() {
        if (parts > 0) items.push_back(cur);
        cur = SweepItem{0u, 0u, 0u, 0u};
        used = 0;
        parts = 0;
    };
    for (const unsigned long long sg : segs) {
        const unsigned row = (unsigned)(sg & 0xffffffffULL);
        const int x0 = (int)((sg >> 32) & 0xffff), len = (int)((sg >> 48) & 0xff);
        const int fa = (int)((sg >> 56) & 15), zt = (int)(sg >> 60);
        const int xl0 = x0 - fa;  // x of the piece's lane 0
        for (int off = 0; off < len;) {
            if (parts == 2 || used == 32) flush();
            const int t = len - off < 32 - used ? len - off : 32 - used;
            int lead = fa - off, trail = off + t - (len - zt);
            lead = lead < 0 ? 0 : (lead > t ? t : lead);
            trail = trail < 0 ? 0 : (trail > t ? t : trail);
            const unsigned w = sweep_word(xl0 + off, t, lead, trail);
            if (parts == 0) {
                cur.row_a = row;
                cur.word_a = w;
            } else {
                cur.row_b = row;
                cur.word_b = w;
            }
            parts++;
            used += t;
            off += t;
        }
    }
    flush();
}

}  // namespace lbmgb
