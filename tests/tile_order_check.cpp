// Host check of the tile orders in tile_order.cuh (built and run by
// tests/test_tile_order.py): every launch form visits each tile it owns
// exactly once, inside the T x T grid, and the launches of a split cover
// the same tiles as the whole launch.
//   single CTAs, mode 0: columns [lo, hi) of T x T; mode 1: block-lower tiles
//     of the tile rows [lo, hi) (lo a multiple of G, hi of G or T);
//   CTA pairs sharing P (pair_tile_rows): both CTAs in one column tile;
//   the batched CTA-pair units (pair_unit, any T): the written tiles (inside
//   the grid, not above the diagonal in mode 1) are each tile owned, once.
// Prints one line per failure and exits 1 if there was any.
#include <cstdio>
#include <set>
#include <utility>
#include <vector>

#include "tile_order.cuh"

using tc::cg::pair_count;
using tc::cg::pair_tile_rows;
using tc::cg::pair_tile_rows_range;
using tc::cg::pair_unit;
using tc::cg::pair_units;
using tc::cg::tile_of;
using tc::cg::tile_of_range;

static int failures = 0;

static void fail(const char* what, int T, int G, int mode, int a, int b) {
    if (failures < 20) std::printf("FAIL %s T=%d G=%d mode=%d (%d, %d)\n", what, T, G, mode, a, b);
    failures++;
}

static long tiles_of_range(int mode, int lo, int hi, int T) {
    return mode == 0 ? (long)T * (hi - lo) : ((long)hi * (hi + 1) - (long)lo * (lo + 1)) / 2;
}

// the tiles a launch form owns: all (mode 0) or the block-lower ones (mode 1)
static std::set<std::pair<int, int>> owned(int mode, int T) {
    std::set<std::pair<int, int>> s;
    for (int I = 0; I < T; I++)
        for (int J = 0; J < T; J++)
            if (mode == 0 || J <= I) s.insert({I, J});
    return s;
}

static void check_single(int T, int G) {
    for (int mode = 0; mode < 2; mode++) {
        std::set<std::pair<int, int>> whole;
        for (long b = 0; b < tiles_of_range(mode, 0, T, T); b++) {
            int I, J;
            tile_of(mode, T, G, (int)b, I, J);
            if (I < 0 || I >= T || J < 0 || J >= T) fail("tile_of out of range", T, G, mode, I, J);
            if (!whole.insert({I, J}).second) fail("tile_of visits twice", T, G, mode, I, J);
        }
        if (whole != owned(mode, T)) fail("tile_of coverage", T, G, mode, 0, 0);
        for (int C = 2; C <= 4; C *= 2) {
            if (T % (C * G) != 0) continue;
            std::set<std::pair<int, int>> split;
            for (int c = 0; c < C; c++) {
                const int lo = c * T / C, hi = (c + 1) * T / C;
                for (long b = 0; b < tiles_of_range(mode, lo, hi, T); b++) {
                    int I, J;
                    tile_of_range(mode, T, G, lo, hi, (int)b, I, J);
                    const bool in = mode == 0 ? (J >= lo && J < hi) : (I >= lo && I < hi && J <= I);
                    if (!in || I < 0 || I >= T) fail("tile_of_range outside its range", T, G, mode, I, J);
                    if (!split.insert({I, J}).second) fail("tile_of_range visits twice", T, G, mode, I, J);
                }
            }
            if (split != whole) fail("split launches differ from the whole launch", T, G, mode, C, 0);
        }
    }
}

static void check_pairs(int T, int G) {
    for (int mode = 0; mode < 2; mode++) {
        // the whole launch: mode 0 T * T / 2 pairs, mode 1 sum over row pairs i of (2 i + 2)
        long pairs = 0;
        if (mode == 0) {
            pairs = (long)T * (T / 2);
        } else {
            for (int i = 0; i < T / 2; i++) pairs += 2 * i + 2;
        }
        if (pair_count(mode, T, 0, T) != pairs) fail("pair_count of the whole launch", T, G, mode, 0, 0);
        std::set<std::pair<int, int>> seen;
        for (long q = 0; q < pairs; q++) {
            int I0, J0, I1, J1;
            pair_tile_rows(mode, T, G, (int)q, 0, I0, J0);
            pair_tile_rows(mode, T, G, (int)q, 1, I1, J1);
            if (J0 != J1) fail("pair_tile_rows: the pair spans two column tiles", T, G, mode, J0, J1);
            if (I1 != I0 + 1 || I0 % 2 != 0) fail("pair_tile_rows: not an even/odd row pair", T, G, mode, I0, I1);
            for (auto t : {std::make_pair(I0, J0), std::make_pair(I1, J1)}) {
                if (t.first < 0 || t.first >= T || t.second < 0 || t.second >= T)
                    fail("pair_tile_rows out of range", T, G, mode, t.first, t.second);
                if (!seen.insert(t).second) fail("pair_tile_rows visits twice", T, G, mode, t.first, t.second);
            }
        }
        for (auto t : owned(mode, T))
            if (!seen.count(t)) fail("pair_tile_rows misses a tile", T, G, mode, t.first, t.second);
        for (auto t : seen)
            if (mode == 1 && t.second > t.first && !(t.second == t.first + 1 && t.first % 2 == 0))
                fail("pair_tile_rows extra tile", T, G, mode, t.first, t.second);
        // split launches over ranges (mode 0: column bands; mode 1: even row bands) cover the same tiles
        for (int C = 2; C <= 4; C *= 2) {
            if (T % (2 * C) != 0) continue;
            std::set<std::pair<int, int>> split;
            for (int c = 0; c < C; c++) {
                const int lo = c * T / C, hi = (c + 1) * T / C;
                const long np = pair_count(mode, T, lo, hi);
                for (long q = 0; q < np; q++)
                    for (int r = 0; r < 2; r++) {
                        int I, J;
                        pair_tile_rows_range(mode, T, G, lo, hi, (int)q, r, I, J);
                        const bool in = mode == 0 ? (J >= lo && J < hi) : (I >= lo && I < hi);
                        if (!in || I < 0 || I >= T || J < 0 || J >= T)
                            fail("pair_tile_rows_range outside its range", T, G, mode, I, J);
                        if (!split.insert({I, J}).second)
                            fail("pair_tile_rows_range visits twice", T, G, mode, I, J);
                    }
            }
            if (split != seen) fail("split pair launches differ from the whole launch", T, G, mode, C, 0);
        }
    }
}

static void check_units(int T, int G) {
    for (int mode = 0; mode < 2; mode++) {
        // count by the definition: ceil(T / 2) row pairs, mode 1 with columns J <= min(2p + 1, T - 1)
        long units = 0;
        for (int p = 0; p < (T + 1) / 2; p++) units += mode == 0 ? T : (2 * p + 2 < T ? 2 * p + 2 : T);
        if (pair_units(mode, T) != units) fail("pair_units", T, G, mode, (int)pair_units(mode, T), (int)units);
        std::set<std::pair<int, int>> written;
        for (long q = 0; q < units; q++) {
            int I0, J0, I1, J1;
            pair_unit(mode, T, G, (int)q, 0, I0, J0);
            pair_unit(mode, T, G, (int)q, 1, I1, J1);
            if (J0 != J1 || J0 < 0 || J0 >= T) fail("pair_unit: column tile", T, G, mode, J0, J1);
            if (I1 != I0 + 1 || I0 % 2 != 0 || I0 < 0 || I0 >= T || I1 > T)
                fail("pair_unit: not an even/odd row pair inside the grid", T, G, mode, I0, I1);
            for (auto t : {std::make_pair(I0, J0), std::make_pair(I1, J1)}) {
                if (t.first >= T || (mode == 1 && t.second > t.first)) continue;   // not written
                if (!written.insert(t).second) fail("pair_unit writes twice", T, G, mode, t.first, t.second);
            }
        }
        if (written != owned(mode, T)) fail("pair_unit coverage", T, G, mode, 0, 0);
    }
}

int main() {
    const std::vector<int> Ts = {1, 2, 3, 4, 8, 16, 32, 64, 128, 256};
    const std::vector<int> Gs = {1, 2, 4, 8, 16};
    for (int T : Ts)
        for (int G : Gs) check_single(T, G);
    for (int T : Ts)
        if (T % 2 == 0)
            for (int G : Gs) check_pairs(T, G);
    for (int T = 1; T <= 40; T++)
        for (int G : Gs) check_units(T, G);
    if (failures) {
        std::printf("%d failures\n", failures);
        return 1;
    }
    std::printf("tile orders ok\n");
    return 0;
}
