// tile_order.cuh -- the order in which the CTAs of a tensor-core GEMM launch
// visit the 128 x 128 output tiles (single CTAs, and CTA pairs sharing an
// operand panel).  Plain C++ with host and device linkage, so that the host
// tests can check the orders' coverage against the launch sizes.
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define TC_HD __host__ __device__
#else
#define TC_HD
#endif

namespace tc {
namespace cg {

TC_HD inline int tile_min(int a, int b) { return a < b ? a : b; }

TC_HD inline void tri_decode(int b, int& i, int& j) {
    int r = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((r + 1) * (r + 2) / 2 <= b) ++r;
    while (r * (r + 1) / 2 > b) --r;
    i = r;
    j = b - r * (r + 1) / 2;
}

// Tile b of the launch -> (I, J).  Both orders keep the CTAs that run at the
// same time on few operand panels, so the panels are re-read from L2:
//  mode 0 (T x T tiles, or the columns [lo, hi)): groups of G row tiles,
//  column by column;
//  mode 1 (block-lower tiles, or those of the rows [lo, hi); lo a multiple of
//  G, hi a multiple of G or T): G x G super-blocks of the lower triangle, row
//  by row; inside a super-block the tiles go column by column (the diagonal
//  super-blocks hold only their lower half).
TC_HD inline void tile_of_range(int mode, int T, int G, int lo, int hi, int b, int& I, int& J) {
    if (G < 1) G = 1;
    if (mode == 0) {
        const int C = hi - lo;
        int per_group = G * C;
        int g = b / per_group;
        int first = g * G;
        int rows = tile_min(G, T - first);
        int in = b % per_group;
        I = first + in % rows;
        J = lo + in / rows;
        return;
    }
    const int SB0 = lo / G, SB1 = (hi + G - 1) / G;
    for (int bi = SB0; bi < SB1; bi++) {
        const int rows = tile_min(G, T - bi * G);
        for (int bj = 0; bj <= bi; bj++) {
            const int cols = tile_min(G, T - bj * G);
            const int cnt = (bi == bj) ? rows * (rows + 1) / 2 : rows * cols;
            if (b < cnt) {
                if (bi == bj) {
                    int ti, tj;
                    tri_decode(b, ti, tj);
                    I = bi * G + ti;
                    J = bj * G + tj;
                } else {
                    I = bi * G + b % rows;
                    J = bj * G + b / rows;
                }
                return;
            }
            b -= cnt;
        }
    }
    I = J = 0;   // not reached for b below the launch's tile count
}

TC_HD inline void tile_of(int mode, int T, int G, int b, int& I, int& J) {
    tile_of_range(mode, T, G, 0, T, b, I, J);
}

// CTA pairs of two row tiles sharing the column tile (the 2-SM MMA: each CTA
// holds its own 128 rows of U and half of the P panel): pair q covers tiles
// (2p, J) and (2p + 1, J), rank r taking I = 2p + r.  Row pairs go in groups
// of G, column by column inside a group, so the pairs that run at the same
// time read few U and few P panels (L2 reuse).  T even.
//  mode 0: the columns [lo, hi) of every row pair (T (hi - lo) / 2 pairs);
//  mode 1: the row pairs of the tile rows [lo, hi) (lo, hi even), each with
//  its columns J <= 2p + 1 (sum over those p of 2p + 2 pairs; the tile
//  (2p, 2p + 1) lies above the diagonal: computed, and overwritten or
//  skipped by the caller).
TC_HD inline void pair_tile_rows_range(int mode, int T, int G, int lo, int hi, int q, int rank, int& I, int& J) {
    const int TP = T / 2;
    if (G < 1) G = 1;
    if (mode == 0) {
        const int C = hi - lo;
        const int per_group = G * C;
        const int g = q / per_group;
        const int rows = tile_min(G, TP - g * G);
        const int in = q % per_group;
        I = 2 * (g * G + in % rows) + rank;
        J = lo + in / rows;
        return;
    }
    const int P1 = hi / 2;
    for (int p0 = lo / 2; p0 < P1; p0 += G) {
        const int last = p0 + tile_min(G, P1 - p0) - 1;
        for (int j = 0; j <= 2 * last + 1; j++) {
            const int first = p0 > j / 2 ? p0 : j / 2;
            const int c = last - first + 1;
            if (q < c) {
                I = 2 * (first + q) + rank;
                J = j;
                return;
            }
            q -= c;
        }
    }
    I = J = 0;   // not reached for q below the launch's pair count
}

TC_HD inline void pair_tile_rows(int mode, int T, int G, int q, int rank, int& I, int& J) {
    pair_tile_rows_range(mode, T, G, 0, T, q, rank, I, J);
}

// Pairs of a launch over the range [lo, hi) (as pair_tile_rows_range).
TC_HD inline long pair_count(int mode, int T, int lo, int hi) {
    if (mode == 0) return (long)(T / 2) * (hi - lo);
    const long p0 = lo / 2, p1 = hi / 2;
    return p1 * (p1 + 1) - p0 * (p0 + 1);
}

// The CTA-pair units of one system in a batched launch, for any T >= 1:
// row pairs (2p, 2p + 1), p < ceil(T / 2); for an odd T the odd CTA's row
// 2p + 1 = T of the last pair lies outside the matrix (its operand loads read
// zeros and its tile is not written).  Row pairs go in groups of G, column by
// column inside a group (as pair_tile_rows).
//  mode 0: every column of every row pair;
//  mode 1: the columns J <= min(2p + 1, T - 1) of row pair p (the tile
//  (2p, 2p + 1) above the diagonal is computed and not written).
TC_HD inline long pair_units(int mode, int T) {
    const long TP = (T + 1) / 2;
    if (mode == 0) return TP * T;
    return T % 2 == 0 ? TP * (TP + 1) : (TP - 1) * TP + T;
}

TC_HD inline void pair_unit(int mode, int T, int G, int q, int rank, int& I, int& J) {
    const int TP = (T + 1) / 2;
    if (G < 1) G = 1;
    if (mode == 0) {
        const int per_group = G * T;
        const int g = q / per_group;
        const int rows = tile_min(G, TP - g * G);
        const int in = q % per_group;
        I = 2 * (g * G + in % rows) + rank;
        J = in / rows;
        return;
    }
    for (int p0 = 0; p0 < TP; p0 += G) {
        const int last = p0 + tile_min(G, TP - p0) - 1;
        const int jmax = tile_min(2 * last + 1, T - 1);
        for (int j = 0; j <= jmax; j++) {
            const int first = p0 > j / 2 ? p0 : j / 2;
            const int c = last - first + 1;
            if (q < c) {
                I = 2 * (first + q) + rank;
                J = j;
                return;
            }
            q -= c;
        }
    }
    I = J = 0;   // not reached for q below pair_units(mode, T)
}

}  // namespace cg
}  // namespace tc
