// cgemm_tc.cuh -- tensor-core complex GEMM Y = U P^H of the low-precision
// step (see cgemm_tc.cu) and the TMA descriptors of its operand planes.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace tc {

// Output side of one launch.  The operand U is given as V = U / c - I
// (c a unit phase), and the epilogue adds the FP32 identity term:
//     Y = P^H + V P^H      (Y = U P^H / c)
//   mode 0: all tiles (the X = U rho of a step).
//   mode 1: Y Hermitian (rho' = U X^H): block-lower tiles computed, the
//           conjugate transpose mirrored.
// Both modes write Y as FP32 planes and as operand parts.
struct CgemmEpi {
    int Np;          // padded dimension, a multiple of 128 (row stride of every plane)
    int tiles;       // Np / 128
    int group;       // mode 0: row tiles per raster group (tiles sharing U panels in L2)
    const float* pr; // FP32 planes of P (the identity term adds conj(P[j][i]))
    const float* pi;
    void* parts;     // [2 * S][Np][Np] operand parts of Y: re parts 0..S-1, then im parts
    float* yr;       // FP32 planes of Y [Np][Np]
    float* yi;
    unsigned* status;
    unsigned long long wait_ns;   // limit of every barrier wait (0 = 2 s)
    int withhold;                 // fault injection: the producer never fills the first stage
    int lo, hi;                   // hi > 0: only the tile columns [lo, hi) (mode 0) or the
                                  // block-lower tiles of the tile rows [lo, hi) (mode 1; lo a
                                  // multiple of group, hi a multiple of group or tiles)
    int shape;                    // tile shape (kShape*; 0 = kShapeAuto)
};

// Tile shape of a tensor-core product launch (the autotuner's choice).  Every
// shape accumulates each output element in the same order (K slice by K
// slice, the part products in one fixed order), so the shape changes speed,
// not results.
//  kShapeSingle:   one CTA per complex 128 x 128 tile (M = 128 MMAs), 32 bytes
//                  of K per operand row in a stage;
//  kShapePair32:   CTA pairs on the 2-SM MMA (M = 256: a 256 x 128 complex
//                  tile per cluster of two), 32-byte K rows;
//  kShapePairWide: CTA pairs with cgemm_pair_rows(precision)-byte K rows;
//  kShapeAuto:     kShapeSingle if TC_GEMM_PAIRS=0 is in the environment,
//                  else kShapePairWide.
// A pair shape runs as single CTAs where pairs do not apply (cgemm_use_pairs).
enum : int { kShapeAuto = 0, kShapeSingle = 1, kShapePair32 = 2, kShapePairWide = 3 };
int cgemm_resolve_shape(int shape);

// stages: TMA ring depth (0 = the largest that fits); the built depths are
// BF16x3 {4, 3}, TF32 {8, 4}, TF32x3 {6, 3}.
// tmU_w, tmP_w (optional): maps of cgemm_pair_rows(precision)-byte rows for
// the CTA-pair kernel (without them the pairs take the 32-byte-row maps).
tc_status cgemm_tc(int precision, int mode, const CUtensorMap& tmU, const CUtensorMap& tmP, const CgemmEpi& ep,
                   cudaStream_t s, int stages = 0, const CUtensorMap* tmU_w = nullptr,
                   const CUtensorMap* tmP_w = nullptr);
// Bytes of K per operand row in a stage of the CTA-pair kernel: 64 for
// BF16x3 and TF32x3, 128 for TF32 (TC_GEMM_ROWS = 32, 64 or 128 in the
// environment overrides, 128 capped at 64 for BF16x3)
int cgemm_pair_rows(int precision);
int cgemm_default_stages(int precision);
// True when a launch of `tiles` tiles a side (and the range lo, hi of
// CgemmEpi) can run as CTA pairs on the 2-SM MMA: an even tile count and
// whole row pairs in a Hermitian row band.
bool cgemm_use_pairs(int tiles, int mode, int lo, int hi);
int cgemm_alt_stages(int precision);

// Test facility: the next `count` launches withhold their first stage (so the
// consumer's wait runs out) and limit every wait to `wait_ns`.
void cgemm_inject_timeout(int count, unsigned long long wait_ns);

int cgemm_parts(int precision);       // S: BF16x3 3, TF32x3 2, TF32 1
int cgemm_products(int precision);    // part products per real product: 6, 3, 1
size_t cgemm_elem_bytes(int precision);

// 3-D tensor map over `planes` consecutive Np x Np planes of operand parts:
// box = 32 bytes of K x 128 rows x 1 plane, 32-byte swizzle.
tc_status make_part_map(CUtensorMap* map, const void* base, int Np, int planes, int precision);
// the same with boxes of `row_bytes` (32, 64 or 128) of K per row and the
// matching swizzle
tc_status make_part_map_rows(CUtensorMap* map, const void* base, int Np, int planes, int precision, int row_bytes);

}  // namespace tc
