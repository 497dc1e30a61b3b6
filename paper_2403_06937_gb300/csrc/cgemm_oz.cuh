// cgemm_oz.cuh -- FP64-accurate complex GEMM Y = U P^H from exact integer
// slices on the BF16 tensor cores (see cgemm_oz.cu).
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace tc {

// Digit width of the slices for the inner dimension K of a product (the
// padded size Np).  One pass sums K products of two digits of magnitude at
// most 2^(bits - 1); K 2^(2 bits - 2) <= 2^24 keeps that FP32 sum exact, so
// the smaller K is, the wider the digits and the fewer the slice pairs:
//   K <= 1024:  8-bit digits, 7 slices (56 bits), 28 pairs
//   K <= 4096:  7-bit digits, 8 slices (56 bits), 36 pairs
//   otherwise:  6-bit digits, 9 slices (54 bits), 45 pairs; K in chunks of 16384
// TC_OZ_BITS=6 in the environment keeps the 6-bit digits at every size.
struct OzDigits {
    int bits;     // digit width
    int slices;   // digits per entry
    int pairs;    // slice pairs (t, u) with t + u < slices
    int kmax;     // K per exact pass, 2^(26 - 2 bits)
};
OzDigits oz_digits(int Np);

struct OzEpi {
    int Np;             // padded dimension, a multiple of 128
    int tiles;          // Np / 128
    int group;          // mode 0 raster group (row tiles)
    const int* eU;      // row exponents of U [Np]
    const int* eP;      // row exponents of P [Np]
    double* yr;         // FP64 planes of Y [Np][Np] (int64 level sums until the last pass)
    double* yi;
    long long* lo_r;    // int64 scratch planes [Np][Np] of the low levels
    long long* lo_i;
    int bits;           // digit width and slices per entry (oz_digits(Np))
    int slices;
    unsigned* status;
    unsigned long long wait_ns;   // limit of every barrier wait (0 = 2 s)
};

// Slices [2 * S][Np][Np] (BF16 digits: re slices, then im slices; S digits of
// `bits` bits, oz_digits(Np)) and row exponents ex[Np] of the N x N matrix
// (zero-padded to Np); conj negates the imaginary part.
tc_status oz_slice(const double* re, const double* im, bool interleaved, bool conj, int N, size_t ld, int Np,
                   const OzDigits& dg, void* slices, int* ex, cudaStream_t s);
size_t oz_slice_bytes(int Np);
// Y = U P^H (mode 0: all tiles; mode 1: block-lower tiles, then oz_mirror);
// tmU, tmP: 32-byte-row maps (single CTAs), tmU_w, tmP_w: maps of
// oz_pair_rows()-byte rows (CTA pairs)
tc_status cgemm_oz(int mode, const CUtensorMap& tmU, const CUtensorMap& tmP, const CUtensorMap& tmU_w,
                   const CUtensorMap& tmP_w, const OzEpi& ep, cudaStream_t s);
// Bytes of K per operand row in a stage of the CTA-pair kernel: 128 (TC_OZ_ROWS
// = 32 or 64 in the environment selects narrower rows)
int oz_pair_rows();
tc_status oz_mirror(double* yr, double* yi, int Np, cudaStream_t s);
// True when the product of `tiles` tiles a side runs as CTA pairs on the 2-SM
// MMA (two tiles a side or more, unless TC_OZ_PAIRS=0 in the environment;
// for an odd count the odd CTA of the last row pair has no rows); else single
// CTAs.  Both give the same bits.
bool oz_use_pairs(int tiles);

// One operand of the emulated product: its digit slices, row exponents and
// TMA map (row r of the operand = row r of A, or row r of B in A B^H).
struct OzMat {
    void* slices;
    int* ex;
    CUtensorMap map;     // 32-byte rows (single-CTA kernel)
    CUtensorMap map_w;   // oz_pair_rows() bytes per row (CTA-pair kernel)
    int Np;
    OzDigits dg;   // oz_digits(Np)
};
struct OzOut {
    double* yr;        // FP64 planes of the result, row stride Np
    double* yi;
    long long* lo_r;   // int64 scratch planes [Np][Np]
    long long* lo_i;
};
size_t oz_mat_bytes(int Np);
tc_status oz_mat_init(OzMat& m, Arena& ar, int Np);
// `view` = `base`'s buffers seen as an operand of the smaller padded size Np
tc_status oz_mat_view(OzMat& view, const OzMat& base, int Np);
tc_status oz_mat_load(OzMat& m, const double* re, const double* im, bool interleaved, bool conj, int N, size_t ld,
                      cudaStream_t s);
// Y = A B^H at FP64 accuracy; mode 1 (Hermitian result): block-lower tiles and the mirror.
tc_status oz_product(int mode, const OzMat& A, const OzMat& B, const OzOut& out, int group, cudaStream_t s);

// The FP64-accurate step loop of one system (evolve_oz.cu): its slices,
// FP64 planes of rho and X (stride Np = max(N, 128)) and int64 scratch, carved
// from an arena; first() slices U and pads rho in, step(k) is one step
// (observable row k when obs is given), tail() writes rho back interleaved.
struct OzSystem {
    int n = 0, N = 0, Np = 0, group = 8, renorm_every = 0;
    OzMat Us{}, Ps{};
    double *Rr = nullptr, *Ri = nullptr, *Xr = nullptr, *Xi = nullptr, *scratch = nullptr;
    long long *Lr = nullptr, *Li = nullptr;
    const Model* m = nullptr;
    double* obs = nullptr;
    tc_status carve(int n, Arena& ar);
    tc_status first(const double* U, const double* rho, const Model* m, double* obs, int renorm_every,
                    cudaStream_t cs);
    tc_status step(int k, cudaStream_t cs);
    tc_status tail(double* rho, cudaStream_t cs);
};

}  // namespace tc
