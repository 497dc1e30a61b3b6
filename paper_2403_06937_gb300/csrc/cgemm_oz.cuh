// cgemm_oz.cuh -- FP64-accurate complex GEMM Y = U P^H from exact integer
// slices on the BF16 tensor cores (see cgemm_oz.cu).
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace tc {

constexpr int kOzSlices = 9;                                   // base-64 digits per entry (54 bits)
constexpr int kOzPairs = kOzSlices * (kOzSlices + 1) / 2;      // slice pairs with t + u <= 8

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
    unsigned* status;
    unsigned long long wait_ns;   // limit of every barrier wait (0 = 2 s)
};

// Slices [2 * kOzSlices][Np][Np] (BF16 digits: re slices, then im slices) and
// row exponents ex[Np] of the N x N matrix (zero-padded to Np); conj negates
// the imaginary part.
tc_status oz_slice(const double* re, const double* im, bool interleaved, bool conj, int N, size_t ld, int Np,
                   void* slices, int* ex, cudaStream_t s);
size_t oz_slice_bytes(int Np);
// Y = U P^H (mode 0: all tiles; mode 1: block-lower tiles, then oz_mirror)
tc_status cgemm_oz(int mode, const CUtensorMap& tmU, const CUtensorMap& tmP, const OzEpi& ep, cudaStream_t s);
tc_status oz_mirror(double* yr, double* yi, int Np, cudaStream_t s);
// CTA pairs sharing the U panels by TMA multicast (even tile counts; on
// unless TC_OZ_CLUSTER=0 in the environment)
bool oz_cluster_enabled();

// One operand of the emulated product: its digit slices, row exponents and
// TMA map (row r of the operand = row r of A, or row r of B in A B^H).
struct OzMat {
    void* slices;
    int* ex;
    CUtensorMap map;
    int Np;
};
struct OzOut {
    double* yr;        // FP64 planes of the result, row stride Np
    double* yi;
    long long* lo_r;   // int64 scratch planes [Np][Np]
    long long* lo_i;
};
size_t oz_mat_bytes(int Np);
tc_status oz_mat_init(OzMat& m, Arena& ar, int Np);
tc_status oz_mat_load(OzMat& m, const double* re, const double* im, bool interleaved, bool conj, int N, size_t ld,
                      cudaStream_t s);
// Y = A B^H at FP64 accuracy; mode 1 (Hermitian result): block-lower tiles and the mirror.
tc_status oz_product(int mode, const OzMat& A, const OzMat& B, const OzOut& out, int group, cudaStream_t s);

}  // namespace tc
