// cgemm_batch.cuh -- per-system descriptor of the batched tensor-core GEMM.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace tc {

// One system of a batch, kept in device memory (the caller's workspace).
// The TMA descriptors must be 64-byte aligned.
struct BatchSys {   // aligned as CUtensorMap (at least 64 bytes)
    CUtensorMap tmU;     // parts of V = U / c - I
    CUtensorMap tmR;     // parts of rho
    CUtensorMap tmX;     // parts of X
    float* Rr;
    float* Ri;
    void* Rparts;
    float* Xr;
    float* Xi;
    void* Xparts;
    int Np;              // padded dimension (multiple of 128)
    int tiles;           // Np / 128
    int tile_begin[2];   // first tile of this system in the X list [0] and the rho' list [1]
};

// One persistent launch over the tiles of all systems of the batch for one
// product (mode 0: X = U rho; mode 1: rho' = U X^H, block-lower tiles).
tc_status cgemm_batch(int precision, int mode, const BatchSys* sys_dev, int nsys, int ntiles, unsigned* status,
                      cudaStream_t s);

}  // namespace tc
