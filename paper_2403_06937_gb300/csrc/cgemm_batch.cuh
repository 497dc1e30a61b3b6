// cgemm_batch.cuh -- per-system descriptor of the batched tensor-core GEMM.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace tc {

// One system of a batch, kept in device memory (the caller's workspace).
// The TMA descriptors must be 64-byte aligned.
struct BatchSys {   // aligned as CUtensorMap (at least 64 bytes)
    CUtensorMap tmU;     // parts of V = U / c - I, 32 bytes of K per row
    CUtensorMap tmR;     // parts of rho
    CUtensorMap tmX;     // parts of X
    CUtensorMap tmU_w;   // the same with rows of the wide CTA-pair shape
    CUtensorMap tmR_w;
    CUtensorMap tmX_w;
    float* Rr;
    float* Ri;
    void* Rparts;
    float* Xr;
    float* Xi;
    void* Xparts;
    int Np;              // padded dimension (multiple of 128)
    int tiles;           // Np / 128
    int tile_begin[2];   // single CTAs: first tile of this system in the X list [0] and the rho' list [1]
    int unit_begin[2];   // CTA pairs: first unit of this system in the two lists
};

// The launches of a batch: the tile shape (kShapeSingle, kShapePair32 or
// kShapePairWide of cgemm_tc.cuh), the raster group (row tiles; CTA pairs
// take group / 2 row pairs), and the lengths of the work lists.
struct BatchPlan {
    int shape;
    int group;
    int rb;         // bytes of K per operand row of the pair shapes
    int tiles[2];   // single-CTA tiles of the two products
    int units[2];   // CTA-pair units of the two products
};

// A plan for `precision` with the tile shape and raster group the autotuner
// chose for n atoms (the batch's largest system), and empty work lists.
BatchPlan batch_plan(int precision, int n);

// Appends one system: writes the six tensor maps of h over its operand parts
// (planes = 2 S planes of Np x Np each), its Np, tiles and list offsets, and
// advances the plan's list lengths.  The caller sets the FP32 plane pointers.
tc_status batch_plan_add(BatchPlan& plan, BatchSys& h, int precision, int Np, const void* Uparts,
                         const void* Rparts, const void* Xparts);

// One persistent launch over the work of all systems of the batch for one
// product (mode 0: X = U rho; mode 1: rho' = U X^H, block-lower tiles), in
// the plan's tile shape.  The results do not depend on the shape.
tc_status cgemm_batch(int precision, int mode, const BatchSys* sys_dev, int nsys, const BatchPlan& plan,
                      unsigned* status, cudaStream_t s);

// the CTA-pair form (cgemm_batch_pair.cu)
tc_status cgemm_batch_pairs(int precision, int mode, int rb, const BatchSys* sys_dev, int nsys, int nunits,
                            int group, unsigned* status, cudaStream_t s);

}  // namespace tc
