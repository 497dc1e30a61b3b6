// lowp.cuh -- buffers and preparation kernels of the low-precision step,
// shared by the single-system loop (evolve_lowp.cu) and the batch (batch.cu).
#pragma once

#include "common.cuh"

namespace tc {

struct LowpBufs {
    int N, Np, S;
    size_t E;
    void* Uparts;    // parts of V = U / c - I
    float* Rr;
    float* Ri;
    void* Rparts;
    float* Xr;
    float* Xi;
    void* Xparts;
    double* scratch;
};

size_t plane_bytes(int Np, size_t E);
size_t lowp_system_bytes(int n, int precision);
tc_status lowp_carve(int n, int precision, Arena& ar, LowpBufs& b);
// unit phase of Tr U, V parts, rho FP32 planes and parts
tc_status lowp_prep(int precision, const double* U, const double* rho, LowpBufs& b, cudaStream_t s);
// rho <- rho / Tr rho (FP64 trace), parts rebuilt
tc_status lowp_renorm(int precision, LowpBufs& b, cudaStream_t s);
// FP32 planes -> interleaved complex128 rho (N x N)
tc_status lowp_finish(const LowpBufs& b, double* rho, cudaStream_t s);

}  // namespace tc
