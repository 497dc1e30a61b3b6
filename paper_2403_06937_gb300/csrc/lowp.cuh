// lowp.cuh -- buffers and preparation kernels of the low-precision step,
// shared by the single-system loop (evolve_lowp.cu) and the batch (batch.cu).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace tc {

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// parts of an FP32 value (rho): the split is taken in FP32
template <int KIND, int S>
__device__ __forceinline__ void split_f32(float v, void* base, size_t plane, size_t idx, int part) {
    if constexpr (KIND == 0) {
        __nv_bfloat16* p = static_cast<__nv_bfloat16*>(base);
        float r = v;
#pragma unroll
        for (int s = 0; s < S; s++) {
            __nv_bfloat16 b = __float2bfloat16_rn(r);
            p[(size_t)(part * S + s) * plane + idx] = b;
            r -= __bfloat162float(b);
        }
    } else {
        float* p = static_cast<float*>(base);
        float r = v;
#pragma unroll
        for (int s = 0; s < S; s++) {
            float t = tf32_rna(r);
            p[(size_t)(part * S + s) * plane + idx] = t;
            r -= t;
        }
    }
}

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
// the two halves of lowp_prep: V parts; rho rows [r0, r1) of the padded planes
tc_status lowp_prep_u(int precision, const double* U, LowpBufs& b, cudaStream_t s);
// (cap > 0: at most `cap` CTAs)
tc_status lowp_prep_rho(int precision, const double* rho, LowpBufs& b, int r0, int r1, cudaStream_t s,
                        unsigned cap = 0);
// FP32 planes -> interleaved complex128 rho (N x N), rows [r0, r1) (r1 < 0:
// N), columns [c0, c1) (c1 < 0: N); cap > 0: at most `cap` CTAs
tc_status lowp_finish(const LowpBufs& b, double* rho, cudaStream_t s, int r0 = 0, int r1 = -1, unsigned cap = 0,
                      int c0 = 0, int c1 = -1);

}  // namespace tc
