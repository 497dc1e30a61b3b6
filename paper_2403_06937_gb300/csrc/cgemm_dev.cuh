// cgemm_dev.cuh -- device code shared by the single-system and the batched
// tensor-core complex GEMM (cgemm_tc.cu, cgemm_batch.cu): operand-part
// splitting, the table of part products, and the epilogue of one 128 x 128
// complex tile  Y = P^H + V P^H  read from the two TMEM accumulators.
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "sm100.cuh"
#include "tile_order.cuh"

namespace tc {
namespace cg {

using namespace sm100;

constexpr int kRowBytes = 32;                 // bytes of K per operand row per stage
constexpr int kATile = 128 * kRowBytes;       // 4 KB
constexpr int kBTile = 256 * kRowBytes;       // 8 KB
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s per wait

// CTA pairs on the 2-SM MMA: a stage of each CTA holds its own S parts of
// U_r and U_i rows and one half of every B part, 3 S tiles of 128 rows x RB
// bytes of K (RB = 32, 64 or 128, with the matching TMA swizzle), and the
// ring holds as many stages as fit in kSplitPairRing bytes.
constexpr int kSplitPairRing = 216 * 1024;
template <int S, int RB>
constexpr int split_pair_stages() {
    return kSplitPairRing / (3 * S * 128 * RB);
}
template <int S, int RB>
constexpr int split_pair_smem() {
    return split_pair_stages<S, RB>() * 3 * S * 128 * RB + 1024 /*align*/ + 512 /*barriers*/;
}

template <int S>
struct Pairs;
template <>
struct Pairs<1> {
    static constexpr int n = 1;
    __device__ static constexpr int a(int) { return 0; }
    __device__ static constexpr int b(int) { return 0; }
};
template <>
struct Pairs<2> {   // big*big, big*small, small*big
    static constexpr int n = 3;
    __device__ static constexpr int a(int p) { return p == 2 ? 1 : 0; }
    __device__ static constexpr int b(int p) { return p == 1 ? 1 : 0; }
};
template <>
struct Pairs<3> {   // x0y0, x0y1, x1y0, x0y2, x1y1, x2y0
    static constexpr int n = 6;
    __device__ static constexpr int a(int p) { return p == 2 ? 1 : (p == 4 ? 1 : (p == 5 ? 2 : 0)); }
    __device__ static constexpr int b(int p) { return p == 1 ? 1 : (p == 3 ? 2 : (p == 4 ? 1 : 0)); }
};

// -------------------------------------------------------------- tile order
// tri_decode, tile_of_range, tile_of and the CTA-pair orders: tile_order.cuh

// -------------------------------------------------------------- splitting
__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// parts of an FP32 value in the operand format of (KIND, S)
template <int KIND, int S>
struct Parts {
    using T = typename std::conditional<KIND == 0, __nv_bfloat16, float>::type;
    __device__ static void split(float x, T (&p)[S]) {
        if constexpr (KIND == 0) {
            float r = x;
#pragma unroll
            for (int s = 0; s < S; s++) {
                p[s] = __float2bfloat16_rn(r);
                r = r - __bfloat162float(p[s]);
            }
        } else {
            float r = x;
#pragma unroll
            for (int s = 0; s < S; s++) {
                p[s] = tf32_rna(r);
                r = r - p[s];
            }
        }
    }
};

template <typename T>
__device__ __forceinline__ void store16(T* dst, const T (&v)[16]) {
    const uint4* src = reinterpret_cast<const uint4*>(v);
    uint4* d = reinterpret_cast<uint4*>(dst);
#pragma unroll
    for (int i = 0; i < (int)(16 * sizeof(T) / 16); i++) d[i] = src[i];
}


// Epilogue of tile (I, J): warps 0-3 read TMEM lanes 32w..32w+31 (row i of the
// tile) and write Y[i][j] = conj(P[j][i]) + (V P^H)[i][j] as FP32 planes and
// operand parts; MODE 1 keeps the block-lower part of a diagonal tile and
// mirrors the conjugate transpose.  src_*: FP32 planes of P (row stride np_).
template <int KIND, int S, int MODE>
__device__ __forceinline__ void epilogue_tile(uint32_t tmem, int warp, int lane, int I, int J, int np_,
                                              const float* __restrict__ src_r, const float* __restrict__ src_i,
                                              void* parts_v, float* out_r, float* out_i) {
    using P = Parts<KIND, S>;
    using T = typename P::T;
    const int row = warp * 32 + lane;                  // TMEM lane = row i of the tile
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    const size_t Np = (size_t)np_;
    const size_t plane = Np * Np;
    const size_t gi = (size_t)I * 128 + row;
    T* parts = reinterpret_cast<T*>(parts_v);
    const bool diag = (MODE == 1) && (I == J);
#pragma unroll 1
    for (int c = 0; c < 128; c += 16) {
        float d1r[16], d1i[16], d2r[16], d2i[16];
        tmem_ld16(tl + c, d1r);            // U_r P_r^T
        tmem_ld16(tl + 128 + c, d1i);      // U_r P_i^T
        tmem_ld16(tl + 256 + c, d2r);      // U_i P_r^T
        tmem_ld16(tl + 384 + c, d2i);      // U_i P_i^T
        tmem_wait_ld();
        const size_t gj0 = (size_t)J * 128 + c;
        float yr[16], yi[16];
#pragma unroll
        for (int q = 0; q < 16; q++) {
            // identity term conj(P[j][i]): lanes read consecutive i
            const size_t t = (gj0 + q) * Np + gi;
            yr[q] = (d1r[q] + d2i[q]) + src_r[t];
            yi[q] = (d2r[q] - d1i[q]) - src_i[t];
        }
        if (MODE == 0 || !diag) {
            // direct tile, full rows of 16: parts (and FP32 planes in mode 1)
            T pr[S][16], pi[S][16];
#pragma unroll
            for (int q = 0; q < 16; q++) {
                T a[S], b[S];
                P::split(yr[q], a);
                P::split(yi[q], b);
#pragma unroll
                for (int s = 0; s < S; s++) { pr[s][q] = a[s]; pi[s][q] = b[s]; }
            }
#pragma unroll
            for (int s = 0; s < S; s++) {
                store16(parts + (size_t)s * plane + gi * Np + gj0, pr[s]);
                store16(parts + (size_t)(S + s) * plane + gi * Np + gj0, pi[s]);
            }
            store16(out_r + gi * Np + gj0, yr);
            store16(out_i + gi * Np + gj0, yi);
        }
        if (MODE == 1) {
#pragma unroll
            for (int q = 0; q < 16; q++) {
                const int col = c + q;
                const size_t gj = gj0 + q;
                if (diag) {
                    if (col > row) continue;
                    float vr = yr[q], vi = (col == row) ? 0.0f : yi[q];
                    T a[S], b[S];
                    P::split(vr, a);
                    P::split(vi, b);
                    for (int s = 0; s < S; s++) {
                        parts[(size_t)s * plane + gi * Np + gj] = a[s];
                        parts[(size_t)(S + s) * plane + gi * Np + gj] = b[s];
                    }
                    out_r[gi * Np + gj] = vr;
                    out_i[gi * Np + gj] = vi;
                    if (col == row) continue;
                }
                // mirror: rho'[j][i] = conj(rho'[i][j]); lanes write consecutive i
                T a[S], b[S];
                P::split(yr[q], a);
                P::split(-yi[q], b);
#pragma unroll
                for (int s = 0; s < S; s++) {
                    parts[(size_t)s * plane + gj * Np + gi] = a[s];
                    parts[(size_t)(S + s) * plane + gj * Np + gi] = b[s];
                }
                out_r[gj * Np + gi] = yr[q];
                out_i[gj * Np + gi] = -yi[q];
            }
        }
    }
}

}  // namespace cg
}  // namespace tc
