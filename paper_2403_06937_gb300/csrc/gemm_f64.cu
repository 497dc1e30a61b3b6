// gemm_f64.cu -- FP64 complex / real GEMM on the DMMA path (mma.sync .f64).
//
// Used for every product of the plain FP64 form: the Taylor polynomial and
// squarings of e^{-iHdt} (Sec. III.A, Eqs. 7-8 and 10), the two products of
// one step rho <- U rho U^dag (Eqs. 6 and 12), and the adjoint products.
//
// On GB300 the FP64 pipe delivers about 1 TFLOP/s for the whole chip (a few
// FP64 FMAs per clock per SM), so this kernel is bound by the FP64 issue rate,
// not by memory: tiles are staged through shared memory with plain loads and
// the design goal is only that every warp always has independent DMMA
// instructions to issue.  Complex products use four real m16n8k8 DMMAs per
// fragment on planar (re, im) operands.
#include <algorithm>

#include "kernels.cuh"

namespace tc {
namespace {

constexpr int BK = 16;
constexpr int LDA_S = BK + 4;   // padded smem strides (doubles): conflict-free fragment reads
constexpr int kThreads = 128;   // 2 x 2 warps, each a (BT/2) x (BT/2) sub-tile

__device__ __forceinline__ void dmma(double (&d)[4], const double (&a)[4], const double (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f64.f64.f64.f64 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
        : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(b[0]), "d"(b[1]));
}

// Tile (bi, bj) of the block-lower triangle numbered row by row.
__device__ __forceinline__ void lower_tile(int b, int& bi, int& bj) {
    int i = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((i + 1) * (i + 2) / 2 <= b) ++i;
    while (i * (i + 1) / 2 > b) --i;
    bi = i;
    bj = b - i * (i + 1) / 2;
}

constexpr int kMaxSplit = 8;

// Split-K: CTA (x, y, z) covers K range [z kc, (z + 1) kc) and, when
// `partial` is set, stores its raw complex accumulator (no alpha, beta or
// mirror) to partial[z][row][col] (re planes, then im planes at offset
// kMaxSplit M N).
template <bool CPLX, int BT>
__global__ void __launch_bounds__(kThreads, 1) gemm_f64_kernel(GemmF64 p, int kc) {
    constexpr int BM = BT, BN = BT;
    constexpr int LDB_S = BN + 4;
    constexpr int MI = BT / 32, NI = BT / 16;   // m16 / n8 fragments per warp
    __shared__ double sAr[BM * LDA_S];
    __shared__ double sBr[BK * LDB_S];
    __shared__ double sAi[CPLX ? BM * LDA_S : 1];
    __shared__ double sBi[CPLX ? BK * LDB_S : 1];

    int tile_m, tile_n;
    if (p.herm_lower) {
        lower_tile(blockIdx.x, tile_m, tile_n);
    } else {
        tile_m = blockIdx.y;
        tile_n = blockIdx.x;
    }
    const int m0 = tile_m * BM, n0 = tile_n * BN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * (BT / 2), wn = (warp & 1) * (BT / 2);
    const int gq = lane >> 2, tq = lane & 3;

    double accr[MI][NI][4], acci[MI][NI][4];
#pragma unroll
    for (int a = 0; a < MI; a++)
#pragma unroll
        for (int b = 0; b < NI; b++)
#pragma unroll
            for (int c = 0; c < 4; c++) { accr[a][b][c] = 0.0; acci[a][b][c] = 0.0; }

    const double sa = p.conjA ? -1.0 : 1.0;
    const double sb = p.conjB ? -1.0 : 1.0;

    const int kbeg = blockIdx.z * kc;
    const int kend = min(p.K, kbeg + kc);
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        // stage A (BM x BK) and B (BK x BN), zero-filled outside the matrix
#pragma unroll
        for (int r = 0; r < (BM * BK) / kThreads; r++) {
            int e = tid + r * kThreads;
            int row = e / BK, col = e % BK;
            int gm = m0 + row, gk = k0 + col;
            bool ok = gm < p.M && gk < kend;
            long off = (long)gm * p.lda + gk;
            sAr[row * LDA_S + col] = ok ? p.Ar[off] : 0.0;
            if (CPLX) sAi[row * LDA_S + col] = ok ? sa * p.Ai[off] : 0.0;
        }
#pragma unroll
        for (int r = 0; r < (BK * BN) / kThreads; r++) {
            int e = tid + r * kThreads;
            int row = e / BN, col = e % BN;
            int gk = k0 + row, gn = n0 + col;
            bool ok = gk < kend && gn < p.N;
            long off = (long)gk * p.ldb + gn;
            sBr[row * LDB_S + col] = ok ? p.Br[off] : 0.0;
            if (CPLX) sBi[row * LDB_S + col] = ok ? sb * p.Bi[off] : 0.0;
        }
        __syncthreads();

#pragma unroll
        for (int kk = 0; kk < BK; kk += 8) {
            double ar[MI][4], ai[MI][4], nai[MI][4], br[NI][2], bi[NI][2];
#pragma unroll
            for (int mi = 0; mi < MI; mi++) {
                int r0 = wm + mi * 16 + gq;
                ar[mi][0] = sAr[r0 * LDA_S + kk + tq];
                ar[mi][1] = sAr[(r0 + 8) * LDA_S + kk + tq];
                ar[mi][2] = sAr[r0 * LDA_S + kk + tq + 4];
                ar[mi][3] = sAr[(r0 + 8) * LDA_S + kk + tq + 4];
                if (CPLX) {
                    ai[mi][0] = sAi[r0 * LDA_S + kk + tq];
                    ai[mi][1] = sAi[(r0 + 8) * LDA_S + kk + tq];
                    ai[mi][2] = sAi[r0 * LDA_S + kk + tq + 4];
                    ai[mi][3] = sAi[(r0 + 8) * LDA_S + kk + tq + 4];
#pragma unroll
                    for (int q = 0; q < 4; q++) nai[mi][q] = -ai[mi][q];
                }
            }
#pragma unroll
            for (int ni = 0; ni < NI; ni++) {
                int c0 = wn + ni * 8 + gq;
                br[ni][0] = sBr[(kk + tq) * LDB_S + c0];
                br[ni][1] = sBr[(kk + tq + 4) * LDB_S + c0];
                if (CPLX) {
                    bi[ni][0] = sBi[(kk + tq) * LDB_S + c0];
                    bi[ni][1] = sBi[(kk + tq + 4) * LDB_S + c0];
                }
            }
#pragma unroll
            for (int mi = 0; mi < MI; mi++)
#pragma unroll
                for (int ni = 0; ni < NI; ni++) {
                    dmma(accr[mi][ni], ar[mi], br[ni]);
                    if (CPLX) {
                        dmma(accr[mi][ni], nai[mi], bi[ni]);   // - Ai Bi
                        dmma(acci[mi][ni], ar[mi], bi[ni]);    //   Ar Bi
                        dmma(acci[mi][ni], ai[mi], br[ni]);    //   Ai Br
                    }
                }
        }
        __syncthreads();
    }

    // epilogue: C = alpha * acc + beta * C  (fragment c0..c3 -> rows g, g+8; cols 2t, 2t+1)
    const bool diag_tile = p.herm_lower && tile_m == tile_n;
#pragma unroll
    for (int mi = 0; mi < MI; mi++)
#pragma unroll
        for (int ni = 0; ni < NI; ni++)
#pragma unroll
            for (int q = 0; q < 4; q++) {
                int row = m0 + wm + mi * 16 + gq + ((q >> 1) << 3);
                int col = n0 + wn + ni * 8 + 2 * tq + (q & 1);
                if (row >= p.M || col >= p.N) continue;
                if (p.partial) {
                    const size_t MN = (size_t)p.M * p.N;
                    const size_t o = (size_t)blockIdx.z * MN + (size_t)row * p.N + col;
                    p.partial[o] = accr[mi][ni][q];
                    if (CPLX) p.partial[(size_t)kMaxSplit * MN + o] = acci[mi][ni][q];
                    continue;
                }
                double vr = p.alpha * accr[mi][ni][q];
                double vi = CPLX ? p.alpha * acci[mi][ni][q] : 0.0;
                long off = (long)row * p.ldc + col;
                if (p.beta != 0.0) {
                    vr += p.beta * p.Cr[off];
                    if (CPLX) vi += p.beta * p.Ci[off];
                }
                if (!p.herm_lower) {
                    p.Cr[off] = vr;
                    if (CPLX) p.Ci[off] = vi;
                    continue;
                }
                // Hermitian result: keep row >= col of a diagonal tile, mirror the rest
                if (diag_tile && row < col) continue;
                long mir = (long)col * p.ldc + row;
                if (row == col) {
                    p.Cr[off] = vr;
                    if (CPLX) p.Ci[off] = 0.0;
                } else {
                    p.Cr[off] = vr;
                    p.Cr[mir] = vr;
                    if (CPLX) { p.Ci[off] = vi; p.Ci[mir] = -vi; }
                }
            }
}

// Sum of the split-K partials in chunk order, then C = alpha sum + beta C,
// or the Hermitian lower triangle and its mirror.
template <bool CPLX>
__global__ void splitk_reduce_kernel(GemmF64 p, int splits) {
    const size_t MN = (size_t)p.M * p.N;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < MN; e += (size_t)gridDim.x * blockDim.x) {
        const int row = (int)(e / p.N), col = (int)(e % p.N);
        if (p.herm_lower && row < col) continue;   // the upper half is written as the mirror
        double sr = 0.0, si = 0.0;
        for (int z = 0; z < splits; z++) {
            sr += p.partial[(size_t)z * MN + e];
            if (CPLX) si += p.partial[(size_t)(kMaxSplit + z) * MN + e];
        }
        double vr = p.alpha * sr;
        double vi = CPLX ? p.alpha * si : 0.0;
        const long off = (long)row * p.ldc + col;
        if (p.beta != 0.0) {
            vr += p.beta * p.Cr[off];
            if (CPLX) vi += p.beta * p.Ci[off];
        }
        if (!p.herm_lower) {
            p.Cr[off] = vr;
            if (CPLX) p.Ci[off] = vi;
        } else if (row == col) {
            p.Cr[off] = vr;
            if (CPLX) p.Ci[off] = 0.0;
        } else {
            const long mir = (long)col * p.ldc + row;
            p.Cr[off] = vr;
            p.Cr[mir] = vr;
            if (CPLX) {
                p.Ci[off] = vi;
                p.Ci[mir] = -vi;
            }
        }
    }
}

int sm_count() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

template <int BT>
tc_status launch_bt(const GemmF64& g, cudaStream_t s) {
    dim3 block(kThreads);
    dim3 grid;
    long tiles;
    if (g.herm_lower) {
        long t = (g.N + BT - 1) / BT;
        tiles = t * (t + 1) / 2;
        grid = dim3((unsigned)tiles);
    } else {
        grid = dim3((g.N + BT - 1) / BT, (g.M + BT - 1) / BT);
        tiles = (long)grid.x * grid.y;
    }
    // split K while the tiles leave SMs idle: about two CTAs per SM, chunks of
    // at least four BK steps
    int splits = 1, kc = g.K;
    if (g.partial && g.M <= kSplitMaxDim && g.N <= kSplitMaxDim) {
        const long want = (2L * sm_count() + tiles - 1) / tiles;
        const int most = g.K / (4 * BK);
        splits = (int)std::min<long>(std::min<long>(want, most), kMaxSplit);
        if (splits < 1) splits = 1;
        kc = ((g.K + splits - 1) / splits + BK - 1) / BK * BK;
        splits = (g.K + kc - 1) / kc;
    }
    GemmF64 gk = g;
    if (splits <= 1) gk.partial = nullptr;
    grid.z = (unsigned)splits;
    if (g.cplx)
        gemm_f64_kernel<true, BT><<<grid, block, 0, s>>>(gk, kc);
    else
        gemm_f64_kernel<false, BT><<<grid, block, 0, s>>>(gk, kc);
    TC_LAUNCH_CHECK();
    if (splits > 1) {
        const size_t MN = (size_t)g.M * g.N;
        const unsigned blocks = (unsigned)std::min<size_t>((MN + 255) / 256, (size_t)sm_count() * 8);
        if (g.cplx)
            splitk_reduce_kernel<true><<<blocks, 256, 0, s>>>(gk, splits);
        else
            splitk_reduce_kernel<false><<<blocks, 256, 0, s>>>(gk, splits);
        TC_LAUNCH_CHECK();
    }
    return TC_OK;
}

}  // namespace

int gemm_f64_default_tile(int N) { return N >= 4096 ? 64 : 32; }

size_t gemm_f64_splitk_bytes() {
    return round256(2 * (size_t)kMaxSplit * kSplitMaxDim * kSplitMaxDim * sizeof(double));
}

tc_status gemm_f64(const GemmF64& g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0 || g.K <= 0) return TC_OK;
    if (g.herm_lower && (g.M != g.N || g.beta != 0.0))
        return fail(TC_ERR_INVALID_ARG, "gemm_f64: Hermitian mode needs M == N and beta == 0");
    const int tile = g.tile ? g.tile : tuned_f64_tile(g.N > g.M ? g.N : g.M);
    if (tile == 32) return launch_bt<32>(g, s);
    if (tile == 64) return launch_bt<64>(g, s);
    return fail(TC_ERR_INVALID_ARG, "gemm_f64: tile %d not built (32 or 64)", tile);
}

}  // namespace tc
