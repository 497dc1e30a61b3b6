// kernels.cuh -- launchers shared between the C-ABI layer and the kernels.
#pragma once

#include "common.cuh"

namespace tc {

// ---------------------------------------------------------------- H (Eq. 4)
tc_status launch_build_h(const Model& m, double* H, cudaStream_t s);

// ---------------------------------------------------------------- layout
// interleaved c128 <-> planar (re, im) FP64 / FP32
tc_status launch_split_c128(const double* src, double* re, double* im, size_t count, cudaStream_t s);
tc_status launch_join_c128(const double* re, const double* im, double* dst, size_t count, cudaStream_t s);
tc_status launch_split_c128_f32(const double* src, float* re, float* im, size_t count, cudaStream_t s);
tc_status launch_join_c128_f32(const float* re, const float* im, double* dst, size_t count, cudaStream_t s);

// ---------------------------------------------------------------- host buffers
// Device address of page-locked host memory at `host` (16-byte aligned), or
// nullptr for pageable or misaligned memory.  Through it the SMs read and
// write the host buffer directly; that path keeps its rate (~190 GB/s each
// way on GB300) where copy-engine reads of host memory slow down many-fold
// after heavy host CPU or memory activity.
tc_status host_mapping(const void* host, const void** dev);
// dst <- src (bytes, 16-byte aligned, a multiple of 16) by a kernel
tc_status copy_by_sms(void* dst, const void* src, size_t bytes, cudaStream_t s);

// ---------------------------------------------------------------- FP64 GEMM
// C = alpha * op(A) op(B) + beta * C on planar row-major operands.
//   A[m][k] at m*lda + k, B[k][n] at k*ldb + n, C[m][n] at m*ldc + n.
//   conjA/conjB negate the imaginary plane of the operand.
//   cplx = false: real product of the re planes only (im pointers unused).
//   herm_lower: M == N, only block-lower tiles are computed and the
//   conjugate transpose is written to the mirrored tile (result Hermitian).
struct GemmF64 {
    int M, N, K;
    const double* Ar; const double* Ai; long lda;
    const double* Br; const double* Bi; long ldb;
    double* Cr; double* Ci; long ldc;
    double alpha, beta;
    int conjA, conjB;
    int cplx;
    int herm_lower;
    int tile;        // 32 or 64 (square CTA tile); 0 = the tuned or default choice for this size
    // Split-K for products too small to fill the GPU: when `partial` is given
    // (gemm_f64_splitk_bytes() bytes of scratch), M, N <= kSplitMaxDim and the
    // tiles are fewer than the SMs, K is cut into chunks whose partial products
    // go to `partial` and a second kernel sums them in chunk order
    // (deterministic), applying alpha / beta and the Hermitian mirror.
    double* partial;
};
tc_status gemm_f64(const GemmF64& g, cudaStream_t s);
int gemm_f64_default_tile(int N);
constexpr int kSplitMaxDim = 1024;
size_t gemm_f64_splitk_bytes();

// ---------------------------------------------------------------- tuning
// Kernel configuration chosen by tc_autotune (or the default) per (N, precision).
struct TuneChoice {
    int f64_tile;    // FP64 DMMA GEMM tile: 32 or 64
    int tc_group;    // tensor-core GEMM: row tiles per raster group (L2 reuse of U panels)
    int tc_stages;   // tensor-core GEMM: TMA ring depth (single-CTA shape)
    int tc_shape;    // tensor-core GEMM: tile shape (kShape* of cgemm_tc.cuh; 0 = automatic)
};
TuneChoice tune_lookup(int n, int precision);
// the choice tc_batch_autotune made for a batch of this composition (false: none)
bool tune_batch_lookup(int count, const int* n, int precision, TuneChoice* c);
int tuned_f64_tile(int N);
// bytes of tc_batch_evolve's workspace (batch.cu)
size_t batch_bytes(int count, const int* n, int precision);

// ---------------------------------------------------------------- elementwise
// out = c0*I + sum_j c[j] * M_j (real N x N, up to 4 terms; M_j may alias out)
tc_status launch_lincomb(int N, double c_identity, int terms, const double* const* mats,
                         const double* coef, double* out, cudaStream_t s);
// out[i][j] = (A[i][j] + A[j][i]) / 2 for planar complex, then optional phase
// multiply by (cr + i ci) and interleaved write.  Used at the end of expm.
tc_status launch_expm_finish(int N, const double* Cm, const double* Sm, double phase_re,
                             double phase_im, double* U, cudaStream_t s);
// B = (H - mu I) * dt  (real)
tc_status launch_shift_scale(int N, const double* H, double mu, double dt, double* B, cudaStream_t s);
// diag sum and max column abs sum of (H - mu I) on device -> host via stream sync
tc_status matrix_trace_and_norm1(int N, const double* H, double mu_for_norm, double* trace,
                                 double* norm1, double* scratch, cudaStream_t s);

// ---------------------------------------------------------------- observables
// Deterministic observable row of a density matrix in one of three layouts.
enum RhoLayout { kRhoInterleaved = 0, kRhoPlanarF64 = 1, kRhoPlanarF32 = 2 };
size_t observables_scratch_bytes(int n);
// ld: row stride in elements (0 = N).
tc_status launch_observables(int layout, const void* re_or_c128, const void* im, const Model* m,
                             int n, double* out, double* scratch, cudaStream_t s, size_t ld = 0);
// rho <- rho / Tr rho with the trace taken in FP64 from the planar diagonal.
tc_status launch_renormalise(int layout, void* re, void* im, int n, double* scratch, cudaStream_t s);

}  // namespace tc
