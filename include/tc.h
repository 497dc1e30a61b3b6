/*
 * tc.h -- C ABI of libtc, a GB300 (sm_103a) library for the unitary evolution
 * of a Tavis-Cummings cavity-QED system (arXiv 2403.06937, "Distributed
 * computing quantum unitary evolution").
 *
 * The library computes, on one GPU:
 *   H  -- the dense Hamiltonian of Eq. 4 on the basis of Eq. 2;
 *   U  -- e^{-iH dt} by a scaled Taylor polynomial (Eqs. 6-8, 10): dense FP64,
 *          or from the model with H applied as a stencil (no dense H);
 *   rho <- U rho U^dag step after step (Eqs. 6 and 12), on FP64 DMMA, on
 *          tcgen05 tensor cores in split-BF16 / TF32 arithmetic, or at FP64
 *          accuracy from exact integer digit slices on the BF16 tensor cores;
 *   observables read from rho by reduction (populations, the photon-number
 *          probabilities of Eq. 13, trace, purity, energy);
 *   the gradient of a diagonal observable at the final time with respect to
 *          the couplings and frequencies (reverse mode through Eq. 6);
 *   the open system of Eq. 5 with photon leakage (excitation blocks, exact
 *          damping channel, symmetric split step);
 *   many independent systems of uneven size in one call.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - n atoms, N = 2^n (Eq. 2).  Basis index s: atom i (1-based) is bit (n-i)
 *    of s (atom 1 = most significant bit).  Photon number p(s) = n - popcount(s)
 *    (closed system, Sec. II).  hbar = 1.
 *  - Matrices are row-major.  "c128" means interleaved complex double
 *    (re, im), the layout of std::complex<double> and torch.complex128.
 *  - Device pointers are owned by the caller; the library never frees or
 *    keeps them after the call returns.  No call allocates device memory:
 *    scratch space is the caller's `work` buffer, sized by tc_workspace_size
 *    and aligned to 256 bytes.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call is stream-ordered and returns once its work is
 *    enqueued; host arguments (tc_params and its g array) are read before the
 *    call returns.
 *  - Errors: every call returns a tc_status.  TC_OK means the work was
 *    enqueued.  Argument and device errors are detected before any launch and
 *    leave the outputs untouched.  Device-side conditions (non-finite trace,
 *    timeouts of bounded waits) are recorded in a device status word and
 *    reported by tc_sync_status.  tc_last_error() gives a message for the
 *    last non-OK status of the calling thread.
 *  - There is no CPU fallback: without an sm_103 device every compute call
 *    returns TC_ERR_UNSUPPORTED_DEVICE.
 */
#ifndef TC_H_
#define TC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define TC_API __attribute__((visibility("default")))
#else
#define TC_API
#endif

typedef enum tc_status {
    TC_OK = 0,
    TC_ERR_INVALID_ARG = 1,         /* bad size, null pointer, unknown enum   */
    TC_ERR_UNSUPPORTED_DEVICE = 2,  /* current device is not sm_103           */
    TC_ERR_WORKSPACE = 3,           /* work buffer missing, short or misaligned */
    TC_ERR_CUDA = 4,                /* a CUDA runtime call failed             */
    TC_ERR_TIMEOUT = 5,             /* a bounded device wait gave up          */
    TC_ERR_NUMERIC = 6              /* non-finite or non-positive trace       */
} tc_status;

/* Arithmetic of the rho <- U rho U^dag products (the tensor-core path).
 *  TC_FP64   : FP64 DMMA (mma.sync .f64), rho stored in FP64.
 *  TC_BF16X3 : each FP32 operand split in three BF16 parts, six BF16 products
 *              accumulated in FP32 in tensor memory (tcgen05 kind::f16).
 *  TC_TF32   : one TF32 product, FP32 accumulate (tcgen05 kind::tf32).
 *  TC_TF32X3 : big/small TF32 split, three products (kind::tf32).
 *  TC_FP64_OZAKI : FP64-accurate products on the BF16 tensor cores: every
 *              operand row scaled by a power of two and written as S
 *              balanced base-2^b integer digits (exact in BF16): b = 6,
 *              S = 9 in general; b = 7, S = 8 for inner dimensions
 *              K <= 4096; b = 8, S = 7 for K <= 1024 (TC_OZ_BITS=6 in the
 *              environment keeps b = 6).  The S(S+1)/2 digit products with
 *              t + u < S (45 / 36 / 28) accumulate exactly in FP32 (sums
 *              stay below 2^24) and are scaled and summed in FP64.  Within
 *              2^-48 of the row and column scales per product term (worst
 *              case); rho stored in FP64.  tc_evolve, tc_evolve_host,
 *              tc_lindblad_evolve, tc_evolve_backward and tc_batch_evolve
 *              (there the systems run side by side on concurrent branches).
 * In the BF16/TF32 forms U is computed in FP64 and rho is stored in FP32
 * between steps. */
typedef enum tc_precision {
    TC_FP64 = 0,
    TC_BF16X3 = 1,
    TC_TF32 = 2,
    TC_TF32X3 = 3,
    TC_FP64_OZAKI = 4
} tc_precision;

/* Coupling matrix element between s_e (atom i excited, p photons) and s_g
 * (atom i relaxed, p + 1 photons).
 *  TC_COUPLING_BOSONIC      : g_i sqrt(p(s_e) + 1), one bosonic cavity mode
 *                             (Eq. 4, a^dag |p> = sqrt(p+1) |p+1>).
 *  TC_COUPLING_QUBIT_PHOTON : g_i, the reading of Eq. 1 in which each atom
 *                             owns one photon qubit. */
typedef enum tc_coupling {
    TC_COUPLING_BOSONIC = 0,
    TC_COUPLING_QUBIT_PHOTON = 1
} tc_coupling;

/* Model parameters of Eq. 4.  g points to n host doubles (g_1..g_n). */
typedef struct tc_params {
    int n;              /* 1 <= n <= 16 */
    const double* g;    /* host, n values */
    double omega_a;     /* atomic transition frequency */
    double omega_c;     /* cavity frequency */
    int coupling;       /* tc_coupling */
} tc_params;

/* Taylor plan of tc_expm and tc_expm_model.  The paper's Eq. 10 is {10, 0, 0}. */
typedef struct tc_expm_opts {
    int taylor_degree;  /* 0 = smallest degree meeting FP64 accuracy; else 1..30 (tc_expm_model: 1..64) */
    int squarings;      /* -1 = chosen with the degree; else 0..40 */
    int shift;          /* 1 = subtract the mean diagonal before the series */
} tc_expm_opts;

/* Observable row written per time point, TC_OBS_STRIDE(n) doubles:
 *  [0 .. n-1]        P_i = sum_s rho_ss l_i(s), excited population of atom i
 *  [n]               <p> = sum_s rho_ss p(s), mean free-photon number
 *  [n+1 .. 2n+1]     P(m), m = 0..n: probability of m free photons, the
 *                    projector onto popcount(s) = n - m (Eq. 13)
 *  [2n+2]            Tr rho
 *  [2n+3]            Tr rho^2 = sum_ij |rho_ij|^2 (purity)
 *  [2n+4]            E = Tr(H rho)                                          */
#define TC_OBS_STRIDE(n) (2 * (n) + 5)

/* Operation selectors for tc_workspace_size (may be OR-ed). */
#define TC_OP_EXPM 1
#define TC_OP_EVOLVE 2
#define TC_OP_OBSERVABLES 4
#define TC_OP_BACKWARD 8
#define TC_OP_EVOLVE_HOST 16
#define TC_OP_EXPM_MODEL 32
#define TC_OP_LINDBLAD 64
/* tc_evolve_host with a page-locked rho_host: in the tensor-core forms with
 * at least one step and N >= 2048 (row blocks in, row bands out) the SMs read
 * and write the host rows and no device copy of rho is kept, which is what
 * lets n = 16 (64 GiB per complex128 matrix) fit beside U; elsewhere the
 * same as TC_OP_EVOLVE_HOST. */
#define TC_OP_EVOLVE_HOST_PINNED 128

/* ------------------------------------------------------------------ misc */

/* Library version string (static storage). */
TC_API const char* tc_version(void);

/* Message for the last non-OK status returned on this thread (static,
 * thread-local storage; valid until the next failing call on the thread). */
TC_API const char* tc_last_error(void);

/* TC_OK if the current CUDA device is an sm_103 GPU the kernels were built for. */
TC_API tc_status tc_device_check(void);

/* Bytes of `work` needed by the operations in `ops` (TC_OP_*) for n atoms at
 * the given precision.  For TC_OP_BACKWARD, `steps` and `ckpt_every` size the
 * checkpoint store; elsewhere they are ignored.  Returns 0 for invalid n. */
TC_API size_t tc_workspace_size(int n, int precision, int ops, int steps, int ckpt_every);

/* ------------------------------------------------------------- the path */

/* tc_build_hamiltonian -- dense H of Eq. 4 (Sec. II) on the basis of Eq. 2.
 *  H : device, N*N doubles, row-major, 16-byte aligned, written in full.
 *      H[s][s]   = omega_c * p(s) + omega_a * popcount(s)
 *      H[s_g][s_e] = H[s_e][s_g] = coupling element (tc_coupling)
 *      every other entry 0.
 *  Each entry is formed by one IEEE multiply/add sequence without
 *  contraction, so the result is reproducible bit for bit.
 *  Errors: TC_ERR_INVALID_ARG (n outside 1..16, null or misaligned pointers,
 *          g not finite). */
TC_API tc_status tc_build_hamiltonian(const tc_params* params, double* H, void* stream);

/* tc_expm -- U = e^{-i H dt} for a real symmetric H (Sec. III.A, Eqs. 6-8,
 * 10).  With B = (H - mu I) dt, mu = Tr H / N (when opts->shift), the series
 * of Eq. 7 splits into the real polynomials C = cos B and S = sin B, each
 * evaluated by Paterson-Stockmeyer with dense FP64 products; `squarings`
 * complex squarings follow; U = e^{-i mu dt} (C - i S), then U <- (U + U^T)/2
 * (U is complex symmetric because H is real symmetric).
 *  H    : device, N*N doubles (row-major), read only.
 *  U    : device, N*N c128, written (H and U 16-byte aligned).
 *  opts : NULL = automatic plan; {10, 0, 0} reproduces Eq. 10 (k_max = 10,
 *         no scaling, no shift).
 *  work : device, >= tc_workspace_size(n, TC_FP64, TC_OP_EXPM, 0, 0) bytes.
 *  The plan is made on the host from Tr H and ||H - mu I||_1, read back from
 *  the device: this call synchronises `stream` (twice with the shift).
 *  Errors: TC_ERR_INVALID_ARG (dt not finite or <= 0, bad opts),
 *          TC_ERR_WORKSPACE (short/misaligned work). */
TC_API tc_status tc_expm(const double* H, int n, double dt, const tc_expm_opts* opts,
                         void* U, void* work, size_t work_bytes, void* stream);

/* tc_expm_model -- U = e^{-i H dt} for the Hamiltonian of `params` (Eq. 4)
 * without forming H: with B = (H - mu I) dt (mu = Tr H / N when
 * opts->shift), the Taylor polynomial of e^{-iB} (Eq. 7) is evaluated by
 * Horner's rule, T <- I + (-iB) T / k, each step applying B as the structured
 * operator it is (row r of B X combines row r and the n rows r xor 2^b of X):
 * O(n N^2) memory-bound work per Taylor term instead of dense FP64 products.
 * The degree is the smallest whose remainder bound is below 2^-53; an
 * argument with ||B||_inf > 1 is first scaled by 2^-s and squared back
 * (dense FP64 complex products).  U is then multiplied by e^{-i mu dt} and
 * symmetrised.
 * Same result as tc_expm on the dense H to rounding (about 1e-15).
 *  params : model (host).
 *  opts   : NULL = automatic; taylor_degree 1..64 and squarings honoured.
 *  U      : device, N*N c128, written, 16-byte aligned.
 *  work   : device, >= 6 N^2 doubles (tc_workspace_size(n, TC_FP64,
 *           TC_OP_EXPM_MODEL, 0, 0)).
 *  Errors: TC_ERR_INVALID_ARG, TC_ERR_WORKSPACE. */
TC_API tc_status tc_expm_model(const tc_params* params, double dt, const tc_expm_opts* opts, void* U, void* work,
                               size_t work_bytes, void* stream);

/* tc_evolve -- `steps` steps of rho <- U rho U^dag (Eq. 6, evaluated as the
 * two products of Eq. 12: X = U rho, then rho' = X U^dag).  U must be
 * complex symmetric (as returned by tc_expm), so U^dag = conj(U).  The second
 * product computes the lower block triangle only and writes its conjugate
 * transpose to the upper one, so rho stays exactly Hermitian.
 *  U        : device, N*N c128, read only, 16-byte aligned.
 *  rho      : device, N*N c128, in/out (rho_0 in, rho_steps out); Hermitian;
 *             16-byte aligned.
 *  precision: tc_precision of the products.
 *  renorm_every: 0 = never; k > 0 = after every k-th step, rho <- rho / Tr rho
 *             with the trace taken in FP64.
 *  params   : model parameters, used only for the energy column; NULL writes
 *             0 there.
 *  obs      : device, (steps + 1) * TC_OBS_STRIDE(n) doubles, or NULL.  Row 0
 *             is rho_0, row k is rho after step k.
 *  work     : device, >= tc_workspace_size(n, precision, TC_OP_EVOLVE, 0, 0).
 *  With steps > 2 (and kernel timing off) steps 2..K are captured into one
 *  CUDA graph and launched on a library-owned stream ordered after `stream`;
 *  `stream` is ordered after it, and the call returns without waiting.  If
 *  `stream` is itself being captured, the launches go into the caller's
 *  graph instead.
 *  Errors: TC_ERR_INVALID_ARG, TC_ERR_WORKSPACE, TC_ERR_CUDA. */
TC_API tc_status tc_evolve(const void* U, void* rho, int n, int steps, int precision,
                           int renorm_every, const tc_params* params, double* obs,
                           void* work, size_t work_bytes, void* stream);

/* tc_observables -- one observable row (layout above) of a density matrix.
 *  rho  : device, N*N c128, read only.
 *  params: for the energy column (NULL writes 0).
 *  out  : device, TC_OBS_STRIDE(n) doubles.
 *  work : device, >= tc_workspace_size(n, *, TC_OP_OBSERVABLES, 0, 0); holds
 *         per-block partial sums, reduced in a fixed order (the result is
 *         bitwise reproducible run to run).
 *  Errors: TC_ERR_INVALID_ARG, TC_ERR_WORKSPACE. */
TC_API tc_status tc_observables(const void* rho, int n, const tc_params* params,
                                double* out, void* work, size_t work_bytes, void* stream);

/* tc_expectation_diag -- <O> = Tr(diag(O) rho) = sum_s O_s Re rho[s][s] for a
 * diagonal observable O (e.g. the population of one atom, the quantity Sec.
 * IV.A follows in Figs. 3-4; the loss of tc_evolve_backward).  One block
 * sums in a fixed order, so reruns are bitwise identical.
 *  rho    : device, N*N c128, read only.
 *  O_diag : device, N doubles.
 *  out    : device, 1 double.
 *  Errors: TC_ERR_INVALID_ARG, TC_ERR_UNSUPPORTED_DEVICE. */
TC_API tc_status tc_expectation_diag(const void* rho, int n, const double* O_diag, double* out, void* stream);

/* tc_observables_noalloc -- tc_observables for callers that cannot allocate
 * device memory at all, so cannot supply a `work` buffer: for example a
 * monitor thread inside a program whose device memory is wholly owned by
 * another allocator (a framework's caching pool or an arena planned at
 * start-up, where one more cudaMalloc may fail or fragment it), or a caller
 * that must not pay the device-wide synchronisation that cudaMalloc and
 * cudaFree can impose on work already running on other streams.  This
 * entry point has no counterpart in the paper.
 *
 * It computes exactly what tc_observables computes (same kernels, same
 * reduction order, bitwise the same row) but keeps the per-block partial sums
 * in a fixed device array inside the library: 1024 x 37 doubles (296 KiB),
 * enough for every n up to 16.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *  - The array exists on every GPU that loads the library, until the process
 *    exits.
 *  - The first call on a device looks up the array's device address with that
 *    device current (cudaGetSymbolAddress); make that first call before any
 *    stream capture on the device.
 *  - Every call shares the one array.  Calls that overlap on the GPU (on
 *    different streams, or from several host threads on one device) race on
 *    it and may return wrong rows; serialise them.  No slot needs clearing:
 *    each call writes every slot it later reads.
 *  rho, n, params, out, stream: as tc_observables.
 *  Errors: TC_ERR_INVALID_ARG (also when n needs more scratch than the array
 *          holds), TC_ERR_UNSUPPORTED_DEVICE, TC_ERR_CUDA. */
TC_API tc_status tc_observables_noalloc(const void* rho, int n, const tc_params* params, double* out,
                                        void* stream);

/* ---------------------------------------------------------------------------
 * Open-system form: the master equation of Sec. III.A (Eq. 5) with its
 * Lindblad term on.  The paper names the term and sets it to zero; the term
 * here is photon leakage at rate kappa, L(rho) = kappa (a rho a^dag -
 * {a^dag a, rho} / 2).  H conserves the excitation number k = popcount(s) + p
 * and a leaked photon lowers it by one, so the state is block diagonal:
 * block k holds the d_k atom strings with popcount(s) <= k, photon count
 * k - popcount(s).  Packed layout: blocks k = 0..n one after another, block
 * k d_k x d_k row-major interleaved complex128, its basis the first d_k
 * entries of `basis` (all 2^n strings ordered by popcount, then by value).
 * Block n is the closed model's space (Eq. 2) in that order.
 * ------------------------------------------------------------------------- */

/* tc_lindblad_layout -- the packed layout for n atoms (host only, no GPU).
 *  dims    : host int[n+1] or NULL: d_k.
 *  offsets : host size_t[n+2] or NULL: element offset of block k; offsets[n+1]
 *            = total elements (complex) of a packed state.
 *  basis   : host int[2^n] or NULL: atom string at each block position.
 *  Errors: TC_ERR_INVALID_ARG (n outside 1..16). */
TC_API tc_status tc_lindblad_layout(int n, int* dims, size_t* offsets, int* basis);

/* tc_lindblad_propagators -- U_k = e^{-i H_k dt} for every block (Eq. 6 per
 * block), by the structured Horner evaluation of tc_expm_model.
 *  U     : device, packed complex128 (offsets[n+1] elements), written,
 *          16-byte aligned.
 *  work  : device, >= tc_workspace_size(n, TC_FP64, TC_OP_LINDBLAD, 0, 0).
 *  Errors: TC_ERR_INVALID_ARG, TC_ERR_WORKSPACE, TC_ERR_CUDA. */
TC_API tc_status tc_lindblad_propagators(const tc_params* params, double dt, void* U, void* work,
                                         size_t work_bytes, void* stream);

/* tc_lindblad_evolve -- `steps` symmetric split steps of Eq. 5:
 *     rho <- D_{dt/2}(U D_{dt/2}(rho) U^dag)
 * with D_tau the exact damping over tau (the bosonic pure-loss channel,
 * mixing block k+m into block k) and U from tc_lindblad_propagators with the
 * same dt.  Second order in dt; kappa = 0 is the closed evolution of Eq. 6.
 * The block products run on the DMMA GEMM (TC_FP64) or on the tcgen05
 * tensor cores (split forms, as tc_evolve: one persistent launch over the
 * tiles of every block per product, CTA pairs by default, rho stored FP32
 * between steps; FP64 emulated: the blocks one after another on CTA pairs).
 *  U, rho      : device packed complex128; rho in/out (Hermitian blocks).
 *  precision   : TC_FP64, TC_BF16X3, TC_TF32, TC_TF32X3, TC_FP64_OZAKI.
 *  renorm_every: 0 = never; else after every renorm_every-th step all
 *                blocks are divided by the total trace (taken in FP64).
 *  obs         : device f64[(steps+1) * TC_OBS_STRIDE(n)] or NULL; the row
 *                of tc_observables summed over blocks, P(m) = probability
 *                of m photons, E = Tr(H rho).
 *  work        : device, >= tc_workspace_size(n, precision, TC_OP_LINDBLAD,
 *                0, 0).
 *  Errors: TC_ERR_INVALID_ARG, TC_ERR_WORKSPACE, TC_ERR_CUDA; a vanishing or
 *  non-finite trace at renormalisation sets TC_ERR_NUMERIC (tc_sync_status). */
TC_API tc_status tc_lindblad_evolve(const tc_params* params, double kappa, double dt, const void* U, void* rho,
                                    int steps, int precision, int renorm_every, double* obs, void* work,
                                    size_t work_bytes, void* stream);

/* tc_evolve_backward -- gradient of L = Tr(O rho_K), O = diag(O_diag), with
 * rho_K = U^K rho_0 U^-K and U = e^{-iH dt}, with respect to
 * theta = (g_1..g_n, omega_a, omega_c).  Reverse mode through Eq. 6:
 * Lambda_K = O, Lambda_k = U^dag Lambda_{k+1} U; W = sum_{k<K} rho_k Lambda_k;
 * M = W U^dag; G = L_exp(-iH dt, M) (Frechet derivative of the exponential);
 * dL/dtheta_j = 2 dt Im Tr(dH/dtheta_j G).  rho_k is recomputed from
 * checkpoints stored every `ckpt_every` steps.
 *  rho0   : device, N*N c128 (Hermitian, read only).
 *  U      : device, N*N c128, e^{-iH dt} of the same params and dt.
 *  precision: TC_FP64 (DMMA products) or TC_FP64_OZAKI (the per-step
 *           products emulated at FP64 accuracy on the BF16 tensor cores;
 *           n >= 7).
 *  O_diag : device, N doubles.
 *  grad   : host, n + 2 doubles, written when the call returns (this call
 *           synchronises `stream`).
 *  loss   : host, 1 double (may be NULL), L at the final time.
 *  work   : device, >= tc_workspace_size(n, precision, TC_OP_BACKWARD, steps,
 *           ckpt_every).
 *  Errors: TC_ERR_INVALID_ARG, TC_ERR_WORKSPACE, TC_ERR_CUDA, TC_ERR_NUMERIC. */
TC_API tc_status tc_evolve_backward(const tc_params* params, double dt, int steps,
                                    const void* rho0, const void* U, int ckpt_every, int precision,
                                    const double* O_diag, double* grad, double* loss,
                                    void* work, size_t work_bytes, void* stream);

/* tc_evolve_host -- tc_evolve with the density matrix and the observables in
 * HOST memory: brings rho_host to the device, runs `steps` steps on the GPU,
 * writes rho and the observable rows back, and synchronises `stream` before
 * returning (the results are in host memory on return).  A page-locked
 * (pinned) rho_host is read and written by the GPU's SMs directly through
 * its device mapping, at full link rate also when the host is busy
 * (copy-engine transfers of host memory, reads above all, were measured to
 * slow down many-fold after heavy host CPU or memory activity); a pageable
 * one is copied by the copy engine through a device staging buffer.  In the
 * tensor-core forms with N >= 2048 the transfers overlap the products: rho
 * comes in by 2 or 4 row blocks on an internal stream while the first product
 * of step 1 runs by column blocks as their rows arrive, and the second
 * product of the last step runs bottom-up by 2 to 8 row bands, the entries
 * each band makes final converted and written out while the rows above are
 * computed; a page-locked rho then needs no device copy at all
 * (TC_OP_EVOLVE_HOST_PINNED).  The results are the same bits as tc_evolve's.
 *  U        : device, N*N c128 (as tc_evolve), 16-byte aligned.
 *  rho_host : host, N*N c128, in/out.
 *  obs_host : host, (steps + 1) * TC_OBS_STRIDE(n) doubles, or NULL.
 *  work     : device, >= tc_workspace_size(n, precision, TC_OP_EVOLVE_HOST,
 *             steps, 0) bytes (includes the device copies of rho and obs);
 *             for a page-locked rho_host TC_OP_EVOLVE_HOST_PINNED suffices.
 *  Errors: as tc_evolve. */
TC_API tc_status tc_evolve_host(const void* U, void* rho_host, int n, int steps, int precision,
                                int renorm_every, const tc_params* params, double* obs_host,
                                void* work, size_t work_bytes, void* stream);

/* ------------------------------------------------------------- tuning */

/* tc_autotune -- time every built configuration of the step products for n
 * atoms at `precision` on synthetic operands in `work` and keep the fastest
 * for later calls in this process (tc_evolve, tc_evolve_host, tc_expm,
 * tc_evolve_backward, tc_batch_evolve, tc_lindblad_evolve):
 *   FP64: the DMMA GEMM tile, 32 x 32 or 64 x 64 (timed on a K slice);
 *   tensor cores: the tile shape (1: one CTA per 128 x 128 complex tile;
 *   2: CTA pairs on the 2-SM MMA, a 256 x 128 tile per pair, 32 bytes of K
 *   per operand row a stage; 3: CTA pairs with 64-byte rows, 128 for TF32),
 *   the raster group G (G row tiles at a time for X = U rho, G x G
 *   super-blocks of the lower triangle for the Hermitian product, so
 *   concurrent CTAs share operand panels in L2; 4, 8, 12, 16) and, for
 *   shape 1, the TMA ring depth (two per precision), each timed as the mean
 *   step over windows of 8 back-to-back steps (150 ms to 1.2 s; the clock a
 *   configuration holds under the power cap depends on its shared-memory and
 *   L2 traffic), in two passes in opposite orders.  The open-system call
 *   takes the shape and group chosen for its n; tc_batch_evolve those of
 *   tc_batch_autotune, else those chosen for its largest n.
 * The choice is also appended, one JSON object per line, to the file named by
 * the environment variable TC_AUTOTUNE_CACHE (when set), which is read on the
 * first lookup of a process.  Every configuration computes each output in the
 * same order, so tuning changes speed, not results.  Synchronises `stream`.
 *  work   : device, >= tc_workspace_size(n, precision, TC_OP_EVOLVE, 0, 0).
 *  choice : host, 4 ints (f64 tile, raster group, ring depth, tile shape),
 *           or NULL. */
TC_API tc_status tc_autotune(int n, int precision, void* work, size_t work_bytes, void* stream, int* choice);

/* The configuration tc_evolve will use for (n, precision): tuned if tuned in
 * this process or found in TC_AUTOTUNE_CACHE, else the default.  Host only. */
TC_API tc_status tc_autotune_lookup(int n, int precision, int* choice);

/* Pin the configuration for (n, precision) in this process (host only):
 * choice = {f64 tile 32 | 64, raster group 1..128, a built ring depth,
 * tile shape 0..3 (0: automatic, CTA pairs with wide rows unless
 * TC_GEMM_PAIRS=0 is in the environment)}.  A pair shape runs as single CTAs
 * where the tile count is odd (tc_evolve). */
TC_API tc_status tc_autotune_set(int n, int precision, const int* choice);

/* ------------------------------------------------------------- batching */

/* Bytes of `work` for tc_batch_evolve of `count` systems with n[b] atoms. */
TC_API size_t tc_batch_workspace_size(int count, const int* n, int precision);

/* tc_batch_evolve -- `count` independent systems of uneven size (n[b] atoms
 * each, own U and rho), each stepped `steps` times by rho <- U rho U^dag
 * (Eq. 6) as in tc_evolve.  The tensor-core forms run each product of a step
 * as ONE persistent launch over the tiles of all systems (systems in
 * decreasing size, static round-robin over the SMs; single CTAs or CTA
 * pairs, see tc_batch_autotune); TC_FP64 runs the systems' DMMA products one
 * after another; TC_FP64_OZAKI runs each system's step loop, with buffers of
 * its own, on one of eight concurrent branches of the graph (library-owned
 * streams, one such call at a time per device).  The step loop is captured
 * into one CUDA graph on a library-owned stream and launched once; the call
 * returns after the batch has finished.  Every system's result (rho, observables) is
 * bitwise the result of tc_evolve on that system alone with the same
 * precision.
 *  n, U, rho, params, obs : host arrays of `count` entries.  U[b] and rho[b]
 *             are device pointers (N_b x N_b c128, 16-byte aligned; rho in/out);
 *             params may be NULL (energy column 0) or give each system's
 *             parameters; obs may be NULL or hold device pointers (entries
 *             may be NULL) of (steps + 1) * TC_OBS_STRIDE(n[b]) doubles.
 *  work     : device, >= tc_batch_workspace_size(count, n, precision).
 *  Errors: as tc_evolve, for any system. */
TC_API tc_status tc_batch_evolve(int count, const int* n, const void* const* U, void* const* rho, int steps,
                                 int precision, int renorm_every, const tc_params* params,
                                 double* const* obs, void* work, size_t work_bytes, void* stream);

/* tc_batch_autotune -- choose the tile shape and raster group of the batched
 * tensor-core products for batches of this composition (the multiset of
 * n[b]): the batch's workspace is filled with synthetic operands and one
 * batch step (both persistent launches) is timed in every shape (single CTAs
 * on 128 x 128 tiles; CTA pairs on the 2-SM MMA, 256 x 128 a pair, with 32-byte
 * or wide K rows) and raster group (4, 8, 12, 16), as tc_autotune times its
 * configurations.  Later tc_batch_evolve calls in this
 * process on a batch of the same composition and precision use the fastest
 * (otherwise the tc_autotune choice for the largest n); the choice is also
 * appended to TC_AUTOTUNE_CACHE when set.  Results do not depend on the
 * choice.  Synchronises `stream`.  No counterpart in the paper.
 *  precision : TC_BF16X3, TC_TF32 or TC_TF32X3 (else TC_ERR_INVALID_ARG).
 *  work      : device, >= tc_batch_workspace_size(count, n, precision).
 *  choice    : host, 2 ints (raster group, tile shape 1..3), or NULL. */
TC_API tc_status tc_batch_autotune(int count, const int* n, int precision, void* work, size_t work_bytes,
                                   void* stream, int* choice);

/* Pin the batch choice for this composition and precision in this process
 * (host only): choice = {raster group 1..128, tile shape 0..3}. */
TC_API tc_status tc_batch_autotune_set(int count, const int* n, int precision, const int* choice);

/* The batch choice for this composition and precision, if tuned or pinned in
 * this process or found in TC_AUTOTUNE_CACHE (host only): *found = 1 and
 * choice = {raster group, tile shape}; else *found = 0 and tc_batch_evolve
 * takes the tc_autotune choice for its largest n. */
TC_API tc_status tc_batch_autotune_lookup(int count, const int* n, int precision, int* choice, int* found);

/* ----------------------------------------------------------- measurement */

/* Number of kernels this library has launched in this process. */
TC_API long long tc_launch_count(void);

/* tc_timing_enable(1): from now on every product-kernel launch (the GEMMs of
 * the step loop) is bracketed by a CUDA event pair recorded on the stream it
 * is launched on, tagged with its algorithmic FLOP count (8 N^3 for X = U rho,
 * 4 N^3 for the Hermitian half of X U^dag, times the number of low-precision
 * products of the precision form).  tc_timing_read synchronises those events
 * and returns the number of timed launches, their summed device time in ms
 * and their FLOPs, then clears the record. */
TC_API tc_status tc_timing_enable(int on);
TC_API tc_status tc_timing_read(long long* launches, double* ms, double* flops);

/* tc_phases_enable(1): from now on tc_evolve_host records a CUDA event at
 * each phase boundary of its call on the stream doing that phase: the start,
 * the end of each host-to-device row-block copy ("h2d<c>"), the operand
 * preparation of U ("prep_u"), each column block of the first product
 * ("x<c>"), each row block of the last second product with its conversion
 * ("y<c>"), the end of each device-to-host row-block copy ("d2h<c>") and the
 * end ("done").  tc_phases_read synchronises the recorded events and returns
 * in ms[i] the time of mark i after the first mark (ms[0] = 0) and in
 * `names` their names, one per line (both for the first `max` marks, names
 * truncated to fit `names_bytes`); *count receives the number recorded.  The
 * record is then cleared.  Measurement support only; no paper counterpart. */
TC_API tc_status tc_phases_enable(int on);
TC_API tc_status tc_phases_read(double* ms, char* names, size_t names_bytes, int max, int* count);

/* ------------------------------------------------------ failure testing */

/* Fault kinds of tc_fault_inject. */
#define TC_FAULT_TC_STAGE_WITHHELD 1

/* tc_fault_inject -- test facility for the timeout path of the tensor-core
 * kernels, injected from the host: the next `count` tensor-core GEMM
 * launches of this process skip filling their first operand stage, so the
 * MMA issuer's wait for it can never complete, and every barrier wait of
 * those launches is limited to `wait_limit_s` seconds (0 < limit <= 10).
 * The kernel then gives up: it records TC_ERR_TIMEOUT in the device status
 * word, stops issuing, waits (bounded) for the copies it did issue, frees its
 * tensor memory and returns, so the context stays usable.  The affected
 * launch's output is garbage; tc_sync_status reports TC_ERR_TIMEOUT.  Use it
 * with launches outside a CUDA graph (steps <= 2 per tc_evolve call). */
TC_API tc_status tc_fault_inject(int kind, int count, double wait_limit_s);

/* tc_sync_status -- synchronise `stream`, then report (and clear) the device
 * status word: TC_ERR_TIMEOUT or TC_ERR_NUMERIC if a kernel recorded one,
 * TC_ERR_CUDA on an asynchronous CUDA error, else TC_OK. */
TC_API tc_status tc_sync_status(void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TC_H_ */
