// backward.cu -- reverse-mode gradient of L = Tr(O rho_K) through the step
// rho <- U rho U^dag (Sec. III.A, Eq. 6) and through U = e^{-iH dt}
// (Eqs. 7-8), in FP64 on the DMMA GEMM.
//
// With Lambda_K = O and Lambda_k = U^dag Lambda_{k+1} U (Hermitian),
//     dL = sum_{k<K} 2 Re Tr(Lambda_{k+1} dU rho_k U^dag)
//        = 2 Re Tr(dU M),   M = W U^dag,   W = sum_{k<K} rho_k Lambda_k,
// using U^dag Lambda_{k+1} = Lambda_k U^dag.  With dU = L(A, dA), the
// Frechet derivative of exp at A = -i H dt, and Tr(L(A, E) M) = Tr(E L(A, M)):
//     dL/dtheta = 2 Re Tr(dA G) = 2 dt Im Tr(dH/dtheta G),   G = L(A, M).
// rho_k is recomputed segment by segment from checkpoints stored every
// `ckpt_every` steps, so memory is (K / ckpt_every + ckpt_every) matrices.
//
// L(A, M) is evaluated for the shifted and scaled A' = -i (H - mu I) dt / 2^s
// by the Taylor recurrence of the derivative of the partial sums,
//     T_0 = I, F_0 = 0,  T_k = A' T_{k-1} / k,  F_k = (A' F_{k-1} + E T_{k-1}) / k,
//     e^{A'} = sum T_k,  L(A', E) = sum F_k,   E = M / 2^s,
// then s squarings D <- X D + D X, X <- X X (chain rule of X^2), and the
// shift back: L(A, M) = e^{-i mu dt} L(A', M).
//
// precision TC_FP64_OZAKI runs the per-step products (the forward steps, the
// adjoint steps and W += rho_k Lambda_k) as FP64-accurate products on the
// BF16 tensor cores (cgemm_oz.cu); the few products of M and of the Frechet
// derivative stay on the DMMA GEMM.
#include <cmath>
#include <vector>

#include "cgemm_oz.cuh"
#include "paths.cuh"

namespace tc {
namespace {

unsigned grid_for(size_t work) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t want = (work + 255) / 256;
    size_t cap = (size_t)sms * 16;
    return (unsigned)(want < cap ? (want ? want : 1) : cap);
}

// planar complex matrix
struct CM {
    double* r;
    double* i;
};

tc_status gemm_c(int N, CM A, int conjA, CM B, int conjB, CM C, double alpha, double beta, int herm,
                 cudaStream_t s) {
    GemmF64 g{};
    g.M = g.N = g.K = N;
    g.Ar = A.r; g.Ai = A.i; g.lda = N;
    g.Br = B.r; g.Bi = B.i; g.ldb = N;
    g.Cr = C.r; g.Ci = C.i; g.ldc = N;
    g.alpha = alpha; g.beta = beta;
    g.conjA = conjA; g.conjB = conjB;
    g.cplx = 1;
    g.herm_lower = herm;
    return gemm_f64(g, s);
}

tc_status gemm_r(int N, const double* A, const double* B, double* C, double alpha, double beta, cudaStream_t s) {
    GemmF64 g{};
    g.M = g.N = g.K = N;
    g.Ar = A; g.lda = N;
    g.Br = B; g.ldb = N;
    g.Cr = C; g.ldc = N;
    g.alpha = alpha; g.beta = beta;
    g.cplx = 0;
    return gemm_f64(g, s);
}

__global__ void copy_kernel(const double* a, double* b, size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        b[e] = a[e];
}

__global__ void diag_set_kernel(const double* d, double* re, double* im, int N) {
    const size_t NN = (size_t)N * N;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < NN; e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = e / N, j = e % N;
        re[e] = (i == j) ? d[i] : 0.0;
        im[e] = 0.0;
    }
}

// out = a * X + b * Y (planar complex, real scalars), out may alias X or Y
__global__ void axpby_kernel(double a, const double* xr, const double* xi, double b, const double* yr,
                             const double* yi, double* outr, double* outi, size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double r = a * xr[e] + b * yr[e];
        const double i = a * xi[e] + b * yi[e];
        outr[e] = r;
        outi[e] = i;
    }
}

// Y = c * (-i B X) = c (B X_i - i B X_r) from the real products P_r = B X_r, P_i = B X_i:
// Y_r = c * P_i, Y_i = -c * P_r
__global__ void minus_i_kernel(double c, const double* pr, const double* pi, double* yr, double* yi, size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double a = pr[e], b = pi[e];
        yr[e] = c * b;
        yi[e] = -c * a;
    }
}

__global__ void identity_kernel(double* re, double* im, int N) {
    const size_t NN = (size_t)N * N;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < NN; e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = e / N, j = e % N;
        re[e] = (i == j) ? 1.0 : 0.0;
        im[e] = 0.0;
    }
}

// loss = sum_s O_s Re rho[s][s]; one block, fixed order
__global__ void loss_kernel(const double* rr, const double* O, int N, double* out) {
    __shared__ double sh[1024];
    double a = 0.0;
    for (int s = threadIdx.x; s < N; s += blockDim.x) a += O[s] * rr[(size_t)s * N + s];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

// grad_j = 2 dt Im Tr(dH/dtheta_j G) with G = (pr + i pi) D.  Block j: parameter j
// (0..n-1: g_{j+1}; n: omega_a; n+1: omega_c), fixed-order reduction.
__global__ void contract_kernel(const double* Dr, const double* Di, Model m, double dt, double pr, double pi,
                                double* grad) {
    __shared__ double sh[1024];
    const int n = m.n, j = blockIdx.x;
    const unsigned N = 1u << n;
    double acc = 0.0;   // Im Tr(dH G)
    if (j < n) {
        const unsigned bit = 1u << (n - 1 - j);
        for (unsigned se = threadIdx.x; se < N; se += blockDim.x) {
            if (!(se & bit)) continue;
            const unsigned sg = se & ~bit;
            const double h = m.coupling == TC_COUPLING_QUBIT_PHOTON ? 1.0 : sqrt((double)(n - __popc(se) + 1));
            // G[se][sg] + G[sg][se]
            const double dr = Dr[(size_t)se * N + sg] + Dr[(size_t)sg * N + se];
            const double di = Di[(size_t)se * N + sg] + Di[(size_t)sg * N + se];
            acc += h * (pr * di + pi * dr);   // Im((pr + i pi)(dr + i di))
        }
    } else {
        for (unsigned s = threadIdx.x; s < N; s += blockDim.x) {
            const int pc = __popc(s);
            const double w = (j == n) ? (double)pc : (double)(n - pc);
            const double dr = Dr[(size_t)s * N + s], di = Di[(size_t)s * N + s];
            acc += w * (pr * di + pi * dr);
        }
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) grad[j] = 2.0 * dt * sh[0];
}

struct Bufs {
    int N;
    size_t NN;
    CM U, L, X, W, seg0;
    int nck, c;
    // Frechet scratch
    double* B;
    CM T, F, Tn, Fn, P, Q;
    double* small;
};

size_t cm_bytes(int n) { return 2 * round256(sizeof(double) << (2 * n)); }
size_t real_bytes(int n) { return round256(sizeof(double) << (2 * n)); }

CM take_cm(Arena& ar, size_t NN) {
    CM m;
    m.r = ar.take<double>(NN);
    m.i = ar.take<double>(NN);
    return m;
}

// one forward step P <- U P U^dag (FP64, Hermitian half); conjU: use conj(U) (adjoint step)
tc_status step(int N, CM U, CM P, CM X, int conjU, cudaStream_t s) {
    // X = U' P  (U' = U or conj U);  P' = X conj(U') (U' symmetric: conj(U') = U'^dag)
    TC_TRY(gemm_c(N, U, conjU, P, 0, X, 1.0, 0.0, 0, s));
    return gemm_c(N, X, 0, U, conjU ? 0 : 1, P, 1.0, 0.0, 1, s);
}

tc_status copy_cm(CM a, CM b, size_t NN, cudaStream_t s) {
    copy_kernel<<<grid_for(NN), 256, 0, s>>>(a.r, b.r, NN);
    TC_LAUNCH_CHECK();
    copy_kernel<<<grid_for(NN), 256, 0, s>>>(a.i, b.i, NN);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

// Y = -i Bs X  (Bs real), via two real products into the scratch planes of Q
tc_status minus_i_times(int N, const double* Bs, CM X, CM Y, CM Q, cudaStream_t s) {
    TC_TRY(gemm_r(N, Bs, X.r, Q.r, 1.0, 0.0, s));
    TC_TRY(gemm_r(N, Bs, X.i, Q.i, 1.0, 0.0, s));
    minus_i_kernel<<<grid_for((size_t)N * N), 256, 0, s>>>(1.0, Q.r, Q.i, Y.r, Y.i, (size_t)N * N);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

// Emulated-FP64 products: slices of U and conj(U) (A operands), of the
// current B operand and of rho_k (A operand of the W product).
struct OzBufs {
    OzMat U, Uc, B, A2;
    double* yr;
    double* yi;
    long long* lo_r;
    long long* lo_i;
    int group;
};

size_t oz_backward_extra(int n) {
    const size_t N = (size_t)1 << n;
    return 4 * oz_mat_bytes((int)N) + 4 * round256(N * N * sizeof(double)) + 256;
}

// P <- U' P U'^dag with U' = U (or conj U for the adjoint step), emulated FP64
tc_status step_oz(int N, OzBufs& z, bool adjoint, CM P, CM X, cudaStream_t s) {
    const OzMat& A = adjoint ? z.Uc : z.U;
    TC_TRY(oz_mat_load(z.B, P.r, P.i, false, false, N, (size_t)N, s));
    TC_TRY(oz_product(0, A, z.B, OzOut{X.r, X.i, z.lo_r, z.lo_i}, z.group, s));       // X = U' P^H = U' P
    TC_TRY(oz_mat_load(z.B, X.r, X.i, false, false, N, (size_t)N, s));
    return oz_product(1, A, z.B, OzOut{P.r, P.i, z.lo_r, z.lo_i}, z.group, s);        // P' = U' X^H
}

// W += rho Lambda = rho Lambda^H (Lambda Hermitian), emulated FP64
tc_status w_accumulate_oz(int N, OzBufs& z, CM rho, CM L, CM W, bool init, cudaStream_t s) {
    TC_TRY(oz_mat_load(z.A2, rho.r, rho.i, false, false, N, (size_t)N, s));
    TC_TRY(oz_mat_load(z.B, L.r, L.i, false, false, N, (size_t)N, s));
    if (init) return oz_product(0, z.A2, z.B, OzOut{W.r, W.i, z.lo_r, z.lo_i}, z.group, s);
    TC_TRY(oz_product(0, z.A2, z.B, OzOut{z.yr, z.yi, z.lo_r, z.lo_i}, z.group, s));
    const size_t NN = (size_t)N * N;
    axpby_kernel<<<grid_for(NN), 256, 0, s>>>(1.0, W.r, W.i, 1.0, z.yr, z.yi, W.r, W.i, NN);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

}  // namespace

size_t backward_bytes(int n, int steps, int ckpt_every, int precision) {
    if (n < 1 || n > kMaxAtoms || steps < 1 || ckpt_every < 1) return 0;
    if (precision == TC_FP64_OZAKI) return backward_bytes(n, steps, ckpt_every, TC_FP64) + oz_backward_extra(n);
    const int nck = (steps + ckpt_every - 1) / ckpt_every;
    const int c = ckpt_every < steps ? ckpt_every : steps;
    // U, Lambda, X, W, seg0 + checkpoints + segment + Frechet (T, F, Tn, Fn, P, Q) + B + small
    return (size_t)(5 + nck + c + 6) * cm_bytes(n) + real_bytes(n) + round256((2 * ((size_t)1 << n) + 64) * 8) + 1024;
}

}  // namespace tc

using namespace tc;

extern "C" TC_API tc_status tc_evolve_backward(const tc_params* params, double dt, int steps, const void* rho0,
                                               const void* U, int ckpt_every, int precision, const double* O_diag,
                                               double* grad, double* loss, void* work, size_t work_bytes,
                                               void* stream) {
    Model m;
    TC_TRY(make_model(params, &m));
    const int n = m.n;
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(TC_ERR_INVALID_ARG, "dt must be finite and > 0");
    if (steps < 1) return fail(TC_ERR_INVALID_ARG, "steps must be >= 1");
    if (ckpt_every < 1) return fail(TC_ERR_INVALID_ARG, "ckpt_every must be >= 1");
    if (precision != TC_FP64 && precision != TC_FP64_OZAKI)
        return fail(TC_ERR_INVALID_ARG, "backward: precision must be TC_FP64 or TC_FP64_OZAKI");
    if (precision == TC_FP64_OZAKI && n < 7)
        return fail(TC_ERR_INVALID_ARG, "backward: the emulated form needs n >= 7 (dimension a multiple of 128)");
    if (!rho0 || !U || !O_diag || !grad) return fail(TC_ERR_INVALID_ARG, "null pointer");
    if ((reinterpret_cast<uintptr_t>(rho0) | reinterpret_cast<uintptr_t>(U)) & 15u)
        return fail(TC_ERR_INVALID_ARG, "rho0 and U must be 16-byte aligned");
    const size_t need = backward_bytes(n, steps, ckpt_every, precision);
    if (!work) return fail(TC_ERR_WORKSPACE, "work is NULL (need %zu bytes)", need);
    if (reinterpret_cast<uintptr_t>(work) & 255u) return fail(TC_ERR_WORKSPACE, "work is not 256-byte aligned");
    if (work_bytes < need) return fail(TC_ERR_WORKSPACE, "work has %zu bytes, need %zu", work_bytes, need);
    TC_TRY(check_device());
    cudaStream_t s = as_stream(stream);

    const int N = 1 << n;
    const size_t NN = (size_t)N * N;
    Arena ar{static_cast<char*>(work), work_bytes, 0};
    Bufs b{};
    b.N = N;
    b.NN = NN;
    b.c = ckpt_every < steps ? ckpt_every : steps;
    b.nck = (steps + ckpt_every - 1) / ckpt_every;
    b.U = take_cm(ar, NN);
    b.L = take_cm(ar, NN);
    b.X = take_cm(ar, NN);
    b.W = take_cm(ar, NN);
    b.seg0 = take_cm(ar, NN);
    std::vector<CM> ck(b.nck), seg(b.c);
    for (int k = 0; k < b.nck; k++) ck[k] = take_cm(ar, NN);
    for (int k = 0; k < b.c; k++) seg[k] = take_cm(ar, NN);
    b.T = take_cm(ar, NN);
    b.F = take_cm(ar, NN);
    b.Tn = take_cm(ar, NN);
    b.Fn = take_cm(ar, NN);
    b.P = take_cm(ar, NN);
    b.Q = take_cm(ar, NN);
    b.B = ar.take<double>(NN);
    b.small = ar.take<double>(2 * (size_t)N + 64);
    if (!b.small) return fail(TC_ERR_WORKSPACE, "backward: workspace too small");
    const bool oz = precision == TC_FP64_OZAKI;
    OzBufs z{};
    if (oz) {
        TC_TRY(oz_mat_init(z.U, ar, N));
        TC_TRY(oz_mat_init(z.Uc, ar, N));
        TC_TRY(oz_mat_init(z.B, ar, N));
        TC_TRY(oz_mat_init(z.A2, ar, N));
        z.yr = ar.take<double>(NN);
        z.yi = ar.take<double>(NN);
        z.lo_r = ar.take<long long>(NN);
        z.lo_i = ar.take<long long>(NN);
        if (!z.lo_i) return fail(TC_ERR_WORKSPACE, "backward: workspace too small");
        z.group = tune_lookup(n, TC_BF16X3).tc_group;
        TC_TRY(oz_mat_load(z.U, static_cast<const double*>(U), nullptr, true, false, N, (size_t)N, s));
        TC_TRY(oz_mat_load(z.Uc, static_cast<const double*>(U), nullptr, true, true, N, (size_t)N, s));
    }
    auto fwd_step = [&](CM P) -> tc_status { return oz ? step_oz(N, z, false, P, b.X, s) : step(N, b.U, P, b.X, 0, s); };

    // ---------------------------------------------------------------- forward
    TC_TRY(launch_split_c128(static_cast<const double*>(U), b.U.r, b.U.i, NN, s));
    TC_TRY(launch_split_c128(static_cast<const double*>(rho0), ck[0].r, ck[0].i, NN, s));
    TC_TRY(copy_cm(ck[0], b.seg0, NN, s));   // seg0 = running rho
    for (int k = 1; k <= steps; k++) {
        TC_TRY(fwd_step(b.seg0));
        if (k < steps && k % ckpt_every == 0) TC_TRY(copy_cm(b.seg0, ck[k / ckpt_every], NN, s));
    }
    // loss from rho_K (in seg0)
    loss_kernel<<<1, 1024, 0, s>>>(b.seg0.r, O_diag, N, b.small);
    TC_LAUNCH_CHECK();

    // ---------------------------------------------------------------- backward
    diag_set_kernel<<<grid_for(NN), 256, 0, s>>>(O_diag, b.L.r, b.L.i, N);   // Lambda_K = O
    TC_LAUNCH_CHECK();
    bool w_init = false;
    for (int j = b.nck - 1; j >= 0; j--) {
        const int k0 = j * ckpt_every;
        const int k1 = (k0 + ckpt_every < steps) ? k0 + ckpt_every : steps;   // segment k0 .. k1-1
        // recompute rho_{k0..k1-1} into seg[0..]
        TC_TRY(copy_cm(ck[j], seg[0], NN, s));
        for (int k = k0 + 1; k < k1; k++) {
            TC_TRY(copy_cm(seg[k - 1 - k0], seg[k - k0], NN, s));
            TC_TRY(fwd_step(seg[k - k0]));
        }
        for (int k = k1 - 1; k >= k0; k--) {
            // Lambda_k = U^dag Lambda_{k+1} U  (the step with conj(U)); W += rho_k Lambda_k
            if (oz) {
                TC_TRY(step_oz(N, z, true, b.L, b.X, s));
                TC_TRY(w_accumulate_oz(N, z, seg[k - k0], b.L, b.W, !w_init, s));
            } else {
                TC_TRY(step(N, b.U, b.L, b.X, 1, s));
                TC_TRY(gemm_c(N, seg[k - k0], 0, b.L, 0, b.W, 1.0, w_init ? 1.0 : 0.0, 0, s));
            }
            w_init = true;
        }
    }
    // M = W U^dag = W conj(U)  -> into L (free now)
    CM M = b.L;
    TC_TRY(gemm_c(N, b.W, 0, b.U, 1, M, 1.0, 0.0, 0, s));

    // ---------------------------------------------------------------- Frechet
    // plan from H's trace and norm (computed on the device, read back)
    double* Hs = b.B;   // build H into B, then shift and scale in place
    TC_TRY(launch_build_h(m, Hs, s));
    double trace = 0.0, norm1 = 0.0;
    TC_TRY(matrix_trace_and_norm1(N, Hs, 0.0, &trace, &norm1, b.small + 8, s));
    const double mu = trace / N;
    TC_TRY(matrix_trace_and_norm1(N, Hs, mu, &trace, &norm1, b.small + 8, s));
    double bn = norm1 * dt;
    int sq = 0;
    while (bn > 0.5 && sq < 40) { bn *= 0.5; sq++; }
    // terms: stop when b^(m+1)/(m+1)! * (m+2) < 2^-53
    int mt = 1;
    {
        double term = bn;
        while (mt < 40) {
            term *= bn / (mt + 1);
            if (term * (mt + 2) < std::ldexp(1.0, -53) || bn == 0.0) break;
            mt++;
        }
        mt += 1;
    }
    const double scale = std::ldexp(dt, -sq);
    TC_TRY(launch_shift_scale(N, Hs, mu, scale, b.B, s));   // B = (H - mu) dt / 2^s ; A' = -i B
    // E = M / 2^s into P
    axpby_kernel<<<grid_for(NN), 256, 0, s>>>(std::ldexp(1.0, -sq), M.r, M.i, 0.0, M.r, M.i, b.P.r, b.P.i, NN);
    TC_LAUNCH_CHECK();
    // X = sum T_k into W (reuse), D = sum F_k into seg0 (reuse)
    CM Xs = b.W, D = b.seg0;
    identity_kernel<<<grid_for(NN), 256, 0, s>>>(b.T.r, b.T.i, N);     // T_0 = I
    TC_LAUNCH_CHECK();
    identity_kernel<<<grid_for(NN), 256, 0, s>>>(Xs.r, Xs.i, N);       // X = T_0
    TC_LAUNCH_CHECK();
    // F_1 = E T_0 = E ; D = F_1
    TC_TRY(copy_cm(b.P, b.F, NN, s));
    TC_TRY(copy_cm(b.P, D, NN, s));
    // T_1 = A' T_0 = -i B
    {
        // T1 = -i B: planes (0, -B)
        identity_kernel<<<grid_for(NN), 256, 0, s>>>(b.Tn.r, b.Tn.i, N);
        TC_LAUNCH_CHECK();
        TC_TRY(minus_i_times(N, b.B, b.Tn, b.T, b.Q, s));
        axpby_kernel<<<grid_for(NN), 256, 0, s>>>(1.0, Xs.r, Xs.i, 1.0, b.T.r, b.T.i, Xs.r, Xs.i, NN);
        TC_LAUNCH_CHECK();
    }
    for (int k = 2; k <= mt; k++) {
        // F_k = (A' F_{k-1} + E T_{k-1}) / k ;  T_k = A' T_{k-1} / k
        TC_TRY(minus_i_times(N, b.B, b.F, b.Fn, b.Q, s));                 // Fn = A' F
        TC_TRY(gemm_c(N, b.P, 0, b.T, 0, b.Fn, 1.0, 1.0, 0, s));          // Fn += E T
        TC_TRY(minus_i_times(N, b.B, b.T, b.Tn, b.Q, s));                 // Tn = A' T
        const double inv = 1.0 / k;
        axpby_kernel<<<grid_for(NN), 256, 0, s>>>(inv, b.Fn.r, b.Fn.i, 0.0, b.Fn.r, b.Fn.i, b.F.r, b.F.i, NN);
        TC_LAUNCH_CHECK();
        axpby_kernel<<<grid_for(NN), 256, 0, s>>>(inv, b.Tn.r, b.Tn.i, 0.0, b.Tn.r, b.Tn.i, b.T.r, b.T.i, NN);
        TC_LAUNCH_CHECK();
        axpby_kernel<<<grid_for(NN), 256, 0, s>>>(1.0, D.r, D.i, 1.0, b.F.r, b.F.i, D.r, D.i, NN);
        TC_LAUNCH_CHECK();
        axpby_kernel<<<grid_for(NN), 256, 0, s>>>(1.0, Xs.r, Xs.i, 1.0, b.T.r, b.T.i, Xs.r, Xs.i, NN);
        TC_LAUNCH_CHECK();
    }
    // squarings: D <- X D + D X ; X <- X X
    for (int q = 0; q < sq; q++) {
        TC_TRY(gemm_c(N, Xs, 0, D, 0, b.Fn, 1.0, 0.0, 0, s));
        TC_TRY(gemm_c(N, D, 0, Xs, 0, b.Fn, 1.0, 1.0, 0, s));
        TC_TRY(copy_cm(b.Fn, D, NN, s));
        TC_TRY(gemm_c(N, Xs, 0, Xs, 0, b.Tn, 1.0, 0.0, 0, s));
        TC_TRY(copy_cm(b.Tn, Xs, NN, s));
    }
    // G = e^{-i mu dt} D; grad_j = 2 dt Im Tr(dH_j G)
    double* gdev = b.small + 2 * (size_t)N + 16;
    contract_kernel<<<n + 2, 1024, 0, s>>>(D.r, D.i, m, dt, std::cos(mu * dt), -std::sin(mu * dt), gdev);
    TC_LAUNCH_CHECK();
    TC_CUDA(cudaMemcpyAsync(grad, gdev, sizeof(double) * (n + 2), cudaMemcpyDeviceToHost, s));
    double lv = 0.0;
    TC_CUDA(cudaMemcpyAsync(&lv, b.small, sizeof(double), cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    if (loss) *loss = lv;
    for (int j = 0; j < n + 2; j++)
        if (!std::isfinite(grad[j])) return fail(TC_ERR_NUMERIC, "non-finite gradient");
    return TC_OK;
}
