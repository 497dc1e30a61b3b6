// expm_model.cu -- U = e^{-iH dt} straight from the model (Sec. II, Eq. 4;
// Sec. III.A, Eqs. 6-7), with H applied as the structured operator it is
// (n + 1 nonzeros per row: the diagonal and one coupling per atom) instead of
// a dense matrix.
//
// With mu = Tr H / N and B = (H - mu I) dt, the Taylor polynomial of e^{-iB}
// of degree m is evaluated by Horner's rule on a complex N x N matrix T:
//     T <- I,   T <- I + (-i B) T / k   for k = m, m-1, ..., 1,
// each step one application of B to the two planes of T (a row "stencil":
// row r of B X combines row r and the n rows r xor 2^b of X), memory-bound
// and O(n N^2) instead of an O(N^3) FP64 product.  m is the smallest degree
// whose Taylor remainder bound is below 2^-53; ||B|| above 1 is scaled by
// 2^-s and squared back with dense FP64 complex products (a time step of the
// paper's size has ||B|| of a few hundredths and needs no squaring).  Then
// U = e^{-i mu dt} T, symmetrised (U = U^T).
#include <algorithm>
#include <cmath>

#include "model_dev.cuh"
#include "paths.cuh"

namespace tc {
namespace {

constexpr int kCols = 4;        // columns per thread
constexpr int kThreads = 256;   // a block covers kCols * kThreads columns of one row

// One Horner step: T' = I + (-i B) T / k with B = (H_blk - mu I) dt, planar
// d x d T.  (-i B)(T_r + i T_i) = B T_i - i B T_r.  Block (x, y) handles
// row r = x and a chunk of columns; the row's n + 1 entries of B are
// computed once into shared memory (col[b] < 0: the neighbour is outside the
// block), and every thread reads rows r and col[b] of T at its columns
// (coalesced along the row).  first: T = I, so B T = B.  Rows run along grid
// x (d reaches 2^16, above the grid-y limit).
__global__ void __launch_bounds__(kThreads) horner_step_kernel(Model m, ExcitationBlock blk, double mu, double dt,
                                                                double inv_k, const double* __restrict__ Tr,
                                                                const double* __restrict__ Ti, double* __restrict__ Or,
                                                                double* __restrict__ Oi, int first) {
    __shared__ double hb[kMaxAtoms + 1];
    __shared__ int nb[kMaxAtoms];
    const unsigned d = (unsigned)blk.d;
    const unsigned r = blockIdx.x;
    const unsigned s = blk.order ? (unsigned)blk.order[r] : r;
    if (threadIdx.x < (unsigned)m.n) {
        const unsigned t = s ^ (1u << threadIdx.x);
        const unsigned c = blk.pos ? (unsigned)blk.pos[t] : t;
        nb[threadIdx.x] = c < d ? (int)c : -1;
        hb[threadIdx.x] = c < d ? h_pair(m, blk.k, s, threadIdx.x) * dt : 0.0;
    }
    if (threadIdx.x == (unsigned)m.n) hb[m.n] = (h_diag(m, blk.k, s) - mu) * dt;
    __syncthreads();
    const double dg = hb[m.n];
    const size_t row = (size_t)r * d;
#pragma unroll
    for (int j = 0; j < kCols; j++) {
        const unsigned c = (blockIdx.y * kCols + j) * kThreads + threadIdx.x;
        if (c >= d) break;
        double br = 0.0, bi = 0.0;   // (B T_r)[r][c], (B T_i)[r][c]
        if (first) {
            if (c == r) {
                br = dg;
            } else {
                for (int b = 0; b < m.n; b++)
                    if (nb[b] == (int)c) br = hb[b];
            }
        } else {
            br = dg * Tr[row + c];
            bi = dg * Ti[row + c];
            for (int b = 0; b < m.n; b++) {
                if (nb[b] < 0) continue;
                const size_t o = (size_t)nb[b] * d + c;
                br += hb[b] * Tr[o];
                bi += hb[b] * Ti[o];
            }
        }
        Or[row + c] = (r == c ? 1.0 : 0.0) + bi * inv_k;
        Oi[row + c] = -br * inv_k;
    }
}

tc_status launch_horner(const Model& m, const ExcitationBlock& blk, double mu, double dt, double inv_k,
                        const double* Tr, const double* Ti, double* Or, double* Oi, int first, cudaStream_t s) {
    const unsigned d = (unsigned)blk.d;
    dim3 grid(d, (d + kCols * kThreads - 1) / (kCols * kThreads));
    horner_step_kernel<<<grid, kThreads, 0, s>>>(m, blk, mu, dt, inv_k, Tr, Ti, Or, Oi, first);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

int popcount_host(unsigned s) {
    int pc = 0;
    for (unsigned t = s; t; t >>= 1) pc += (int)(t & 1u);
    return pc;
}

// exact ||B||_inf = max over rows of |H_ss - mu| + sum_b |h(s, s^b)| (times dt)
// and the trace shift mu = Tr H_blk / d, on the host from the block's basis
void block_norm_and_shift(const Model& m, const ExcitationBlock& blk, const int* host_order, int shift, double dt,
                          double* norm, double* mu_out) {
    const unsigned d = (unsigned)blk.d;
    double tr = 0.0;
    for (unsigned r = 0; r < d; r++) {
        const unsigned s = host_order ? (unsigned)host_order[r] : r;
        const int pc = popcount_host(s);
        tr += m.omega_c * (double)(blk.k - pc) + m.omega_a * (double)pc;
    }
    const double mu = shift ? tr / (double)d : 0.0;
    double best = 0.0;
    for (unsigned r = 0; r < d; r++) {
        const unsigned s = host_order ? (unsigned)host_order[r] : r;
        const int pc = popcount_host(s);
        double row = std::fabs(m.omega_c * (double)(blk.k - pc) + m.omega_a * (double)pc - mu);
        for (int b = 0; b < m.n; b++) {
            const unsigned se = s | (1u << b);
            if (popcount_host(se) > blk.k) continue;   // neighbour outside the block
            const int atom0 = m.n - 1 - b;
            row += m.coupling == TC_COUPLING_QUBIT_PHOTON
                       ? std::fabs(m.g[atom0])
                       : std::fabs(m.g[atom0]) * std::sqrt((double)(blk.k - popcount_host(se) + 1));
        }
        if (row > best) best = row;
    }
    *norm = best * dt;
    *mu_out = mu;
}

}  // namespace

size_t expm_block_bytes(size_t d) {
    return 6 * round256(sizeof(double) * d * d) + 256;
}

tc_status expm_block_impl(const Model& m, const ExcitationBlock& blk, const int* host_order, double dt,
                          const tc_expm_opts* opts, double* U, Arena& ar, cudaStream_t s, int* used_degree,
                          int* used_squarings) {
    const int N = blk.d;
    const size_t NN = (size_t)N * N;
    double* P[4];
    for (int k = 0; k < 4; k++) P[k] = ar.take<double>(NN);
    double* Q[2] = {ar.take<double>(NN), ar.take<double>(NN)};
    if (!Q[1]) return fail(TC_ERR_WORKSPACE, "expm_model: workspace too small");
    const int shift = opts ? opts->shift : 1;
    double bn = 0.0, mu = 0.0;   // ||B||_inf, Tr H / d
    block_norm_and_shift(m, blk, host_order, shift, dt, &bn, &mu);
    const double u = std::ldexp(1.0, -53);
    // smallest degree whose Taylor remainder bound b^{m+1}/(m+1)! / (1 - b/(m+2))
    // is below 2^-53 / 2^s (errors double with each squaring); 0 if above 64
    auto degree_for = [&](double b, int sqr) -> int {
        if (b == 0.0) return 1;
        double term = 1.0;
        for (int k = 1; k <= 65; k++) {
            term *= b / k;   // b^k / k!
            if (b < k + 1 && term / (1.0 - b / (k + 1)) <= std::ldexp(u, -sqr)) return k - 1 > 1 ? k - 1 : 1;
        }
        return 0;
    };
    // scale until ||B|| / 2^s <= 1: Horner's intermediate sums of a Taylor
    // series at b carry rounding of order u e^b, so larger b loses digits to
    // cancellation (e^b u at b = 8 is already 3e-13)
    int sq = 0;
    if (opts && opts->squarings >= 0) {
        sq = opts->squarings;
    } else {
        while (sq < 40 && std::ldexp(bn, -sq) > 1.0) sq++;
    }
    int deg = opts && opts->taylor_degree > 0 ? opts->taylor_degree : degree_for(std::ldexp(bn, -sq), sq);
    if (deg == 0) deg = 64;
    if (used_degree) *used_degree = deg;
    if (used_squarings) *used_squarings = sq;
    const double dts = std::ldexp(dt, -sq);

    // Horner: T_m = I + (-iB) I / m, then T = I + (-iB) T / k down to k = 1
    double *Tr = P[0], *Ti = P[1], *Or = P[2], *Oi = P[3];
    TC_TRY(launch_horner(m, blk, mu, dts, 1.0 / deg, nullptr, nullptr, Tr, Ti, 1, s));
    for (int k = deg - 1; k >= 1; k--) {
        TC_TRY(launch_horner(m, blk, mu, dts, 1.0 / k, Tr, Ti, Or, Oi, 0, s));
        std::swap(Tr, Or);
        std::swap(Ti, Oi);
    }
    // squarings (dense FP64 complex products), only for large ||B||
    for (int q = 0; q < sq; q++) {
        GemmF64 g{};
        g.M = g.N = g.K = N;
        g.Ar = Tr; g.Ai = Ti; g.lda = N;
        g.Br = Tr; g.Bi = Ti; g.ldb = N;
        g.Cr = Or; g.Ci = Oi; g.ldc = N;
        g.alpha = 1.0; g.cplx = 1;
        TC_TRY(gemm_f64(g, s));
        std::swap(Tr, Or);
        std::swap(Ti, Oi);
    }
    // U = e^{-i mu dt} (C - i S) with C = T_r, S = -T_i, symmetrised
    const double* mats[1] = {Ti};
    const double coef[1] = {-1.0};
    TC_TRY(launch_lincomb(N, 0.0, 1, mats, coef, Q[0], s));
    return launch_expm_finish(N, Tr, Q[0], std::cos(mu * dt), -std::sin(mu * dt), U, s);
}

size_t expm_model_bytes(int n) {
    return expm_block_bytes((size_t)1 << n);
}

tc_status expm_model_impl(const Model& m, double dt, const tc_expm_opts* opts, double* U, Arena& ar,
                          cudaStream_t s, int* used_degree, int* used_squarings) {
    ExcitationBlock blk{m.n, 1 << m.n, nullptr, nullptr};
    return expm_block_impl(m, blk, nullptr, dt, opts, U, ar, s, used_degree, used_squarings);
}

}  // namespace tc

using namespace tc;

extern "C" TC_API tc_status tc_expm_model(const tc_params* params, double dt, const tc_expm_opts* opts, void* U,
                                          void* work, size_t work_bytes, void* stream) {
    Model m;
    TC_TRY(make_model(params, &m));
    if (!U) return fail(TC_ERR_INVALID_ARG, "U is NULL");
    if (reinterpret_cast<uintptr_t>(U) & 15u) return fail(TC_ERR_INVALID_ARG, "U must be 16-byte aligned");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(TC_ERR_INVALID_ARG, "dt must be finite and > 0");
    if (opts && (opts->taylor_degree < 0 || opts->taylor_degree > 64 || opts->squarings < -1 || opts->squarings > 40))
        return fail(TC_ERR_INVALID_ARG, "expm opts out of range");
    const size_t need = expm_model_bytes(m.n);
    if (!work) return fail(TC_ERR_WORKSPACE, "work is NULL (need %zu bytes)", need);
    if (reinterpret_cast<uintptr_t>(work) & 255u) return fail(TC_ERR_WORKSPACE, "work is not 256-byte aligned");
    if (work_bytes < need) return fail(TC_ERR_WORKSPACE, "work has %zu bytes, need %zu", work_bytes, need);
    TC_TRY(check_device());
    Arena ar{static_cast<char*>(work), work_bytes, 0};
    return expm_model_impl(m, dt, opts, static_cast<double*>(U), ar, as_stream(stream), nullptr, nullptr);
}
