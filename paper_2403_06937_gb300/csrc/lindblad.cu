// lindblad.cu -- the open-system form of the evolution: the quantum master
// equation of Sec. III.A (Eq. 5) with its Lindblad term switched on.  The
// paper names the term and sets it to zero; the term used here is photon
// leakage from the cavity at rate kappa,
//     L(rho) = kappa (a rho a^dag - {a^dag a, rho} / 2).
//
// Structure.  H conserves the excitation number k = popcount(s) + p and a
// leaked photon lowers it by one, so a state that starts inside one k stays
// block diagonal: rho = sum_k rho_k, block k living on the d_k atom strings
// with popcount(s) <= k (photon count k - popcount(s)).  With the strings
// ordered by popcount (then value), block k's basis is the first d_k strings
// of one common order, so element (i, j) means the same pair of strings in
// every block that holds it.  Blocks are stored packed, k = 0..n.
//
// One step of length dt is the symmetric split
//     rho <- D_{dt/2}( U rho U^dag ), after rho <- D_{dt/2}(rho),
// with U = e^{-iH dt} block by block (each U_k complex symmetric, so the two
// products are those of the closed form, Eq. 12) and D_tau the exact
// solution of the damping part alone (the bosonic pure-loss channel):
//     rho_k'(i, j) = sum_m F[p][m] F[q][m] rho_{k+m}(i, j),
//     F[p][m] = sqrt((1 - eta)^m / m! * (p + m)! / p!) * eta^{p/2},
// eta = e^{-kappa tau}, p and q the photon counts of strings i and j in
// block k.  D_tau is one HBM-bound pass over all blocks; the products are
// dense complex GEMMs per block: the FP64 DMMA GEMM block by block, or, in
// the tensor-core forms, one persistent launch over the tiles of every block
// per product (the batch GEMM, blocks zero-padded to multiples of 128, U_k in
// increment form, rho_k in FP32 planes plus operand parts), with D_tau then
// reading and writing the FP32 planes and rebuilding the parts.  The
// FP64-emulated form (exact digit slices on the BF16 tensor cores) steps the
// blocks one after another on FP64 planes padded to multiples of 128.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "cgemm_batch.cuh"
#include "cgemm_oz.cuh"
#include "cgemm_tc.cuh"
#include "graph.cuh"
#include "lowp.cuh"
#include "model_dev.cuh"
#include "paths.cuh"
#include "timing.cuh"

namespace tc {
namespace {

int popcount_host(unsigned s) {
    int pc = 0;
    for (unsigned t = s; t; t >>= 1) pc += (int)(t & 1u);
    return pc;
}

struct Layout {
    int n = 0;
    int N = 0;
    int dims[kMaxAtoms + 1] = {};
    size_t off[kMaxAtoms + 2] = {};   // element offsets of the blocks; off[n + 1] = total
    std::vector<int> order;           // strings by popcount, then value
};

const Layout& layout_of(int n) {
    static std::mutex mu;
    static Layout* cache[kMaxAtoms + 1] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (!cache[n]) {
        Layout* L = new Layout;   // kept for the life of the process
        L->n = n;
        L->N = 1 << n;
        L->order.resize(L->N);
        for (int s = 0; s < L->N; s++) L->order[s] = s;
        std::stable_sort(L->order.begin(), L->order.end(),
                         [](int a, int b) { return popcount_host((unsigned)a) < popcount_host((unsigned)b); });
        for (int k = 0; k <= n; k++) {
            int d = 0;
            for (int s = 0; s < L->N; s++) d += popcount_host((unsigned)s) <= k;
            L->dims[k] = d;
            L->off[k + 1] = L->off[k] + (size_t)d * d;
        }
        cache[n] = L;
    }
    return *cache[n];
}

// Block dimensions, row strides and plane offsets by value, for kernels.
// FP64 packed planes: ld = d, off = the packed offsets.  FP32 planes of the
// tensor-core forms: ld = Np (d rounded up to 128), off = sum of Np^2.
struct BlockSet {
    int n;
    int d[kMaxAtoms + 1];
    int ld[kMaxAtoms + 1];
    unsigned long long off[kMaxAtoms + 1];
    int cum[kMaxAtoms + 2];   // number of strings with popcount < c
};

int padded(int d) { return d < 128 ? 128 : (d + 127) / 128 * 128; }

BlockSet block_set(const Layout& L, bool pad = false) {
    BlockSet b{};
    b.n = L.n;
    unsigned long long o = 0;
    for (int k = 0; k <= L.n; k++) {
        b.d[k] = L.dims[k];
        b.ld[k] = pad ? padded(L.dims[k]) : L.dims[k];
        b.off[k] = pad ? o : (unsigned long long)L.off[k];
        o += (unsigned long long)b.ld[k] * b.ld[k];
    }
    b.cum[0] = 0;
    for (int c = 0; c <= L.n; c++) b.cum[c + 1] = L.dims[c];
    return b;
}

size_t padded_total(const Layout& L) {
    size_t t = 0;
    for (int k = 0; k <= L.n; k++) t += (size_t)padded(L.dims[k]) * padded(L.dims[k]);
    return t;
}

// Operand-part planes of each block (tensor-core forms): [2 S][Np][Np].
struct PartsSet {
    void* p[kMaxAtoms + 1];
};

// Position of string s in the popcount order: the strings of smaller popcount,
// plus the rank of s among strings of its popcount in increasing value, which
// is the combinatorial number system sum_t C(b_t, t) over its set bits
// b_1 < b_2 < ... (t from 1).
__global__ void layout_kernel(BlockSet bs, int* __restrict__ order, int* __restrict__ pos) {
    const unsigned N = 1u << bs.n;
    for (unsigned s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        unsigned rank = 0;
        int t = 0;
        for (int b = 0; b < bs.n; b++) {
            if (!((s >> b) & 1u)) continue;
            t++;
            unsigned c = 1;   // C(b, t)
            for (int q = 1; q <= t; q++) c = c * (unsigned)(b - t + q) / (unsigned)q;
            rank += b >= t ? c : 0u;
        }
        const unsigned p = (unsigned)bs.cum[__popc(s)] + rank;
        pos[s] = (int)p;
        order[p] = (int)s;
    }
}

template <typename A>
struct DampTable {
    A F[kMaxAtoms + 1][kMaxAtoms + 1];   // F[p][m]
};

// F[p][m] = sqrt(C(p + m, m) (1 - eta)^m) eta^{p/2}, evaluated in FP64 and
// stored in the arithmetic type of the pass
template <typename A>
DampTable<A> damp_table(int n, double kappa, double tau) {
    DampTable<A> t{};
    const double eta = std::exp(-kappa * tau);
    const double loss = -std::expm1(-kappa * tau);   // 1 - eta without cancellation
    for (int p = 0; p <= n; p++) {
        for (int m = 0; p + m <= n; m++) {
            double ratio = 1.0;   // (p + m)! / p! / m!  =  C(p + m, m)
            for (int q = 1; q <= m; q++) ratio = ratio * (double)(p + q) / (double)q;
            t.F[p][m] = (A)(std::sqrt(ratio * std::pow(loss, (double)m)) * std::pow(eta, 0.5 * (double)p));
        }
    }
    return t;
}

// D_tau on all blocks in place.  Block x = row i of every block; threads run
// along j (coalesced in each block; consecutive positions mostly share a
// popcount, so the block range below is nearly warp-uniform).  Element (i, j)
// is in blocks k >= max(level(i), level(j)); the new block-k value needs the
// old values of blocks >= k only, so ascending k can overwrite in place.
// The arithmetic is that of the storage: FP64 for the FP64 form; FP32 for
// the FP32 planes of the tensor-core forms (about (n + 2) 2^-24 relative per
// pass, the order of the FP32 store itself; FP64 arithmetic here would make
// the pass FP64-issue-bound), which with S > 0 also rebuild the operand parts.
template <typename T, int KIND, int S>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) damping_kernel(BlockSet bs, DampTable<T> t, const int* __restrict__ order,
                                                      T* __restrict__ re, T* __restrict__ im, PartsSet ps) {
    const int n = bs.n;
    const unsigned N = 1u << n;
    const unsigned i = blockIdx.x;
    const int li = __popc((unsigned)order[i]);
    for (unsigned j = blockIdx.y * blockDim.x + threadIdx.x; j < N; j += gridDim.y * blockDim.x) {
        const int lj = __popc((unsigned)order[j]);
        const int k0 = li > lj ? li : lj;
        T vr[kMaxAtoms + 1], vi[kMaxAtoms + 1];
#pragma unroll
        for (int k = 0; k <= kMaxAtoms; k++) {
            vr[k] = 0;
            vi[k] = 0;
            if (k >= k0 && k <= n) {
                const size_t o = bs.off[k] + (size_t)i * bs.ld[k] + j;
                vr[k] = re[o];
                vi[k] = im[o];
            }
        }
#pragma unroll
        for (int k = 0; k <= kMaxAtoms; k++) {
            if (k < k0 || k > n) continue;
            const int p = k - li, q = k - lj;
            T ar = 0, ai = 0;
#pragma unroll
            for (int m = 0; m + k <= kMaxAtoms; m++) {
                if (k + m > n) break;
                const T c = t.F[p][m] * t.F[q][m];
                ar += c * vr[k + m];
                ai += c * vi[k + m];
            }
            const size_t idx = (size_t)i * bs.ld[k] + j;
            const size_t o = bs.off[k] + idx;
            re[o] = ar;
            im[o] = ai;
            if constexpr (S > 0) {
                const size_t plane = (size_t)bs.ld[k] * bs.ld[k];
                split_f32<KIND, S>((float)ar, ps.p[k], plane, idx, 0);
                split_f32<KIND, S>((float)ai, ps.p[k], plane, idx, 1);
            }
        }
    }
}

// Trace over all blocks in FP64, one CTA, fixed order.
template <typename T>
__global__ void block_trace_kernel(BlockSet bs, const T* __restrict__ re, double* __restrict__ out) {
    __shared__ double sh[1024];
    double a = 0.0;
    for (int k = 0; k <= bs.n; k++)
        for (int i = threadIdx.x; i < bs.d[k]; i += blockDim.x)
            a += (double)re[bs.off[k] + (size_t)i * bs.ld[k] + i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

// rho <- rho / Tr rho on every block (grid y = block); parts rebuilt when S > 0.
template <typename T, int KIND, int S>
__global__ void block_rescale_kernel(BlockSet bs, T* __restrict__ re, T* __restrict__ im, PartsSet ps,
                                     const double* __restrict__ trace, unsigned* status) {
    const double tr = trace[0];
    if (!(tr > 0.0) || !isfinite(tr)) {
        if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) atomicOr(status, kStatusNumeric);
        return;
    }
    const double inv = 1.0 / tr;
    const int k = blockIdx.y;
    const size_t d = (size_t)bs.d[k], ld = (size_t)bs.ld[k];
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += (size_t)gridDim.x * blockDim.x) {
        const size_t idx = (e / d) * ld + e % d;
        const size_t o = bs.off[k] + idx;
        const T wr = (T)((double)re[o] * inv), wi = (T)((double)im[o] * inv);
        re[o] = wr;
        im[o] = wi;
        if constexpr (S > 0) {
            split_f32<KIND, S>((float)wr, ps.p[k], ld * ld, idx, 0);
            split_f32<KIND, S>((float)wi, ps.p[k], ld * ld, idx, 1);
        }
    }
}

// Observable row over all blocks, deterministic: one warp per row of one
// block (rows of all blocks enumerated block by block), per-CTA partials in a
// fixed order, then one CTA sums the partials.
constexpr int kObsWarps = 8;
constexpr int kMaxStride = 2 * kMaxAtoms + 5;

unsigned obs_grid(const Layout& L) {
    size_t rows = 0;
    for (int k = 0; k <= L.n; k++) rows += (size_t)L.dims[k];
    size_t g = (rows + kObsWarps - 1) / kObsWarps;
    return (unsigned)(g > 1024 ? 1024 : g);
}

template <typename T>
__global__ void obs_partial_kernel(BlockSet bs, Model m, int has_model, const int* __restrict__ order,
                                   const int* __restrict__ pos, const T* __restrict__ re, const T* __restrict__ im,
                                   double* __restrict__ partials) {
    __shared__ double acc[kObsWarps][kMaxStride];
    const int n = bs.n;
    const int stride = 2 * n + 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = lane; j < stride; j += 32) acc[warp][j] = 0.0;
    __syncwarp();
    unsigned rows = 0;
    for (int k = 0; k <= n; k++) rows += (unsigned)bs.d[k];
    double pur = 0.0, epair = 0.0;
    for (unsigned q = blockIdx.x * kObsWarps + warp; q < rows; q += gridDim.x * kObsWarps) {
        int k = 0;
        unsigned i = q;
        while (i >= (unsigned)bs.d[k]) {
            i -= (unsigned)bs.d[k];
            k++;
        }
        const unsigned d = (unsigned)bs.d[k];
        const size_t row = bs.off[k] + (size_t)i * bs.ld[k];
        // four independent loads per lane in flight, fixed summation order
        double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
        unsigned c = lane;
        if constexpr (std::is_same<T, float>::value) {
            // FP32 planes: the squares of each group of four entries summed in FP32
            // (fused multiply-adds), the group sums carried in FP64 (GB300 issues FP64
            // at a small fraction of its FP32 rate)
            for (; c + 96 < d; c += 128) {
                const float x0 = re[row + c], x1 = re[row + c + 32], x2 = re[row + c + 64], x3 = re[row + c + 96];
                const float y0 = im[row + c], y1 = im[row + c + 32], y2 = im[row + c + 64], y3 = im[row + c + 96];
                const float q01 = fmaf(y1, y1, fmaf(x1, x1, fmaf(y0, y0, x0 * x0)));
                const float q23 = fmaf(y3, y3, fmaf(x3, x3, fmaf(y2, y2, x2 * x2)));
                p0 += (double)q01;
                p2 += (double)q23;
            }
            for (; c < d; c += 32) {
                const float x = re[row + c], y = im[row + c];
                p1 += (double)fmaf(y, y, x * x);
            }
        } else {
            for (; c + 96 < d; c += 128) {
                const double x0 = (double)re[row + c], x1 = (double)re[row + c + 32], x2 = (double)re[row + c + 64],
                             x3 = (double)re[row + c + 96];
                const double y0 = (double)im[row + c], y1 = (double)im[row + c + 32], y2 = (double)im[row + c + 64],
                             y3 = (double)im[row + c + 96];
                p0 += x0 * x0 + y0 * y0;
                p1 += x1 * x1 + y1 * y1;
                p2 += x2 * x2 + y2 * y2;
                p3 += x3 * x3 + y3 * y3;
            }
            for (; c < d; c += 32) {
                const double x = (double)re[row + c], y = (double)im[row + c];
                p0 += x * x + y * y;
            }
        }
        pur += (p0 + p1) + (p2 + p3);
        const unsigned s = (unsigned)order[i];
        if (has_model && lane < n) {
            const unsigned c = (unsigned)pos[s ^ (1u << lane)];
            if (c < d) epair += h_pair(m, k, s, lane) * (double)re[row + c];
        }
        if (lane == 0) {
            const double v = (double)re[row + i];
            const int pc = __popc(s), p = k - pc;
            for (int a = 0; a < n; a++)
                if ((s >> (n - 1 - a)) & 1u) acc[warp][a] += v;
            acc[warp][n] += v * (double)p;
            acc[warp][n + 1 + p] += v;
            acc[warp][2 * n + 2] += v;
            if (has_model) acc[warp][2 * n + 4] += h_diag(m, k, s) * v;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        pur += __shfl_xor_sync(0xffffffffu, pur, o);
        epair += __shfl_xor_sync(0xffffffffu, epair, o);
    }
    if (lane == 0) {
        acc[warp][2 * n + 3] += pur;
        acc[warp][2 * n + 4] += epair;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < stride; j += blockDim.x) {
        double sum = 0.0;
        for (int w = 0; w < kObsWarps; w++) sum += acc[w][j];
        partials[(size_t)blockIdx.x * stride + j] = sum;
    }
}

__global__ void obs_final_kernel(const double* __restrict__ partials, int blocks, int stride,
                                 double* __restrict__ out) {
    for (int j = threadIdx.x; j < stride; j += blockDim.x) {
        double sum = 0.0;
        for (int b = 0; b < blocks; b++) sum += partials[(size_t)b * stride + j];
        out[j] = sum;
    }
}

struct Tables {
    int* order;
    int* pos;
};

tc_status take_tables(const Layout& L, Arena& ar, Tables* t) {
    t->order = ar.take<int>((size_t)L.N);
    t->pos = ar.take<int>((size_t)L.N);
    if (!t->pos) return fail(TC_ERR_WORKSPACE, "lindblad: workspace too small");
    return TC_OK;
}

tc_status launch_layout(const Layout& L, const Tables& t, cudaStream_t s) {
    const unsigned blocks = (unsigned)((L.N + 255) / 256);
    layout_kernel<<<blocks, 256, 0, s>>>(block_set(L), t.order, t.pos);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

template <typename T, int KIND, int S>
tc_status launch_damping(const Layout& L, const BlockSet& bs, double kappa, double tau, const Tables& t, T* re, T* im,
                         const PartsSet& ps, cudaStream_t s) {
    dim3 grid((unsigned)L.N, (unsigned)((L.N + 255) / 256));
    damping_kernel<T, KIND, S><<<grid, 256, 0, s>>>(bs, damp_table<T>(L.n, kappa, tau), t.order, re, im, ps);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

template <typename T, int KIND, int S>
tc_status launch_block_renorm(const Layout& L, const BlockSet& bs, T* re, T* im, const PartsSet& ps, double* scratch,
                              cudaStream_t s) {
    block_trace_kernel<T><<<1, 1024, 0, s>>>(bs, re, scratch);
    TC_LAUNCH_CHECK();
    dim3 grid(256, (unsigned)(L.n + 1));
    block_rescale_kernel<T, KIND, S><<<grid, 256, 0, s>>>(bs, re, im, ps, scratch, device_status_word());
    TC_LAUNCH_CHECK();
    return TC_OK;
}

size_t obs_scratch_bytes(const Layout& L) {
    return round256((size_t)obs_grid(L) * (2 * L.n + 5) * sizeof(double)) + 256;
}

template <typename T>
tc_status launch_block_observables(const Layout& L, const BlockSet& bs, const Model& m, const Tables& t, const T* re,
                                   const T* im, double* out, double* scratch, cudaStream_t s) {
    const unsigned grid = obs_grid(L);
    obs_partial_kernel<T><<<grid, 32 * kObsWarps, 0, s>>>(bs, m, 1, t.order, t.pos, re, im, scratch);
    TC_LAUNCH_CHECK();
    obs_final_kernel<<<1, 64, 0, s>>>(scratch, (int)grid, 2 * L.n + 5, out);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

size_t tables_bytes(int n) {
    return 2 * round256(sizeof(int) << n);
}

size_t propagators_bytes(int n) {
    return tables_bytes(n) + expm_block_bytes((size_t)1 << n) + 256;
}

size_t evolve_f64_bytes(int n) {
    const Layout& L = layout_of(n);
    const size_t total = L.off[n + 1];
    const size_t NN = (size_t)L.N * L.N;
    return tables_bytes(n) + 4 * round256(total * sizeof(double)) + 2 * round256(NN * sizeof(double)) +
           obs_scratch_bytes(L) + gemm_f64_splitk_bytes() + 256;
}

tc_status evolve_f64(const Layout& L, const Model& m, double kappa, double dt, const double* U, double* rho,
                     int steps, int renorm_every, double* obs, Arena& ar, cudaStream_t s) {
    const int n = L.n;
    const size_t total = L.off[n + 1];
    const size_t NN = (size_t)L.N * L.N;
    Tables t{};
    TC_TRY(take_tables(L, ar, &t));
    double* Ur = ar.take<double>(total);
    double* Ui = ar.take<double>(total);
    double* Rr = ar.take<double>(total);
    double* Ri = ar.take<double>(total);
    double* Xr = ar.take<double>(NN);
    double* Xi = ar.take<double>(NN);
    double* scratch = ar.take<double>(obs_scratch_bytes(L) / sizeof(double));
    double* partial = ar.take<double>(gemm_f64_splitk_bytes() / sizeof(double));
    if (!partial) return fail(TC_ERR_WORKSPACE, "lindblad evolve: workspace too small");
    const int stride = TC_OBS_STRIDE(n);
    const bool damp = kappa > 0.0;
    const BlockSet bs = block_set(L);
    const PartsSet none{};

    auto products = [&](cudaStream_t cs) -> tc_status {
        for (int k = 0; k <= n; k++) {
            const int d = L.dims[k];
            const size_t o = L.off[k];
            GemmF64 g1{};
            g1.M = g1.N = g1.K = d;
            g1.Ar = Ur + o; g1.Ai = Ui + o; g1.lda = d;
            g1.Br = Rr + o; g1.Bi = Ri + o; g1.ldb = d;
            g1.Cr = Xr; g1.Ci = Xi; g1.ldc = d;
            g1.alpha = 1.0;
            g1.cplx = 1;
            g1.partial = partial;   // used by the blocks of dimension <= 1024
            GemmF64 g2 = g1;
            g2.Ar = Xr; g2.Ai = Xi;
            g2.Br = Ur + o; g2.Bi = Ui + o; g2.conjB = 1;
            g2.Cr = Rr + o; g2.Ci = Ri + o;
            g2.herm_lower = 1;
            const double d3 = (double)d * d * d;
            {
                ProductTimer pt(8.0 * d3, cs);   // X = U_k rho_k
                TC_TRY(gemm_f64(g1, cs));
            }
            {
                ProductTimer pt(4.0 * d3, cs);   // rho_k = X U_k^dag, Hermitian half
                TC_TRY(gemm_f64(g2, cs));
            }
        }
        return TC_OK;
    };
    auto one_step = [&](int k, cudaStream_t cs) -> tc_status {
        if (damp) TC_TRY((launch_damping<double, 0, 0>(L, bs, kappa, 0.5 * dt, t, Rr, Ri, none, cs)));
        TC_TRY(products(cs));
        if (damp) TC_TRY((launch_damping<double, 0, 0>(L, bs, kappa, 0.5 * dt, t, Rr, Ri, none, cs)));
        if (renorm_every > 0 && k % renorm_every == 0)
            TC_TRY((launch_block_renorm<double, 0, 0>(L, bs, Rr, Ri, none, scratch, cs)));
        if (obs) TC_TRY(launch_block_observables<double>(L, bs, m, t, Rr, Ri, obs + (size_t)k * stride, scratch, cs));
        return TC_OK;
    };
    auto first = [&](cudaStream_t cs) -> tc_status {
        TC_TRY(launch_layout(L, t, cs));
        TC_TRY(launch_split_c128(U, Ur, Ui, total, cs));
        TC_TRY(launch_split_c128(rho, Rr, Ri, total, cs));
        if (obs) TC_TRY(launch_block_observables<double>(L, bs, m, t, Rr, Ri, obs, scratch, cs));
        if (steps >= 1) TC_TRY(one_step(1, cs));
        return TC_OK;
    };
    auto rest = [&](cudaStream_t cs) -> tc_status {
        for (int k = 2; k <= steps; k++) TC_TRY(one_step(k, cs));
        return TC_OK;
    };
    auto tail = [&](cudaStream_t cs) -> tc_status { return launch_join_c128(Rr, Ri, rho, total, cs); };
    return run_captured(s, first, rest, tail, steps > 2 && !timing_enabled());
}

// ---------------------------------------------------------------- tensor-core forms
size_t evolve_lowp_bytes_blocks(int n, int precision) {
    const Layout& L = layout_of(n);
    const int S = cgemm_parts(precision);
    const size_t E = cgemm_elem_bytes(precision);
    size_t b = tables_bytes(n) + round256(sizeof(BatchSys) * (n + 1)) + 256;
    for (int k = 0; k <= n; k++) b += 3 * (size_t)(2 * S) * plane_bytes(padded(L.dims[k]), E);
    b += 4 * round256(padded_total(L) * sizeof(float));
    return b + obs_scratch_bytes(L) + 256;
}

template <int KIND, int S>
tc_status evolve_lowp_t(const Layout& L, const Model& m, int precision, double kappa, double dt, const double* U,
                        double* rho, int steps, int renorm_every, double* obs, Arena& ar, cudaStream_t s) {
    const int n = L.n;
    const size_t E = cgemm_elem_bytes(precision);
    const size_t PT = padded_total(L);
    Tables t{};
    TC_TRY(take_tables(L, ar, &t));
    BatchSys* sys_dev = ar.take<BatchSys>((size_t)(n + 1));
    float* Rr = ar.take<float>(PT);
    float* Ri = ar.take<float>(PT);
    float* Xr = ar.take<float>(PT);
    float* Xi = ar.take<float>(PT);
    PartsSet up{}, rp{}, xp{};
    for (int k = 0; k <= n; k++) {
        const size_t pb = (size_t)(2 * S) * plane_bytes(padded(L.dims[k]), E);
        up.p[k] = ar.take<uint8_t>(pb);
        rp.p[k] = ar.take<uint8_t>(pb);
        xp.p[k] = ar.take<uint8_t>(pb);
    }
    double* scratch = ar.take<double>(obs_scratch_bytes(L) / sizeof(double));
    if (!scratch) return fail(TC_ERR_WORKSPACE, "lindblad evolve: workspace too small");
    const BlockSet bs = block_set(L, true);
    const int stride = TC_OBS_STRIDE(n);
    const bool damp = kappa > 0.0;
    unsigned* status = device_status_word();

    // descriptors, blocks in decreasing size (the longest tiles first)
    std::vector<BatchSys> host(n + 1);
    // the tile shape and raster group the autotuner chose for the whole space's n
    BatchPlan plan = batch_plan(precision, n);
    double flops = 0.0;
    for (int q = 0; q <= n; q++) {
        const int k = n - q;
        const int Np = bs.ld[k];
        BatchSys& h = host[q];
        std::memset(&h, 0, sizeof(h));
        TC_TRY(batch_plan_add(plan, h, precision, Np, up.p[k], rp.p[k], xp.p[k]));
        h.Rr = Rr + bs.off[k];
        h.Ri = Ri + bs.off[k];
        h.Rparts = rp.p[k];
        h.Xr = Xr + bs.off[k];
        h.Xi = Xi + bs.off[k];
        h.Xparts = xp.p[k];
        flops += 12.0 * (double)L.dims[k] * L.dims[k] * L.dims[k];
    }
    const double prod = (double)cgemm_products(precision);

    auto one_step = [&](int k, cudaStream_t cs) -> tc_status {
        if (damp) TC_TRY((launch_damping<float, KIND, S>(L, bs, kappa, 0.5 * dt, t, Rr, Ri, rp, cs)));
        {
            ProductTimer pt(flops * prod * (8.0 / 12.0), cs);   // X_k = U_k rho_k, every block
            TC_TRY(cgemm_batch(precision, 0, sys_dev, n + 1, plan, status, cs));
        }
        {
            ProductTimer pt(flops * prod * (4.0 / 12.0), cs);   // rho_k = X_k U_k^dag, Hermitian halves
            TC_TRY(cgemm_batch(precision, 1, sys_dev, n + 1, plan, status, cs));
        }
        if (damp) TC_TRY((launch_damping<float, KIND, S>(L, bs, kappa, 0.5 * dt, t, Rr, Ri, rp, cs)));
        if (renorm_every > 0 && k % renorm_every == 0)
            TC_TRY((launch_block_renorm<float, KIND, S>(L, bs, Rr, Ri, rp, scratch, cs)));
        if (obs) TC_TRY(launch_block_observables<float>(L, bs, m, t, Rr, Ri, obs + (size_t)k * stride, scratch, cs));
        return TC_OK;
    };
    auto block_bufs = [&](int k) {
        LowpBufs b{};
        b.N = L.dims[k];
        b.Np = bs.ld[k];
        b.S = S;
        b.E = E;
        b.Uparts = up.p[k];
        b.Rr = Rr + bs.off[k];
        b.Ri = Ri + bs.off[k];
        b.Rparts = rp.p[k];
        b.Xr = Xr + bs.off[k];
        b.Xi = Xi + bs.off[k];
        b.Xparts = xp.p[k];
        b.scratch = scratch;
        return b;
    };
    auto first = [&](cudaStream_t cs) -> tc_status {
        TC_CUDA(cudaMemcpyAsync(sys_dev, host.data(), sizeof(BatchSys) * (n + 1), cudaMemcpyHostToDevice, cs));
        TC_CUDA(cudaStreamSynchronize(cs));   // the host copy of the descriptors may go
        TC_TRY(launch_layout(L, t, cs));
        for (int k = 0; k <= n; k++) {
            LowpBufs b = block_bufs(k);
            TC_TRY(lowp_prep(precision, U + 2 * L.off[k], rho + 2 * L.off[k], b, cs));
        }
        if (obs) TC_TRY(launch_block_observables<float>(L, bs, m, t, Rr, Ri, obs, scratch, cs));
        if (steps >= 1) TC_TRY(one_step(1, cs));
        return TC_OK;
    };
    auto rest = [&](cudaStream_t cs) -> tc_status {
        for (int k = 2; k <= steps; k++) TC_TRY(one_step(k, cs));
        return TC_OK;
    };
    auto tail = [&](cudaStream_t cs) -> tc_status {
        for (int k = 0; k <= n; k++) TC_TRY(lowp_finish(block_bufs(k), rho + 2 * L.off[k], cs));
        return TC_OK;
    };
    return run_captured(s, first, rest, tail, steps > 2 && !timing_enabled());
}

tc_status evolve_lowp_blocks(const Layout& L, const Model& m, int precision, double kappa, double dt,
                             const double* U, double* rho, int steps, int renorm_every, double* obs, Arena& ar,
                             cudaStream_t s) {
    switch (precision) {
        case TC_BF16X3:
            return evolve_lowp_t<0, 3>(L, m, precision, kappa, dt, U, rho, steps, renorm_every, obs, ar, s);
        case TC_TF32:
            return evolve_lowp_t<1, 1>(L, m, precision, kappa, dt, U, rho, steps, renorm_every, obs, ar, s);
        case TC_TF32X3:
            return evolve_lowp_t<1, 2>(L, m, precision, kappa, dt, U, rho, steps, renorm_every, obs, ar, s);
    }
    return fail(TC_ERR_INVALID_ARG, "unknown precision %d", precision);
}

// ---------------------------------------------------------------- FP64 emulated on BF16
// packed interleaved blocks <-> FP64 planes padded to Np_k (grid y = block)
__global__ void blocks_split_pad_kernel(BlockSet bs, BlockSet pk, const double2* __restrict__ src,
                                        double* __restrict__ re, double* __restrict__ im) {
    const int k = blockIdx.y;
    const size_t d = (size_t)bs.d[k], ld = (size_t)bs.ld[k];
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < ld * ld; e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = e / ld, j = e % ld;
        double2 v = make_double2(0.0, 0.0);
        if (i < d && j < d) v = src[pk.off[k] + i * d + j];
        re[bs.off[k] + e] = v.x;
        im[bs.off[k] + e] = v.y;
    }
}

__global__ void blocks_join_pad_kernel(BlockSet bs, BlockSet pk, const double* __restrict__ re,
                                       const double* __restrict__ im, double2* __restrict__ dst) {
    const int k = blockIdx.y;
    const size_t d = (size_t)bs.d[k], ld = (size_t)bs.ld[k];
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = e / d, j = e % d;
        dst[pk.off[k] + e] = make_double2(re[bs.off[k] + i * ld + j], im[bs.off[k] + i * ld + j]);
    }
}

size_t evolve_oz_bytes_blocks(int n) {
    const Layout& L = layout_of(n);
    const size_t PT = padded_total(L);
    const int NpMax = padded(L.N);
    size_t b = tables_bytes(n) + 2 * round256(PT * sizeof(double));
    for (int k = 0; k <= n; k++) b += oz_mat_bytes(padded(L.dims[k]));   // U_k slices
    b += oz_mat_bytes(NpMax);                                             // B operand slices
    b += 4 * round256((size_t)NpMax * NpMax * sizeof(double));            // X planes, int64 scratch
    return b + obs_scratch_bytes(L) + 256;
}

tc_status evolve_oz_blocks(const Layout& L, const Model& m, double kappa, double dt, const double* U, double* rho,
                           int steps, int renorm_every, double* obs, Arena& ar, cudaStream_t s) {
    const int n = L.n;
    const size_t PT = padded_total(L);
    const int NpMax = padded(L.N);
    const size_t NN = (size_t)NpMax * NpMax;
    Tables t{};
    TC_TRY(take_tables(L, ar, &t));
    double* Rr = ar.take<double>(PT);
    double* Ri = ar.take<double>(PT);
    std::vector<OzMat> Uk(n + 1);
    for (int k = 0; k <= n; k++) TC_TRY(oz_mat_init(Uk[k], ar, padded(L.dims[k])));
    OzMat Bmax{};
    TC_TRY(oz_mat_init(Bmax, ar, NpMax));
    double* Xr = ar.take<double>(NN);
    double* Xi = ar.take<double>(NN);
    long long* Lr = ar.take<long long>(NN);
    long long* Li = ar.take<long long>(NN);
    double* scratch = ar.take<double>(obs_scratch_bytes(L) / sizeof(double));
    if (!scratch) return fail(TC_ERR_WORKSPACE, "lindblad evolve: workspace too small");
    // the B operand slices seen at each block's padded size (one map per block)
    std::vector<OzMat> Bk(n + 1);
    for (int k = 0; k <= n; k++) TC_TRY(oz_mat_view(Bk[k], Bmax, padded(L.dims[k])));
    const BlockSet bs = block_set(L, true);
    const BlockSet pk = block_set(L, false);
    const PartsSet none{};
    const int stride = TC_OBS_STRIDE(n);
    const bool damp = kappa > 0.0;
    const int group = tune_lookup(n, TC_BF16X3).tc_group;

    auto products = [&](cudaStream_t cs) -> tc_status {
        for (int k = 0; k <= n; k++) {
            const int d = L.dims[k], Np = bs.ld[k];
            double* rr = Rr + bs.off[k];
            double* ri = Ri + bs.off[k];
            const double d3 = (double)d * d * d;
            TC_TRY(oz_mat_load(Bk[k], rr, ri, false, false, d, (size_t)Np, cs));
            {
                ProductTimer pt(8.0 * d3 * Uk[k].dg.pairs, cs);   // X_k = U_k rho_k
                TC_TRY(oz_product(0, Uk[k], Bk[k], OzOut{Xr, Xi, Lr, Li}, group, cs));
            }
            TC_TRY(oz_mat_load(Bk[k], Xr, Xi, false, false, d, (size_t)Np, cs));
            {
                ProductTimer pt(4.0 * d3 * Uk[k].dg.pairs, cs);   // rho_k = U_k X_k^H, Hermitian
                TC_TRY(oz_product(1, Uk[k], Bk[k], OzOut{rr, ri, Lr, Li}, group, cs));
            }
        }
        return TC_OK;
    };
    auto one_step = [&](int k, cudaStream_t cs) -> tc_status {
        if (damp) TC_TRY((launch_damping<double, 0, 0>(L, bs, kappa, 0.5 * dt, t, Rr, Ri, none, cs)));
        TC_TRY(products(cs));
        if (damp) TC_TRY((launch_damping<double, 0, 0>(L, bs, kappa, 0.5 * dt, t, Rr, Ri, none, cs)));
        if (renorm_every > 0 && k % renorm_every == 0)
            TC_TRY((launch_block_renorm<double, 0, 0>(L, bs, Rr, Ri, none, scratch, cs)));
        if (obs) TC_TRY(launch_block_observables<double>(L, bs, m, t, Rr, Ri, obs + (size_t)k * stride, scratch, cs));
        return TC_OK;
    };
    auto first = [&](cudaStream_t cs) -> tc_status {
        TC_TRY(launch_layout(L, t, cs));
        for (int k = 0; k <= n; k++)
            TC_TRY(oz_mat_load(Uk[k], U + 2 * L.off[k], nullptr, true, false, L.dims[k], (size_t)L.dims[k], cs));
        dim3 g(256, (unsigned)(n + 1));
        blocks_split_pad_kernel<<<g, 256, 0, cs>>>(bs, pk, reinterpret_cast<const double2*>(rho), Rr, Ri);
        TC_LAUNCH_CHECK();
        if (obs) TC_TRY(launch_block_observables<double>(L, bs, m, t, Rr, Ri, obs, scratch, cs));
        if (steps >= 1) TC_TRY(one_step(1, cs));
        return TC_OK;
    };
    auto rest = [&](cudaStream_t cs) -> tc_status {
        for (int k = 2; k <= steps; k++) TC_TRY(one_step(k, cs));
        return TC_OK;
    };
    auto tail = [&](cudaStream_t cs) -> tc_status {
        dim3 g(256, (unsigned)(n + 1));
        blocks_join_pad_kernel<<<g, 256, 0, cs>>>(bs, pk, Rr, Ri, reinterpret_cast<double2*>(rho));
        TC_LAUNCH_CHECK();
        return TC_OK;
    };
    return run_captured(s, first, rest, tail, steps > 2 && !timing_enabled());
}

size_t evolve_bytes(int n, int precision) {
    if (precision == TC_FP64_OZAKI) return evolve_oz_bytes_blocks(n);
    return precision == TC_FP64 ? evolve_f64_bytes(n) : evolve_lowp_bytes_blocks(n, precision);
}

}  // namespace

size_t lindblad_bytes(int n, int precision) {
    if (precision < TC_FP64 || precision > TC_FP64_OZAKI) return 0;
    return std::max(propagators_bytes(n), evolve_bytes(n, precision));
}

}  // namespace tc

using namespace tc;

extern "C" TC_API tc_status tc_lindblad_layout(int n, int* dims, size_t* offsets, int* basis) {
    if (n < 1 || n > kMaxAtoms) return fail(TC_ERR_INVALID_ARG, "n = %d outside 1..16", n);
    const Layout& L = layout_of(n);
    if (dims)
        for (int k = 0; k <= n; k++) dims[k] = L.dims[k];
    if (offsets)
        for (int k = 0; k <= n + 1; k++) offsets[k] = L.off[k];
    if (basis)
        for (int s = 0; s < L.N; s++) basis[s] = L.order[s];
    return TC_OK;
}

extern "C" TC_API tc_status tc_lindblad_propagators(const tc_params* params, double dt, void* U, void* work,
                                                    size_t work_bytes, void* stream) {
    Model m;
    TC_TRY(make_model(params, &m));
    if (!U) return fail(TC_ERR_INVALID_ARG, "U is NULL");
    if (reinterpret_cast<uintptr_t>(U) & 15u) return fail(TC_ERR_INVALID_ARG, "U must be 16-byte aligned");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(TC_ERR_INVALID_ARG, "dt must be finite and > 0");
    TC_TRY(check_work(work, work_bytes, propagators_bytes(m.n)));
    TC_TRY(check_device());
    const Layout& L = layout_of(m.n);
    cudaStream_t s = as_stream(stream);
    Arena ar{static_cast<char*>(work), work_bytes, 0};
    Tables t{};
    TC_TRY(take_tables(L, ar, &t));
    TC_TRY(launch_layout(L, t, s));
    double* Ud = static_cast<double*>(U);
    for (int k = 0; k <= m.n; k++) {
        Arena blk_ar = ar;   // every block reuses the same scratch
        ExcitationBlock blk{k, L.dims[k], t.order, t.pos};
        TC_TRY(expm_block_impl(m, blk, L.order.data(), dt, nullptr, Ud + 2 * L.off[k], blk_ar, s, nullptr,
                               nullptr));
    }
    return TC_OK;
}

extern "C" TC_API tc_status tc_lindblad_evolve(const tc_params* params, double kappa, double dt, const void* U,
                                               void* rho, int steps, int precision, int renorm_every, double* obs,
                                               void* work, size_t work_bytes, void* stream) {
    Model m;
    TC_TRY(make_model(params, &m));
    if (!U || !rho) return fail(TC_ERR_INVALID_ARG, "U or rho is NULL");
    if ((reinterpret_cast<uintptr_t>(U) | reinterpret_cast<uintptr_t>(rho)) & 15u)
        return fail(TC_ERR_INVALID_ARG, "U and rho must be 16-byte aligned");
    if (obs && (reinterpret_cast<uintptr_t>(obs) & 7u)) return fail(TC_ERR_INVALID_ARG, "obs must be 8-byte aligned");
    if (!(kappa >= 0.0) || !std::isfinite(kappa)) return fail(TC_ERR_INVALID_ARG, "kappa must be finite and >= 0");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(TC_ERR_INVALID_ARG, "dt must be finite and > 0");
    if (steps < 0 || renorm_every < 0) return fail(TC_ERR_INVALID_ARG, "steps / renorm_every < 0");
    if (precision < TC_FP64 || precision > TC_FP64_OZAKI)
        return fail(TC_ERR_INVALID_ARG, "unknown precision %d", precision);
    TC_TRY(check_work(work, work_bytes, evolve_bytes(m.n, precision)));
    TC_TRY(check_device());
    const Layout& L = layout_of(m.n);
    Arena ar{static_cast<char*>(work), work_bytes, 0};
    const double* Ud = static_cast<const double*>(U);
    double* Rd = static_cast<double*>(rho);
    if (precision == TC_FP64)
        return evolve_f64(L, m, kappa, dt, Ud, Rd, steps, renorm_every, obs, ar, as_stream(stream));
    if (precision == TC_FP64_OZAKI)
        return evolve_oz_blocks(L, m, kappa, dt, Ud, Rd, steps, renorm_every, obs, ar, as_stream(stream));
    return evolve_lowp_blocks(L, m, precision, kappa, dt, Ud, Rd, steps, renorm_every, obs, ar, as_stream(stream));
}
