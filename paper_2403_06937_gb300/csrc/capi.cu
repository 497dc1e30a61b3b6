// capi.cu -- the extern "C" entry points of libtc (include/tc.h) and the host
// orchestration behind them: argument checks, workspace carving, the Taylor
// plan of e^{-iHdt} and the FP64 step loop.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "kernels.cuh"
#include "cgemm_tc.cuh"
#include "paths.cuh"

namespace tc {

namespace {
thread_local std::string g_last_error;
__device__ unsigned g_status_word;
std::mutex g_dev_mutex;
int g_dev_checked[64];      // 0 = unknown, 1 = ok, 2 = unsupported
unsigned* g_status_ptr[64];
}  // namespace

tc_status fail(tc_status s, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

tc_status check_device() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(TC_ERR_UNSUPPORTED_DEVICE, "no CUDA device: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return fail(TC_ERR_UNSUPPORTED_DEVICE, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_dev_mutex);
    if (g_dev_checked[dev] == 0) {
        int major = 0, minor = 0;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        if (major == 10 && minor == 3) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_status_word);
            if (e != cudaSuccess) return fail(TC_ERR_CUDA, "status word: %s", cudaGetErrorString(e));
            g_status_ptr[dev] = static_cast<unsigned*>(p);
            g_dev_checked[dev] = 1;
        } else {
            g_dev_checked[dev] = 2;
        }
    }
    if (g_dev_checked[dev] != 1)
        return fail(TC_ERR_UNSUPPORTED_DEVICE, "device %d is not sm_103 (GB300); no other target is built", dev);
    return TC_OK;
}

unsigned* device_status_word() {
    int dev = 0;
    cudaGetDevice(&dev);
    return (dev >= 0 && dev < 64) ? g_status_ptr[dev] : nullptr;
}

tc_status make_model(const tc_params* p, Model* m) {
    if (!p) return fail(TC_ERR_INVALID_ARG, "params is NULL");
    if (p->n < 1 || p->n > kMaxAtoms) return fail(TC_ERR_INVALID_ARG, "n = %d outside 1..16", p->n);
    if (!p->g) return fail(TC_ERR_INVALID_ARG, "params->g is NULL");
    if (p->coupling != TC_COUPLING_BOSONIC && p->coupling != TC_COUPLING_QUBIT_PHOTON)
        return fail(TC_ERR_INVALID_ARG, "unknown coupling %d", p->coupling);
    if (!std::isfinite(p->omega_a) || !std::isfinite(p->omega_c))
        return fail(TC_ERR_INVALID_ARG, "omega_a / omega_c not finite");
    std::memset(m, 0, sizeof(*m));
    m->n = p->n;
    m->coupling = p->coupling;
    m->omega_a = p->omega_a;
    m->omega_c = p->omega_c;
    for (int i = 0; i < p->n; i++) {
        if (!std::isfinite(p->g[i])) return fail(TC_ERR_INVALID_ARG, "g[%d] not finite", i);
        m->g[i] = p->g[i];
    }
    return TC_OK;
}

// ------------------------------------------------------------------ sizes
namespace {

inline size_t mat_bytes(int n, size_t elem) { return round256((size_t)elem << (2 * n)); }

size_t expm_bytes(int n) {
    size_t N = (size_t)1 << n;
    return 13 * mat_bytes(n, 8) + round256((2 * N + 4) * sizeof(double));
}

size_t evolve_f64_bytes(int n) {
    return 6 * mat_bytes(n, 8) + observables_scratch_bytes(n) + 256 +
           (((size_t)1 << n) <= (size_t)kSplitMaxDim ? gemm_f64_splitk_bytes() : 0);
}

size_t evolve_bytes(int n, int precision) {
    if (precision == TC_FP64_OZAKI) return evolve_oz_bytes(n);
    return precision == TC_FP64 ? evolve_f64_bytes(n) : evolve_lowp_bytes(n, precision);
}

// device staging of tc_evolve_host: rho (c128) and the observable rows
size_t evolve_host_extra(int n, int steps) {
    return mat_bytes(n, 16) + round256((size_t)(steps + 1) * (2 * n + 5) * sizeof(double));
}

// True when tc_evolve_host with a page-locked rho_host runs without a device
// copy of rho: a tensor-core form, at least one step, and the products cut in
// row blocks in and row bands out (the SMs read and write the host rows)
bool host_without_staging(int n, int steps, int precision) {
    if (precision != TC_BF16X3 && precision != TC_TF32 && precision != TC_TF32X3) return false;
    return steps >= 1 && lowp_host_chunks(n, precision) > 1 && lowp_host_bands(n, precision) > 1;
}

size_t evolve_host_pinned_extra(int n, int steps, int precision) {
    const size_t rows = round256((size_t)(steps + 1) * (2 * n + 5) * sizeof(double));
    return host_without_staging(n, steps, precision) ? rows + 256 : evolve_host_extra(n, steps);
}

// ------------------------------------------------------------------ expm plan
// Real GEMMs to evaluate a degree-d polynomial in Y by Horner in Y^q blocks
// (Paterson-Stockmeyer), given Y^1..Y^q.
int horner_gemms(int d, int q) {
    if (d <= q) return 0;
    int r = d / q;
    return (d == r * q) ? r - 1 : r;
}

struct Plan {
    int m, s, q;
    int gemms;
};

// cost of degree m: Y^1..Y^q, Horner for cos (degree m/2 in Y) and for the sin
// factor (degree (m-1)/2), one product B * S'.
Plan cost_of_degree(int m) {
    Plan best{m, 0, 0, 1 << 30};
    int dc = m / 2, ds = (m - 1) / 2;
    if (m <= 1) { best.q = 0; best.gemms = 0; return best; }
    for (int q = 1; q <= 4; q++) {
        int g = q + horner_gemms(dc, q) + horner_gemms(ds, q) + (ds >= 1 ? 1 : 0);
        if (g < best.gemms) { best.q = q; best.gemms = g; }
    }
    return best;
}

// Smallest (gemms + 3 per squaring) meeting the truncation bound
// b^{m+1}/(m+1)! / (1 - b/(m+2)) * 2^s <= 2^-53, b = ||B||_1 / 2^s.
Plan choose_plan(double norm1) {
    const double u = std::ldexp(1.0, -53);
    Plan best{0, 0, 0, 1 << 30};
    for (int s = 0; s <= 40; s++) {
        double b = std::ldexp(norm1, -s);
        for (int m = 1; m <= 30; m++) {
            if (b >= m + 2) continue;
            double term = 1.0;
            for (int k = 1; k <= m + 1; k++) term *= b / k;
            double err = term / (1.0 - b / (m + 2)) * std::ldexp(1.0, s);
            if (err <= u || (b == 0.0)) {
                Plan p = cost_of_degree(m);
                p.s = s;
                int total = p.gemms + 3 * s;
                if (total < best.gemms + 3 * best.s || best.gemms == (1 << 30)) {
                    best = p;
                }
                break;
            }
        }
        if (b < 1e-3) break;
    }
    return best;
}

struct ExpmBufs {
    double* B;
    double* Y[5];   // Y[1..4]
    double* T;
    double* tmp;
    double* C;
    double* S;
    double* C2;
    double* S2;
    double* CS;
    double* small;
};

tc_status gemm_real(int N, const double* A, const double* B, double* C, cudaStream_t s) {
    GemmF64 g{};
    g.M = g.N = g.K = N;
    g.Ar = A; g.lda = N;
    g.Br = B; g.ldb = N;
    g.Cr = C; g.ldc = N;
    g.alpha = 1.0; g.beta = 0.0;
    g.cplx = 0;
    return gemm_f64(g, s);
}

// out = p(Y) = sum_{j<=d} a[j] Y^j with Y^1..Y^q in Y[1..q]; q >= 1.
tc_status eval_poly(int N, const double* a, int d, int q, double* const* Y, double* out, double* tmp,
                    cudaStream_t s) {
    if (d <= q) {
        const double* mats[4];
        double coef[4];
        int t = 0;
        for (int j = 1; j <= d; j++) { mats[t] = Y[j]; coef[t] = a[j]; t++; }
        return launch_lincomb(N, a[0], t, mats, coef, out, s);
    }
    int r = d / q;
    int b = r;
    // T = P_r (possibly a scalar block) ...
    if (d == r * q) {
        // top block is a_d I: T = a_d Y^q + P_{r-1}
        const double* mats[4];
        double coef[4];
        int t = 0;
        mats[t] = Y[q]; coef[t] = a[d]; t++;
        for (int i = 1; i < q; i++) { mats[t] = Y[i]; coef[t] = a[(r - 1) * q + i]; t++; }
        TC_TRY(launch_lincomb(N, a[(r - 1) * q], t, mats, coef, out, s));
        b = r - 1;
    } else {
        const double* mats[4];
        double coef[4];
        int t = 0;
        for (int i = 1; i <= d - r * q; i++) { mats[t] = Y[i]; coef[t] = a[r * q + i]; t++; }
        TC_TRY(launch_lincomb(N, a[r * q], t, mats, coef, out, s));
    }
    // ... then T = Y^q T + P_b for b = b-1 .. 0
    for (int k = b - 1; k >= 0; k--) {
        TC_TRY(gemm_real(N, Y[q], out, tmp, s));
        const double* mats[4];
        double coef[4];
        int t = 0;
        mats[t] = tmp; coef[t] = 1.0; t++;
        for (int i = 1; i < q; i++) { mats[t] = Y[i]; coef[t] = a[k * q + i]; t++; }
        TC_TRY(launch_lincomb(N, a[k * q], t, mats, coef, out, s));
    }
    return TC_OK;
}

}  // namespace

tc_status check_work(void* work, size_t have, size_t need) {
    if (need == 0) return TC_OK;
    if (!work) return fail(TC_ERR_WORKSPACE, "work is NULL (need %zu bytes)", need);
    if (reinterpret_cast<uintptr_t>(work) & 255u) return fail(TC_ERR_WORKSPACE, "work is not 256-byte aligned");
    if (have < need) return fail(TC_ERR_WORKSPACE, "work has %zu bytes, need %zu", have, need);
    return TC_OK;
}

tc_status expm_impl(const double* H, int n, double dt, const tc_expm_opts* opts, double* U, Arena& ar,
                    cudaStream_t s, int* used_degree, int* used_squarings) {
    const int N = 1 << n;
    ExpmBufs b{};
    b.B = ar.take<double>((size_t)N * N);
    for (int i = 1; i <= 4; i++) b.Y[i] = ar.take<double>((size_t)N * N);
    b.T = ar.take<double>((size_t)N * N);
    b.tmp = ar.take<double>((size_t)N * N);
    b.C = ar.take<double>((size_t)N * N);
    b.S = ar.take<double>((size_t)N * N);
    b.C2 = ar.take<double>((size_t)N * N);
    b.S2 = ar.take<double>((size_t)N * N);
    b.CS = ar.take<double>((size_t)N * N);
    b.small = ar.take<double>(2 * (size_t)N + 4);
    if (!b.small) return fail(TC_ERR_WORKSPACE, "expm: workspace too small");

    int shift = opts ? opts->shift : 1;
    double trace = 0.0, norm1 = 0.0, mu = 0.0;
    TC_TRY(matrix_trace_and_norm1(N, H, 0.0, &trace, &norm1, b.small, s));
    if (!std::isfinite(trace) || !std::isfinite(norm1)) return fail(TC_ERR_NUMERIC, "expm: H is not finite");
    if (shift) {
        mu = trace / N;
        TC_TRY(matrix_trace_and_norm1(N, H, mu, &trace, &norm1, b.small, s));
    }
    Plan plan;
    if (opts && opts->taylor_degree > 0) {
        plan = cost_of_degree(opts->taylor_degree);
        plan.s = opts->squarings >= 0 ? opts->squarings : 0;
        if (opts->squarings < 0) {
            // pick squarings for the requested degree
            Plan auto_p = choose_plan(norm1 * dt);
            plan.s = auto_p.s;
        }
    } else {
        plan = choose_plan(norm1 * dt);
        if (opts && opts->squarings >= 0) plan.s = opts->squarings;
    }
    const int m = plan.m, q = plan.q, sq = plan.s;
    if (used_degree) *used_degree = m;
    if (used_squarings) *used_squarings = sq;

    // B = (H - mu I) dt / 2^s
    TC_TRY(launch_shift_scale(N, H, mu, std::ldexp(dt, -sq), b.B, s));

    // cos / sin coefficients: c_j = (-1)^j/(2j)!, s_j = (-1)^j/(2j+1)!
    double cc[32], sc[32];
    {
        double f = 1.0;
        for (int k = 0; k <= 2 * 16 + 1; k++) {
            if (k > 0) f *= k;
            int j = k / 2;
            double sign = (j % 2) ? -1.0 : 1.0;
            if (k % 2 == 0 && j < 32) cc[j] = sign / f;
            if (k % 2 == 1 && j < 32) sc[j] = sign / f;
        }
    }
    const int dc = m / 2, ds = (m - 1) / 2;
    if (m <= 1) {
        // C = I, S = B (degree 1); degree 0 is never planned
        const double* one[1] = {b.B};
        double cz[1] = {0.0};
        TC_TRY(launch_lincomb(N, 1.0, 0, one, cz, b.C, s));
        double c1[1] = {1.0};
        TC_TRY(launch_lincomb(N, 0.0, 1, one, c1, b.S, s));
    } else {
        TC_TRY(gemm_real(N, b.B, b.B, b.Y[1], s));
        for (int j = 2; j <= q; j++) TC_TRY(gemm_real(N, b.Y[j - 1], b.Y[1], b.Y[j], s));
        TC_TRY(eval_poly(N, cc, dc, q, b.Y, b.C, b.tmp, s));
        if (ds >= 1) {
            TC_TRY(eval_poly(N, sc, ds, q, b.Y, b.T, b.tmp, s));
            TC_TRY(gemm_real(N, b.B, b.T, b.S, s));
        } else {
            const double* one[1] = {b.B};
            double c1[1] = {1.0};
            TC_TRY(launch_lincomb(N, 0.0, 1, one, c1, b.S, s));
        }
    }
    // squarings: (C - iS)^2 = (C^2 - S^2) - i 2 C S   (C and S commute)
    double* C = b.C;
    double* S = b.S;
    for (int k = 0; k < sq; k++) {
        TC_TRY(gemm_real(N, C, C, b.C2, s));
        TC_TRY(gemm_real(N, S, S, b.S2, s));
        TC_TRY(gemm_real(N, C, S, b.CS, s));
        const double* m2[2] = {b.C2, b.S2};
        double c2[2] = {1.0, -1.0};
        TC_TRY(launch_lincomb(N, 0.0, 2, m2, c2, C, s));
        const double* m1[1] = {b.CS};
        double c1[1] = {2.0};
        TC_TRY(launch_lincomb(N, 0.0, 1, m1, c1, S, s));
    }
    // U = e^{-i mu dt} (C - i S), symmetrised
    double phi = mu * dt;
    TC_TRY(launch_expm_finish(N, C, S, std::cos(phi), -std::sin(phi), U, s));
    return TC_OK;
}

}  // namespace tc

using namespace tc;

// ======================================================================== ABI
extern "C" {

TC_API const char* tc_version(void) { return "libtc 0.1 (sm_103a)"; }

TC_API const char* tc_last_error(void) { return g_last_error.c_str(); }

TC_API tc_status tc_device_check(void) { return check_device(); }

TC_API size_t tc_workspace_size(int n, int precision, int ops, int steps, int ckpt_every) {
    if (n < 1 || n > kMaxAtoms) return 0;
    size_t need = 0;
    auto upd = [&](size_t b) { if (b > need) need = b; };
    if (ops & TC_OP_EXPM) upd(expm_bytes(n));
    if (ops & TC_OP_EVOLVE) upd(evolve_bytes(n, precision));
    if (ops & TC_OP_OBSERVABLES) upd(observables_scratch_bytes(n));
    if (ops & TC_OP_EXPM_MODEL) upd(expm_model_bytes(n));
    if (ops & TC_OP_LINDBLAD) upd(lindblad_bytes(n, precision));
    if (ops & TC_OP_EVOLVE_HOST) upd(evolve_bytes(n, precision) + evolve_host_extra(n, steps));
    if (ops & TC_OP_EVOLVE_HOST_PINNED) upd(evolve_bytes(n, precision) + evolve_host_pinned_extra(n, steps, precision));
    if (ops & TC_OP_BACKWARD) upd(backward_bytes(n, steps, ckpt_every, precision));
    return need;
}

TC_API tc_status tc_build_hamiltonian(const tc_params* params, double* H, void* stream) {
    Model m;
    TC_TRY(make_model(params, &m));
    if (!H) return fail(TC_ERR_INVALID_ARG, "H is NULL");
    if (reinterpret_cast<uintptr_t>(H) & 15u) return fail(TC_ERR_INVALID_ARG, "H must be 16-byte aligned");
    TC_TRY(check_device());
    return launch_build_h(m, H, as_stream(stream));
}

TC_API tc_status tc_expm(const double* H, int n, double dt, const tc_expm_opts* opts, void* U, void* work,
                         size_t work_bytes, void* stream) {
    if (n < 1 || n > kMaxAtoms) return fail(TC_ERR_INVALID_ARG, "n = %d outside 1..16", n);
    if (!H || !U) return fail(TC_ERR_INVALID_ARG, "H or U is NULL");
    if ((reinterpret_cast<uintptr_t>(H) | reinterpret_cast<uintptr_t>(U)) & 15u)
        return fail(TC_ERR_INVALID_ARG, "H and U must be 16-byte aligned");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(TC_ERR_INVALID_ARG, "dt must be finite and > 0");
    if (opts && (opts->taylor_degree < 0 || opts->taylor_degree > 30 || opts->squarings < -1 ||
                 opts->squarings > 40))
        return fail(TC_ERR_INVALID_ARG, "expm opts out of range");
    TC_TRY(check_work(work, work_bytes, expm_bytes(n)));
    TC_TRY(check_device());
    Arena ar{static_cast<char*>(work), work_bytes, 0};
    return expm_impl(H, n, dt, opts, static_cast<double*>(U), ar, as_stream(stream), nullptr, nullptr);
}

TC_API tc_status tc_observables(const void* rho, int n, const tc_params* params, double* out, void* work,
                                size_t work_bytes, void* stream) {
    if (n < 1 || n > kMaxAtoms) return fail(TC_ERR_INVALID_ARG, "n = %d outside 1..16", n);
    if (!rho || !out) return fail(TC_ERR_INVALID_ARG, "rho or out is NULL");
    if ((reinterpret_cast<uintptr_t>(rho) | reinterpret_cast<uintptr_t>(out)) & 7u)
        return fail(TC_ERR_INVALID_ARG, "rho and out must be 8-byte aligned");
    Model m;
    if (params) {
        TC_TRY(make_model(params, &m));
        if (m.n != n) return fail(TC_ERR_INVALID_ARG, "params->n != n");
    }
    TC_TRY(check_work(work, work_bytes, observables_scratch_bytes(n)));
    TC_TRY(check_device());
    return launch_observables(kRhoInterleaved, rho, nullptr, params ? &m : nullptr, n, out,
                              static_cast<double*>(work), as_stream(stream));
}

TC_API tc_status tc_evolve(const void* U, void* rho, int n, int steps, int precision, int renorm_every,
                           const tc_params* params, double* obs, void* work, size_t work_bytes, void* stream) {
    if (n < 1 || n > kMaxAtoms) return fail(TC_ERR_INVALID_ARG, "n = %d outside 1..16", n);
    if (!U || !rho) return fail(TC_ERR_INVALID_ARG, "U or rho is NULL");
    if ((reinterpret_cast<uintptr_t>(U) | reinterpret_cast<uintptr_t>(rho)) & 15u)
        return fail(TC_ERR_INVALID_ARG, "U and rho must be 16-byte aligned");
    if (obs && (reinterpret_cast<uintptr_t>(obs) & 7u)) return fail(TC_ERR_INVALID_ARG, "obs must be 8-byte aligned");
    if (steps < 0) return fail(TC_ERR_INVALID_ARG, "steps < 0");
    if (renorm_every < 0) return fail(TC_ERR_INVALID_ARG, "renorm_every < 0");
    if (precision < TC_FP64 || precision > TC_FP64_OZAKI)
        return fail(TC_ERR_INVALID_ARG, "unknown precision %d", precision);
    Model m;
    const Model* mp = nullptr;
    if (params) {
        TC_TRY(make_model(params, &m));
        if (m.n != n) return fail(TC_ERR_INVALID_ARG, "params->n != n");
        mp = &m;
    }
    TC_TRY(check_work(work, work_bytes, evolve_bytes(n, precision)));
    TC_TRY(check_device());
    cudaStream_t s = as_stream(stream);
    Arena ar{static_cast<char*>(work), work_bytes, 0};
    if (precision == TC_FP64_OZAKI)
        return evolve_oz(static_cast<const double*>(U), static_cast<double*>(rho), n, steps, renorm_every, mp, obs,
                         ar, s);
    if (precision != TC_FP64)
        return evolve_lowp(static_cast<const double*>(U), static_cast<double*>(rho), n, steps, precision,
                           renorm_every, mp, obs, ar, s);
    return evolve_f64(static_cast<const double*>(U), static_cast<double*>(rho), n, steps, renorm_every, mp, obs,
                      ar, s);
}

TC_API tc_status tc_evolve_host(const void* U, void* rho_host, int n, int steps, int precision, int renorm_every,
                                const tc_params* params, double* obs_host, void* work, size_t work_bytes,
                                void* stream) {
    if (n < 1 || n > kMaxAtoms) return fail(TC_ERR_INVALID_ARG, "n = %d outside 1..16", n);
    if (!U || !rho_host) return fail(TC_ERR_INVALID_ARG, "U or rho_host is NULL");
    if (reinterpret_cast<uintptr_t>(U) & 15u) return fail(TC_ERR_INVALID_ARG, "U must be 16-byte aligned");
    if (steps < 0 || renorm_every < 0) return fail(TC_ERR_INVALID_ARG, "steps / renorm_every < 0");
    if (precision < TC_FP64 || precision > TC_FP64_OZAKI)
        return fail(TC_ERR_INVALID_ARG, "unknown precision %d", precision);
    Model m;
    const Model* mp = nullptr;
    if (params) {
        TC_TRY(make_model(params, &m));
        if (m.n != n) return fail(TC_ERR_INVALID_ARG, "params->n != n");
        mp = &m;
    }
    TC_TRY(check_device());
    // a page-locked rho_host in the pipelined tensor-core forms needs no device copy of rho
    const void* mapped_rho = nullptr;
    TC_TRY(host_mapping(rho_host, &mapped_rho));
    const bool no_staging = mapped_rho && host_without_staging(n, steps, precision);
    TC_TRY(check_work(work, work_bytes,
                      evolve_bytes(n, precision) +
                          (no_staging ? evolve_host_pinned_extra(n, steps, precision) : evolve_host_extra(n, steps))));
    cudaStream_t s = as_stream(stream);
    const size_t N = (size_t)1 << n;
    Arena ar{static_cast<char*>(work), work_bytes, 0};
    double* rho_dev = no_staging ? nullptr : ar.take<double>(2 * N * N);
    double* obs_dev = ar.take<double>((size_t)(steps + 1) * (2 * n + 5));
    double* od = obs_host ? obs_dev : nullptr;
    const double* Ud = static_cast<const double*>(U);
    if (precision == TC_FP64 || precision == TC_FP64_OZAKI) {
        // page-locked rho_host: the SMs copy it (copy-engine reads of host memory slow down under host load)
        const void* mapped = nullptr;
        TC_TRY(host_mapping(rho_host, &mapped));
        if (mapped)
            TC_TRY(copy_by_sms(rho_dev, mapped, 16 * N * N, s));
        else
            TC_CUDA(cudaMemcpyAsync(rho_dev, rho_host, 16 * N * N, cudaMemcpyHostToDevice, s));
        TC_TRY(precision == TC_FP64 ? evolve_f64(Ud, rho_dev, n, steps, renorm_every, mp, od, ar, s)
                                    : evolve_oz(Ud, rho_dev, n, steps, renorm_every, mp, od, ar, s));
        if (mapped)
            TC_TRY(copy_by_sms(const_cast<void*>(mapped), rho_dev, 16 * N * N, s));
        else
            TC_CUDA(cudaMemcpyAsync(rho_host, rho_dev, 16 * N * N, cudaMemcpyDeviceToHost, s));
    } else {
        // copies overlapped with the first and last products (row blocks on a copy stream)
        TC_TRY(evolve_lowp_host(Ud, static_cast<double*>(rho_host), rho_dev, n, steps, precision, renorm_every, mp,
                                od, ar, s));
    }
    if (obs_host)
        TC_CUDA(cudaMemcpyAsync(obs_host, obs_dev, (size_t)(steps + 1) * (2 * n + 5) * sizeof(double),
                                cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    return TC_OK;
}

TC_API tc_status tc_fault_inject(int kind, int count, double wait_limit_s) {
    if (kind != TC_FAULT_TC_STAGE_WITHHELD) return fail(TC_ERR_INVALID_ARG, "unknown fault kind %d", kind);
    if (count < 0 || !(wait_limit_s > 0.0) || wait_limit_s > 10.0)
        return fail(TC_ERR_INVALID_ARG, "count >= 0 and 0 < wait_limit_s <= 10 required");
    cgemm_inject_timeout(count, (unsigned long long)(wait_limit_s * 1e9));
    return TC_OK;
}

TC_API tc_status tc_sync_status(void* stream) {
    TC_TRY(check_device());
    cudaStream_t s = as_stream(stream);
    TC_CUDA(cudaStreamSynchronize(s));
    TC_CUDA(cudaGetLastError());
    unsigned* w = device_status_word();
    unsigned v = 0;
    TC_CUDA(cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost));
    unsigned z = 0;
    TC_CUDA(cudaMemcpy(w, &z, sizeof(z), cudaMemcpyHostToDevice));
    if (v & kStatusTimeout) return fail(TC_ERR_TIMEOUT, "a bounded device wait timed out");
    if (v & kStatusNumeric) return fail(TC_ERR_NUMERIC, "non-finite or non-positive trace");
    return TC_OK;
}

}  // extern "C"
