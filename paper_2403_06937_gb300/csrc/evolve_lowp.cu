// evolve_lowp.cu -- the low-precision forms of the step loop
// rho <- U rho U^dag (Sec. III.A, Eqs. 6, 12) on the tcgen05 tensor cores.
//
// U arrives in FP64 (from tc_expm).  It is used in increment form: with the
// unit phase c = Tr U / |Tr U| (which cancels in U rho U^dag), V = U / c - I
// is formed in FP64 and split once per call into operand parts (BF16x3:
// three BF16 parts; TF32x3: big/small TF32; TF32: one TF32 part).  rho and
// X = U rho / c live in FP32 planes plus the operand parts of those values.
// Each step is two launches of the tensor-core GEMM Y = P^H + V P^H:
//     X    = rho^H + V rho^H   (all tiles)
//     rho' = X^H + V X^H       (block-lower tiles + mirror)
// (rho' = U rho U^dag: the two phases cancel.)
// then, every `renorm_every` steps, rho <- rho / Tr rho with the trace in
// FP64, and the observable row from the FP32 planes.
// Dimensions below 128 (n < 7) are zero-padded to one 128 x 128 tile: the
// padded rows and columns of U and rho are zero and stay zero.
// evolve_lowp_host is the same loop with rho in host memory: its copies run
// by row blocks on a second stream, overlapped with the first product of the
// first step and the second product of the last.
#include <cuda_bf16.h>

#include <cstdio>

#include "cgemm_tc.cuh"
#include "graph.cuh"
#include "lowp.cuh"
#include "paths.cuh"
#include "timing.cuh"

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

// v as an FP32 pair hi + lo read off its bit fields, with no FP64
// instruction (GB300 issues FP64 at a small fraction of its FP32 rate):
// hi = v truncated to FP32's 24 significand bits, lo = the 29 bits below
// them rounded to 24, so |v - hi - lo| <= 2^-47 |v|.  |v| < 2^-126 (zero,
// the smallest normals and FP64 subnormals) gives a signed zero hi and lo = 0,
// |v| >= 2^128 an infinite hi, NaN a NaN.
__device__ __forceinline__ void f64_pair(double v, float& hi, float& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FFu) - 1023;
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    lo = 0.0f;
    if (e < -126) {
        hi = __uint_as_float(sign);
        return;
    }
    if (e > 127) {
        hi = __uint_as_float(sign | 0x7F800000u | (e == 1024 && m ? 0x400000u : 0u));
        return;
    }
    hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)(m >> 29));
    // bit 0 of m is worth 2^(e - 52): scale by two powers of two, each a normal FP32
    const int q = (e - 52) >> 1, r = (e - 52) - q;
    const float low = __uint2float_rn((unsigned)(m & 0x1FFFFFFFu)) * __uint_as_float((unsigned)(q + 127) << 23) *
                      __uint_as_float((unsigned)(r + 127) << 23);
    lo = sign ? -low : low;
}

// a + b = s + err exactly (Knuth's two-sum; no product, so nothing is contracted)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
    s = a + b;
    const float bb = s - a;
    err = (a - (s - bb)) + (b - bb);
}

// (ah + al)(bh + bl) = p + e to about 2^-46 relative (al bl dropped); p = RN(ah bh), its
// rounding error recovered exactly by the FMA
__device__ __forceinline__ void pair_mul(float ah, float al, float bh, float bl, float& p, float& e) {
    p = ah * bh;
    e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
}

// parts of a value held as the FP32 pair hi + lo: BF16 parts b0 = RN(hi),
// b1 = RN((hi - b0) + lo), b2 = RN(r - b1) (hi - b0 and r - b1 exact), TF32
// parts likewise; they represent hi + lo to about 2^-26 of its size.
template <int KIND, int S>
__device__ __forceinline__ void split_pair(float hi, float lo, void* base, size_t plane, size_t idx, int part) {
    if constexpr (KIND == 0) {
        __nv_bfloat16* p = static_cast<__nv_bfloat16*>(base);
        float r = hi;
#pragma unroll
        for (int s = 0; s < S; s++) {
            __nv_bfloat16 b = __float2bfloat16_rn(r);
            p[(size_t)(part * S + s) * plane + idx] = b;
            r -= __bfloat162float(b);
            if (s == 0) r += lo;
        }
    } else {
        float* p = static_cast<float*>(base);
        float r = hi;
#pragma unroll
        for (int s = 0; s < S; s++) {
            float t = tf32_rna(r);
            p[(size_t)(part * S + s) * plane + idx] = t;
            r -= t;
            if (s == 0) r += lo;
        }
    }
}

// c = Tr U / |Tr U| into out[0..1] (1 if the trace vanishes); one block, fixed order
__global__ void unit_phase_kernel(const double2* U, int N, double* out) {
    __shared__ double sr[1024], si[1024];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double2 u = U[(size_t)i * N + i];
        a += u.x;
        b += u.y;
    }
    sr[threadIdx.x] = a;
    si[threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sr[threadIdx.x] += sr[threadIdx.x + w];
            si[threadIdx.x] += si[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double m = hypot(sr[0], si[0]);
        out[0] = m > 1e-300 ? sr[0] / m : 1.0;
        out[1] = m > 1e-300 ? si[0] / m : 0.0;
    }
}

// V = U conj(c) - I (zero in the padding), formed in FP32-pair arithmetic
// (U's entries and c read off as FP32 pairs, products by FMA, sums by
// two-sum: about 2^-44 relative, far below the parts' 2^-26) and split into
// operand parts; blocks take rows, threads columns (no index division), four
// loads in flight per thread.
template <int KIND, int S>
__global__ void prep_u_kernel(const double2* U, int N, int Np, const double* phase, void* parts) {
    const size_t plane = (size_t)Np * Np;
    float crh, crl, cih, cil;   // conj(c) = cr + i ci
    f64_pair(phase[0], crh, crl);
    f64_pair(-phase[1], cih, cil);
    for (int i = blockIdx.x; i < Np; i += gridDim.x) {
        for (int j0 = threadIdx.x; j0 < Np; j0 += 4 * blockDim.x) {
            double2 u[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int j = j0 + k * blockDim.x;
                u[k] = (i < N && j < N) ? U[(size_t)i * N + j] : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int j = j0 + k * blockDim.x;
                if (j >= Np) break;
                float xh, xl, yh, yl;
                f64_pair(u[k].x, xh, xl);
                f64_pair(u[k].y, yh, yl);
                float p1, e1, p2, e2, p3, e3, p4, e4;
                pair_mul(xh, xl, crh, crl, p1, e1);   // Re u cr
                pair_mul(yh, yl, cih, cil, p2, e2);   // Im u ci
                pair_mul(xh, xl, cih, cil, p3, e3);   // Re u ci
                pair_mul(yh, yl, crh, crl, p4, e4);   // Im u cr
                float vr, tr, vi, ti;
                two_sum(p1, -p2, vr, tr);
                tr += e1 - e2;
                two_sum(p3, p4, vi, ti);
                ti += e3 + e4;
                if (i == j && i < N) {
                    float d;
                    two_sum(vr, -1.0f, vr, d);
                    tr += d;
                }
                const size_t e = (size_t)i * Np + j;
                split_pair<KIND, S>(vr, tr, parts, plane, e, 0);
                split_pair<KIND, S>(vi, ti, parts, plane, e, 1);
            }
        }
    }
}

// rows [r0, r1) of the padded plane; blocks take rows, threads columns, four
// loads in flight per thread (rho may be page-locked host memory read through
// its device mapping)
template <int KIND, int S>
__global__ void prep_rho_kernel(const double2* rho, int N, int Np, int r0, int r1, float* Rr, float* Ri,
                                void* parts) {
    const size_t plane = (size_t)Np * Np;
    for (int i = r0 + blockIdx.x; i < r1; i += gridDim.x) {
        for (int j0 = threadIdx.x; j0 < Np; j0 += 4 * blockDim.x) {
            double2 v[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int j = j0 + u * blockDim.x;
                v[u] = (i < N && j < N) ? rho[(size_t)i * N + j] : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int j = j0 + u * blockDim.x;
                if (j >= Np) break;
                const size_t e = (size_t)i * Np + j;
                const float fr = (float)v[u].x, fi = (float)v[u].y;
                Rr[e] = fr;
                Ri[e] = fi;
                split_f32<KIND, S>(fr, parts, plane, e, 0);
                split_f32<KIND, S>(fi, parts, plane, e, 1);
            }
        }
    }
}

// rho <- rho / trace (trace read on the device; skipped and flagged if not positive finite),
// then the operand parts are rebuilt from the rescaled FP32 values.
template <int KIND, int S>
__global__ void rescale_resplit_kernel(float* Rr, float* Ri, int Np, void* parts, const double* trace,
                                       unsigned* status) {
    const double tr = trace[0];
    if (!(tr > 0.0) || !isfinite(tr)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kStatusNumeric);
        return;
    }
    const double inv = 1.0 / tr;
    const size_t plane = (size_t)Np * Np;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < plane; e += (size_t)gridDim.x * blockDim.x) {
        const float fr = (float)((double)Rr[e] * inv), fi = (float)((double)Ri[e] * inv);
        Rr[e] = fr;
        Ri[e] = fi;
        split_f32<KIND, S>(fr, parts, plane, e, 0);
        split_f32<KIND, S>(fi, parts, plane, e, 1);
    }
}

__global__ void trace_f32_kernel(const float* Rr, int N, int Np, double* out) {
    __shared__ double s[1024];
    double a = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) a += (double)Rr[(size_t)i * Np + i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = s[0];
}

// rows [r0, r1) of the N x N result; blocks take rows, threads columns (rho
// may be page-locked host memory written through its device mapping)
__global__ void finish_kernel(const float* Rr, const float* Ri, int N, int Np, int r0, int r1, int c0, int c1,
                              double2* rho) {
    for (int i = r0 + blockIdx.x; i < r1; i += gridDim.x)
        for (int j = c0 + threadIdx.x; j < c1; j += blockDim.x)
            rho[(size_t)i * N + j] = make_double2((double)Rr[(size_t)i * Np + j], (double)Ri[(size_t)i * Np + j]);
}

}  // namespace

size_t plane_bytes(int Np, size_t E) { return round256((size_t)Np * Np * E); }

namespace {

template <int KIND, int S>
tc_status run_prep_u(const double* U, LowpBufs& b, cudaStream_t s) {
    const size_t plane = (size_t)b.Np * b.Np;
    double* phase = b.scratch;   // consumed by prep_u before any other use of scratch
    unit_phase_kernel<<<1, 1024, 0, s>>>(reinterpret_cast<const double2*>(U), b.N, phase);
    TC_LAUNCH_CHECK();
    const unsigned rows_grid = grid_for(plane) < (unsigned)b.Np ? grid_for(plane) : (unsigned)b.Np;
    prep_u_kernel<KIND, S><<<rows_grid, 256, 0, s>>>(reinterpret_cast<const double2*>(U), b.N, b.Np, phase,
                                                            b.Uparts);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

// CTAs over rows: at most grid_for's cap, and at most `cap` when given (the
// host-memory transfers run beside the products, on a few CTAs per SM)
unsigned rows_grid(int rows, size_t work, unsigned cap) {
    unsigned g = grid_for(work);
    if (g > (unsigned)rows) g = (unsigned)rows;
    if (cap && g > cap) g = cap;
    return g ? g : 1u;
}

template <int KIND, int S>
tc_status run_prep_rho(const double* rho, LowpBufs& b, int r0, int r1, cudaStream_t s, unsigned cap) {
    prep_rho_kernel<KIND, S><<<rows_grid(r1 - r0, (size_t)(r1 - r0) * b.Np, cap), 256, 0, s>>>(
        reinterpret_cast<const double2*>(rho), b.N, b.Np, r0, r1, b.Rr, b.Ri, b.Rparts);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

template <int KIND, int S>
tc_status run_prep(const double* U, const double* rho, LowpBufs& b, cudaStream_t s) {
    TC_TRY((run_prep_u<KIND, S>(U, b, s)));
    return run_prep_rho<KIND, S>(rho, b, 0, b.Np, s, 0u);
}

template <int KIND, int S>
tc_status run_renorm(LowpBufs& b, cudaStream_t s) {
    trace_f32_kernel<<<1, 1024, 0, s>>>(b.Rr, b.N, b.Np, b.scratch);
    TC_LAUNCH_CHECK();
    rescale_resplit_kernel<KIND, S><<<grid_for((size_t)b.Np * b.Np), 256, 0, s>>>(b.Rr, b.Ri, b.Np, b.Rparts, b.scratch,
                                                                                  device_status_word());
    TC_LAUNCH_CHECK();
    return TC_OK;
}

}  // namespace

tc_status lowp_prep(int precision, const double* U, const double* rho, LowpBufs& b, cudaStream_t s) {
    switch (precision) {
        case TC_BF16X3: return run_prep<0, 3>(U, rho, b, s);
        case TC_TF32: return run_prep<1, 1>(U, rho, b, s);
        case TC_TF32X3: return run_prep<1, 2>(U, rho, b, s);
    }
    return fail(TC_ERR_INVALID_ARG, "precision");
}

tc_status lowp_renorm(int precision, LowpBufs& b, cudaStream_t s) {
    switch (precision) {
        case TC_BF16X3: return run_renorm<0, 3>(b, s);
        case TC_TF32: return run_renorm<1, 1>(b, s);
        case TC_TF32X3: return run_renorm<1, 2>(b, s);
    }
    return fail(TC_ERR_INVALID_ARG, "precision");
}

tc_status lowp_prep_u(int precision, const double* U, LowpBufs& b, cudaStream_t s) {
    switch (precision) {
        case TC_BF16X3: return run_prep_u<0, 3>(U, b, s);
        case TC_TF32: return run_prep_u<1, 1>(U, b, s);
        case TC_TF32X3: return run_prep_u<1, 2>(U, b, s);
    }
    return fail(TC_ERR_INVALID_ARG, "precision");
}

tc_status lowp_prep_rho(int precision, const double* rho, LowpBufs& b, int r0, int r1, cudaStream_t s,
                        unsigned cap) {
    if (r0 < 0 || r0 >= r1 || r1 > b.Np) return fail(TC_ERR_INVALID_ARG, "prep: row range");
    switch (precision) {
        case TC_BF16X3: return run_prep_rho<0, 3>(rho, b, r0, r1, s, cap);
        case TC_TF32: return run_prep_rho<1, 1>(rho, b, r0, r1, s, cap);
        case TC_TF32X3: return run_prep_rho<1, 2>(rho, b, r0, r1, s, cap);
    }
    return fail(TC_ERR_INVALID_ARG, "precision");
}

tc_status lowp_finish(const LowpBufs& b, double* rho, cudaStream_t s, int r0, int r1, unsigned cap, int c0, int c1) {
    if (r1 < 0) r1 = b.N;
    if (c1 < 0) c1 = b.N;
    if (r0 < 0 || r0 >= r1 || r1 > b.N) return fail(TC_ERR_INVALID_ARG, "finish: row range");
    if (c0 < 0 || c0 >= c1 || c1 > b.N) return fail(TC_ERR_INVALID_ARG, "finish: column range");
    finish_kernel<<<rows_grid(r1 - r0, (size_t)(r1 - r0) * (c1 - c0), cap), 256, 0, s>>>(
        b.Rr, b.Ri, b.N, b.Np, r0, r1, c0, c1, reinterpret_cast<double2*>(rho));
    TC_LAUNCH_CHECK();
    return TC_OK;
}

size_t lowp_system_bytes(int n, int precision) {
    const int N = 1 << n;
    const int Np = N < 128 ? 128 : N;
    const int S = cgemm_parts(precision);
    const size_t E = cgemm_elem_bytes(precision);
    return 3 * (size_t)(2 * S) * plane_bytes(Np, E) + 4 * plane_bytes(Np, 4) + observables_scratch_bytes(n) + 512;
}

tc_status lowp_carve(int n, int precision, Arena& ar, LowpBufs& b) {
    b.N = 1 << n;
    b.Np = b.N < 128 ? 128 : b.N;
    b.S = cgemm_parts(precision);
    b.E = cgemm_elem_bytes(precision);
    auto take_planes = [&](int planes, size_t E) -> void* {
        return ar.take<uint8_t>((size_t)planes * plane_bytes(b.Np, E));
    };
    b.Uparts = take_planes(2 * b.S, b.E);
    b.Rparts = take_planes(2 * b.S, b.E);
    b.Xparts = take_planes(2 * b.S, b.E);
    b.Rr = static_cast<float*>(take_planes(1, 4));
    b.Ri = static_cast<float*>(take_planes(1, 4));
    b.Xr = static_cast<float*>(take_planes(1, 4));
    b.Xi = static_cast<float*>(take_planes(1, 4));
    b.scratch = ar.take<double>(observables_scratch_bytes(n) / sizeof(double));
    if (!b.scratch) return fail(TC_ERR_WORKSPACE, "low-precision workspace too small");
    return TC_OK;
}

size_t evolve_lowp_bytes(int n, int precision) {
    if (precision != TC_BF16X3 && precision != TC_TF32 && precision != TC_TF32X3) return 0;
    return lowp_system_bytes(n, precision);
}

namespace {

// Tensor maps and epilogues of the two products of a step on the buffers b.
struct StepPlan {
    CUtensorMap tmU, tmR, tmX;
    CUtensorMap wU, wR, wX;   // cgemm_pair_rows()-byte rows, for the CTA-pair kernel
    CgemmEpi e1;   // X = rho^H + V rho^H
    CgemmEpi e2;   // rho' = X^H + V X^H
    TuneChoice tune;
};

tc_status plan_step(int n, int precision, const LowpBufs& b, StepPlan& p) {
    TC_TRY(make_part_map(&p.tmU, b.Uparts, b.Np, 2 * b.S, precision));
    TC_TRY(make_part_map(&p.tmR, b.Rparts, b.Np, 2 * b.S, precision));
    TC_TRY(make_part_map(&p.tmX, b.Xparts, b.Np, 2 * b.S, precision));
    const int rows = cgemm_pair_rows(precision);
    TC_TRY(make_part_map_rows(&p.wU, b.Uparts, b.Np, 2 * b.S, precision, rows));
    TC_TRY(make_part_map_rows(&p.wR, b.Rparts, b.Np, 2 * b.S, precision, rows));
    TC_TRY(make_part_map_rows(&p.wX, b.Xparts, b.Np, 2 * b.S, precision, rows));
    p.tune = tune_lookup(n, precision);
    p.e1 = CgemmEpi{};
    p.e1.Np = b.Np;
    p.e1.tiles = b.Np / 128;
    p.e1.group = p.tune.tc_group;
    p.e1.shape = p.tune.tc_shape;
    p.e1.pr = b.Rr;
    p.e1.pi = b.Ri;
    p.e1.parts = b.Xparts;
    p.e1.yr = b.Xr;
    p.e1.yi = b.Xi;
    p.e1.status = device_status_word();
    p.e2 = p.e1;
    p.e2.pr = b.Xr;
    p.e2.pi = b.Xi;
    p.e2.parts = b.Rparts;
    p.e2.yr = b.Rr;
    p.e2.yi = b.Ri;
    return TC_OK;
}

}  // namespace

tc_status evolve_lowp(const double* U, double* rho, int n, int steps, int precision, int renorm_every,
                      const Model* m, double* obs, Arena& ar, cudaStream_t s) {
    LowpBufs b{};
    TC_TRY(lowp_carve(n, precision, ar, b));
    const size_t pl = (size_t)b.Np * b.Np;
    if (plane_bytes(b.Np, b.E) != pl * b.E) return fail(TC_ERR_INVALID_ARG, "evolve: plane size");
    StepPlan sp{};
    TC_TRY(plan_step(n, precision, b, sp));
    const CUtensorMap &tmU = sp.tmU, &tmR = sp.tmR, &tmX = sp.tmX;
    const CgemmEpi &e1 = sp.e1, &e2 = sp.e2;
    const TuneChoice& tune = sp.tune;

    const int stride = TC_OBS_STRIDE(n);
    const double N3 = (double)b.N * b.N * b.N;
    const double prod = (double)cgemm_products(precision);

    auto one_step = [&](int k, cudaStream_t cs) -> tc_status {
        {
            ProductTimer t(8.0 * N3 * prod, cs);
            TC_TRY(cgemm_tc(precision, 0, tmU, tmR, e1, cs, tune.tc_stages, &sp.wU, &sp.wR));
        }
        {
            ProductTimer t(4.0 * N3 * prod, cs);
            TC_TRY(cgemm_tc(precision, 1, tmU, tmX, e2, cs, tune.tc_stages, &sp.wU, &sp.wX));
        }
        if (renorm_every > 0 && k % renorm_every == 0) TC_TRY(lowp_renorm(precision, b, cs));
        if (obs)
            TC_TRY(launch_observables(kRhoPlanarF32, b.Rr, b.Ri, m, n, obs + (size_t)k * stride, b.scratch, cs,
                                      (size_t)b.Np));
        return TC_OK;
    };
    auto first = [&](cudaStream_t cs) -> tc_status {
        TC_TRY(lowp_prep(precision, U, rho, b, cs));
        if (obs) TC_TRY(launch_observables(kRhoPlanarF32, b.Rr, b.Ri, m, n, obs, b.scratch, cs, (size_t)b.Np));
        if (steps >= 1) TC_TRY(one_step(1, cs));
        return TC_OK;
    };
    auto rest = [&](cudaStream_t cs) -> tc_status {
        for (int k = 2; k <= steps; k++) TC_TRY(one_step(k, cs));
        return TC_OK;
    };
    auto tail = [&](cudaStream_t cs) -> tc_status { return lowp_finish(b, rho, cs); };
    return run_captured(s, first, rest, tail, steps > 2 && !timing_enabled());
}

int lowp_host_chunks(int n, int precision) {
    const int N = 1 << n;
    if (N < 2048) return 1;
    const int T = N / 128;
    int G = tune_lookup(n, precision).tc_group;
    G = G < 1 ? 1 : G;
    return T % (4 * G) == 0 ? 4 : T % (2 * G) == 0 ? 2 : 1;
}

// Row bands of the last Hermitian product of a host-buffer call: more and
// narrower than the row blocks in, so the bottom band is done (and its rows
// start out) early and the top band's diagonal block, the only copy left
// after the last product, is small.  A band holds whole raster groups and
// whole row pairs.
int lowp_host_bands(int n, int precision) {
    const int N = 1 << n;
    if (N < 2048) return 1;
    const int T = N / 128;
    int G = tune_lookup(n, precision).tc_group;
    G = G < 1 ? 1 : G;
    for (int C : {8, 4, 2})
        if (T % (C * G) == 0 && (T / C) % 2 == 0) return C;
    return 1;
}

namespace {

// Streams and events of one pipelined call, released when it goes out of scope
// (the device finishes the queued work first).
struct CopyLane {
    cudaStream_t cs = nullptr;
    cudaEvent_t ev[24] = {};
    int used = 0;
    ~CopyLane() {
        for (int i = 0; i < used; i++) cudaEventDestroy(ev[i]);
        if (cs) cudaStreamDestroy(cs);
    }
    tc_status init(int events) {
        if (events > 24) return fail(TC_ERR_INVALID_ARG, "copy lane: too many events");
        TC_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        for (; used < events; used++) TC_CUDA(cudaEventCreateWithFlags(&ev[used], cudaEventDisableTiming));
        return TC_OK;
    }
};

}  // namespace

namespace {

tc_status evolve_lowp_host_blocks(const double* U, double* rho_host, double* rho_dev, int n, int steps,
                                  int precision, int renorm_every, const Model* m, double* obs, Arena& ar,
                                  cudaStream_t s, CopyLane& lane);

}  // namespace

tc_status evolve_lowp_host(const double* U, double* rho_host, double* rho_dev, int n, int steps, int precision,
                           int renorm_every, const Model* m, double* obs, Arena& ar, cudaStream_t s) {
    CopyLane lane;
    const tc_status st = evolve_lowp_host_blocks(U, rho_host, rho_dev, n, steps, precision, renorm_every, m, obs, ar,
                                                 s, lane);
    if (st != TC_OK) {
        // copies already queued must not touch the caller's buffers after the call returns
        if (lane.cs) cudaStreamSynchronize(lane.cs);
        cudaStreamSynchronize(s);
    }
    return st;
}

namespace {

tc_status evolve_lowp_host_blocks(const double* U, double* rho_host, double* rho_dev, int n, int steps,
                                  int precision, int renorm_every, const Model* m, double* obs, Arena& ar,
                                  cudaStream_t s, CopyLane& lane) {
    const size_t N = (size_t)1 << n;
    const size_t bytes = 16 * N * N;
    const int C = steps >= 1 ? lowp_host_chunks(n, precision) : 1;
    const int CY = steps >= 1 ? lowp_host_bands(n, precision) : 1;
    // A page-locked rho_host is read and written by the SMs through its device
    // mapping (copy-engine transfers of host memory, reads above all, slow down
    // many-fold after heavy host CPU or memory activity; SM accesses keep
    // their rate); pageable or misaligned buffers go through the copy engine
    // and the device staging.
    const void* mapped_v = nullptr;
    TC_TRY(host_mapping(rho_host, &mapped_v));
    double* mapped = const_cast<double*>(static_cast<const double*>(mapped_v));
    if (C == 1 || CY == 1) {
        if (mapped)
            TC_TRY(copy_by_sms(rho_dev, mapped, bytes, s));
        else
            TC_CUDA(cudaMemcpyAsync(rho_dev, rho_host, bytes, cudaMemcpyHostToDevice, s));
        TC_TRY(evolve_lowp(U, rho_dev, n, steps, precision, renorm_every, m, obs, ar, s));
        if (mapped)
            TC_TRY(copy_by_sms(mapped, rho_dev, bytes, s));
        else
            TC_CUDA(cudaMemcpyAsync(rho_host, rho_dev, bytes, cudaMemcpyDeviceToHost, s));
        return TC_OK;
    }
    LowpBufs b{};
    TC_TRY(lowp_carve(n, precision, ar, b));
    if (b.Np != (int)N) return fail(TC_ERR_INVALID_ARG, "evolve: pipelined copies need N >= 128");
    StepPlan sp{};
    TC_TRY(plan_step(n, precision, b, sp));
    const int T = b.Np / 128;
    // executed FLOPs of one 128 x 128 complex output tile (K = Np, every part product)
    const double tile_flops = 8.0 * 128.0 * 128.0 * (double)b.Np * (double)cgemm_products(precision);
    const size_t R = N / C;                  // rows per block in
    const size_t chunk = 16 * R * N;         // bytes per block in
    const size_t RY = N / CY;                // rows per band out
    const int stride = TC_OBS_STRIDE(n);
    TC_TRY(lane.init(C + CY + 2));
    cudaEvent_t* in = lane.ev;               // [C] rows of block c are in the FP32 planes (or the staging)
    cudaEvent_t* fin = lane.ev + C;          // [CY] the rows of band c of rho' are final
    cudaEvent_t start = lane.ev[C + CY], done = lane.ev[C + CY + 1];
    auto dev_rows = [&](size_t c) { return reinterpret_cast<char*>(rho_dev) + c * chunk; };
    auto host_rows = [&](size_t c) { return reinterpret_cast<char*>(rho_host) + c * chunk; };
    auto rows_lo = [&](int c) { return (int)(c * R); };
    auto rows_hi = [&](int c) { return (int)((c + 1) * R); };
    auto band_lo = [&](int c) { return (int)(c * RY); };
    auto band_hi = [&](int c) { return (int)((c + 1) * RY); };
    // the SM reads of host rows run beside the first products: two CTAs per
    // SM keep the link busy without crowding the GEMM's CTAs
    int dev = 0, sms = 148;
    TC_CUDA(cudaGetDevice(&dev));
    TC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned cap = 2u * (unsigned)sms;
    const unsigned out_cap = (unsigned)sms / 2u > 0u ? (unsigned)sms / 2u : 1u;

    char tag[16];
    auto mark = [&](const char* what, int c, cudaStream_t on) {
        std::snprintf(tag, sizeof(tag), c >= 0 ? "%s%d" : "%s", what, c);
        phase_mark(tag, on);
    };
    // rho in by row blocks on the copy stream (after earlier work on s that may use the planes)
    mark("start", -1, s);
    TC_CUDA(cudaEventRecord(start, s));
    TC_CUDA(cudaStreamWaitEvent(lane.cs, start, 0));
    auto in_rows = [&](int c) -> tc_status {
        if (mapped)
            TC_TRY(lowp_prep_rho(precision, mapped, b, rows_lo(c), rows_hi(c), lane.cs, cap));
        else
            TC_CUDA(cudaMemcpyAsync(dev_rows(c), host_rows(c), chunk, cudaMemcpyHostToDevice, lane.cs));
        TC_CUDA(cudaEventRecord(in[c], lane.cs));
        mark("h2d", c, lane.cs);
        return TC_OK;
    };
    // all row blocks in at once, beside prep_u and the first product's column
    // blocks (an SM read beside a GEMM runs at a fraction of the link rate, so
    // holding the later blocks back made the column blocks wait for them)
    for (int c = 0; c < C; c++) TC_TRY(in_rows(c));
    TC_TRY(lowp_prep_u(precision, U, b, s));
    mark("prep_u", -1, s);
    // step 1, first product by column blocks: X[:, J] needs only the rows J of rho
    for (int c = 0; c < C; c++) {
        TC_CUDA(cudaStreamWaitEvent(s, in[c], 0));
        if (!mapped) TC_TRY(lowp_prep_rho(precision, rho_dev, b, rows_lo(c), rows_hi(c), s));
        CgemmEpi e = sp.e1;
        e.lo = c * T / C;
        e.hi = (c + 1) * T / C;
        {
            ProductTimer t(tile_flops * (double)T * (e.hi - e.lo), s);
            TC_TRY(cgemm_tc(precision, 0, sp.tmU, sp.tmR, e, s, sp.tune.tc_stages, &sp.wU, &sp.wR));
        }
        mark("x", c, s);
    }
    // rho' out once its entries are final (their products done on s).  A
    // mapped host buffer is written by the finish kernel on the copy stream,
    // on a few CTAs while products still run beside it (half a CTA per SM; SM
    // stores to host memory on more CTAs slowed the products by a quarter),
    // as the blocks that the row band c's product has just made final: its
    // own rows left of the band's right edge, and the rows above the band in
    // its columns (the mirrored tiles); the rows of band c right of it were
    // final, and went out, with the bands below.  So only the top band's
    // diagonal block is left to copy after the last product.  Otherwise the
    // rows are converted on s into the staging and copied by the copy engine.
    // Copy-engine writes to host memory slow down after heavy host activity
    // too, though less often than its reads.
    auto out_rows = [&](int c) -> tc_status {
        if (mapped) {
            TC_CUDA(cudaEventRecord(fin[c], s));
            TC_CUDA(cudaStreamWaitEvent(lane.cs, fin[c], 0));
            // the top band's block goes out last, with nothing beside it: the full grid
            const unsigned g = c == 0 ? cap : out_cap;
            TC_TRY(lowp_finish(b, mapped, lane.cs, band_lo(c), band_hi(c), g, 0, band_hi(c)));
            if (c > 0) TC_TRY(lowp_finish(b, mapped, lane.cs, 0, band_lo(c), g, band_lo(c), band_hi(c)));
        } else {
            TC_TRY(lowp_finish(b, rho_dev, s, band_lo(c), band_hi(c)));
            TC_CUDA(cudaEventRecord(fin[c], s));
            TC_CUDA(cudaStreamWaitEvent(lane.cs, fin[c], 0));
            char* off = reinterpret_cast<char*>(rho_dev) + 16 * (size_t)band_lo(c) * N;
            char* hoff = reinterpret_cast<char*>(rho_host) + 16 * (size_t)band_lo(c) * N;
            TC_CUDA(cudaMemcpyAsync(hoff, off, 16 * RY * N, cudaMemcpyDeviceToHost, lane.cs));
        }
        mark("d2h", c, lane.cs);
        return TC_OK;
    };
    if (obs) TC_TRY(launch_observables(kRhoPlanarF32, b.Rr, b.Ri, m, n, obs, b.scratch, s, (size_t)b.Np));
    for (int k = 1; k <= steps; k++) {
        if (k > 1) {
            ProductTimer t(tile_flops * (double)T * T, s);
            TC_TRY(cgemm_tc(precision, 0, sp.tmU, sp.tmR, sp.e1, s, sp.tune.tc_stages, &sp.wU, &sp.wR));
        }
        const bool renorm = renorm_every > 0 && k % renorm_every == 0;
        if (k < steps || renorm) {
            {
                ProductTimer t(tile_flops * 0.5 * T * (T + 1.0), s);
                TC_TRY(cgemm_tc(precision, 1, sp.tmU, sp.tmX, sp.e2, s, sp.tune.tc_stages, &sp.wU, &sp.wX));
            }
            if (renorm) TC_TRY(lowp_renorm(precision, b, s));
            if (obs) TC_TRY(launch_observables(kRhoPlanarF32, b.Rr, b.Ri, m, n, obs + (size_t)k * stride, b.scratch,
                                               s, (size_t)b.Np));
            if (k < steps) continue;
            // last step renormalised: rho' is whole only now; convert and copy out by row blocks
            mark("y", 0, s);
            for (int c = 0; c < CY; c++) TC_TRY(out_rows(c));
            break;
        }
        // last step, second product bottom-up by row bands: once the tile rows >= lo are done
        // (each tile writes itself and its mirror), the rows >= lo * 128 of rho' are final
        for (int c = CY - 1; c >= 0; c--) {
            CgemmEpi e = sp.e2;
            e.lo = c * T / CY;
            e.hi = (c + 1) * T / CY;
            {
                // the block-lower tiles of rows [lo, hi)
                ProductTimer t(tile_flops * 0.5 * ((double)e.hi * (e.hi + 1) - (double)e.lo * (e.lo + 1)), s);
                TC_TRY(cgemm_tc(precision, 1, sp.tmU, sp.tmX, e, s, sp.tune.tc_stages, &sp.wU, &sp.wX));
            }
            mark("y", c, s);
            TC_TRY(out_rows(c));
        }
        if (obs)
            TC_TRY(launch_observables(kRhoPlanarF32, b.Rr, b.Ri, m, n, obs + (size_t)k * stride, b.scratch, s,
                                      (size_t)b.Np));
    }
    TC_CUDA(cudaEventRecord(done, lane.cs));
    TC_CUDA(cudaStreamWaitEvent(s, done, 0));
    mark("done", -1, s);
    return TC_OK;
}

}  // namespace
}  // namespace tc
