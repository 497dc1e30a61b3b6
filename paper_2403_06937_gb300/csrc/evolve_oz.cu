// evolve_oz.cu -- the FP64-accurate tensor-core form of the step loop
// rho <- U rho U^dag (Sec. III.A, Eqs. 6, 12): both products on the BF16
// tensor cores from exact integer slices (cgemm_oz.cu), rho and X kept in
// FP64 planes (row stride Np = max(N, 128), zero padding).
//
// Per step: slice rho, X = U rho^H (all tiles), slice X, rho' = U X^H
// (block-lower tiles, then the mirrored upper half), observables from the
// FP64 planes; U is sliced once per call.  U enters as it is (no increment
// form): the slice products are exact, so there is no accumulation bias to
// scale down.
#include "cgemm_oz.cuh"
#include "cgemm_tc.cuh"
#include "graph.cuh"
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

// interleaved N x N complex128 -> FP64 planes of stride Np (zero outside N x N)
__global__ void split_pad_kernel(const double2* __restrict__ src, int N, int Np, double* __restrict__ re,
                                 double* __restrict__ im) {
    const size_t count = (size_t)Np * Np;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = e / Np, j = e % Np;
        double2 v = make_double2(0.0, 0.0);
        if (i < (size_t)N && j < (size_t)N) v = src[i * N + j];
        re[e] = v.x;
        im[e] = v.y;
    }
}

__global__ void join_pad_kernel(const double* __restrict__ re, const double* __restrict__ im, int N, int Np,
                                double2* __restrict__ dst) {
    const size_t count = (size_t)N * N;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = e / N, j = e % N;
        dst[e] = make_double2(re[i * Np + j], im[i * Np + j]);
    }
}

// trace of the N x N block in FP64 (one CTA, fixed order), then rho / trace
__global__ void trace_pad_kernel(const double* __restrict__ re, int N, int Np, double* __restrict__ out) {
    __shared__ double sh[1024];
    double a = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) a += re[(size_t)i * Np + i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

__global__ void scale_pad_kernel(double* __restrict__ re, double* __restrict__ im, int Np,
                                 const double* __restrict__ trace, unsigned* status) {
    const double tr = trace[0];
    if (!(tr > 0.0) || !isfinite(tr)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kStatusNumeric);
        return;
    }
    const double inv = 1.0 / tr;
    const size_t count = (size_t)Np * Np;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
        re[e] *= inv;
        im[e] *= inv;
    }
}

int padded_dim(int n) { return (1 << n) < 128 ? 128 : (1 << n); }

}  // namespace

size_t evolve_oz_bytes(int n) {
    const size_t Np = (size_t)padded_dim(n);
    return 2 * oz_mat_bytes((int)Np) + 6 * round256(Np * Np * sizeof(double)) + observables_scratch_bytes(n) + 512;
}

tc_status OzSystem::carve(int n_, Arena& ar) {
    n = n_;
    N = 1 << n;
    Np = padded_dim(n);
    const size_t NN = (size_t)Np * Np;
    TC_TRY(oz_mat_init(Us, ar, Np));
    TC_TRY(oz_mat_init(Ps, ar, Np));
    Rr = ar.take<double>(NN);
    Ri = ar.take<double>(NN);
    Xr = ar.take<double>(NN);
    Xi = ar.take<double>(NN);
    Lr = ar.take<long long>(NN);   // low-level integer sums of the products
    Li = ar.take<long long>(NN);
    scratch = ar.take<double>(observables_scratch_bytes(n) / sizeof(double));
    if (!scratch) return fail(TC_ERR_WORKSPACE, "evolve: workspace too small");
    group = tune_lookup(n, TC_BF16X3).tc_group;
    return TC_OK;
}

tc_status OzSystem::first(const double* U, const double* rho, const Model* m_, double* obs_, int renorm_every_,
                          cudaStream_t cs) {
    m = m_;
    obs = obs_;
    renorm_every = renorm_every_;
    const size_t NN = (size_t)Np * Np;
    TC_TRY(oz_mat_load(Us, U, nullptr, true, false, N, (size_t)N, cs));
    split_pad_kernel<<<grid_for(NN), 256, 0, cs>>>(reinterpret_cast<const double2*>(rho), N, Np, Rr, Ri);
    TC_LAUNCH_CHECK();
    if (obs) TC_TRY(launch_observables(kRhoPlanarF64, Rr, Ri, m, n, obs, scratch, cs, (size_t)Np));
    return TC_OK;
}

tc_status OzSystem::step(int k, cudaStream_t cs) {
    const size_t NN = (size_t)Np * Np;
    const double N3 = (double)N * N * N;
    const OzOut X{Xr, Xi, Lr, Li}, R{Rr, Ri, Lr, Li};
    TC_TRY(oz_mat_load(Ps, Rr, Ri, false, false, N, (size_t)Np, cs));
    {
        ProductTimer t(8.0 * N3 * Us.dg.pairs, cs);   // X = U rho^H
        TC_TRY(oz_product(0, Us, Ps, X, group, cs));
    }
    TC_TRY(oz_mat_load(Ps, Xr, Xi, false, false, N, (size_t)Np, cs));
    {
        ProductTimer t(4.0 * N3 * Us.dg.pairs, cs);   // rho' = U X^H, Hermitian half + mirror
        TC_TRY(oz_product(1, Us, Ps, R, group, cs));
    }
    if (renorm_every > 0 && k % renorm_every == 0) {
        trace_pad_kernel<<<1, 1024, 0, cs>>>(Rr, N, Np, scratch);
        TC_LAUNCH_CHECK();
        scale_pad_kernel<<<grid_for(NN), 256, 0, cs>>>(Rr, Ri, Np, scratch, device_status_word());
        TC_LAUNCH_CHECK();
    }
    if (obs)
        TC_TRY(launch_observables(kRhoPlanarF64, Rr, Ri, m, n, obs + (size_t)k * TC_OBS_STRIDE(n), scratch, cs,
                                  (size_t)Np));
    return TC_OK;
}

tc_status OzSystem::tail(double* rho, cudaStream_t cs) {
    join_pad_kernel<<<grid_for((size_t)N * N), 256, 0, cs>>>(Rr, Ri, N, Np, reinterpret_cast<double2*>(rho));
    TC_LAUNCH_CHECK();
    return TC_OK;
}

tc_status evolve_oz(const double* U, double* rho, int n, int steps, int renorm_every, const Model* m, double* obs,
                    Arena& ar, cudaStream_t s) {
    OzSystem z;
    TC_TRY(z.carve(n, ar));
    auto first = [&](cudaStream_t cs) -> tc_status {
        TC_TRY(z.first(U, rho, m, obs, renorm_every, cs));
        if (steps >= 1) TC_TRY(z.step(1, cs));
        return TC_OK;
    };
    auto rest = [&](cudaStream_t cs) -> tc_status {
        for (int k = 2; k <= steps; k++) TC_TRY(z.step(k, cs));
        return TC_OK;
    };
    auto tail = [&](cudaStream_t cs) -> tc_status { return z.tail(rho, cs); };
    return run_captured(s, first, rest, tail, steps > 2 && !timing_enabled());
}

}  // namespace tc
