// elementwise.cu -- layout conversions and the small element-wise and
// reduction kernels around the products: complex128 <-> planar planes, the
// shift/scale and linear combinations of the Taylor polynomial (Sec. III.A,
// Eqs. 7-8, 10), the final phase/symmetrisation of e^{-iHdt}, and the trace
// and 1-norm used to plan the series.  All are HBM-bound, grid-stride loops
// sized to a multiple of the SM count.
#include "kernels.cuh"

namespace tc {
namespace {

unsigned grid_for(size_t work, int per_block = 256) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t want = (work + per_block - 1) / per_block;
    size_t cap = (size_t)sms * 16;
    if (want > cap) want = cap;
    return (unsigned)(want ? want : 1);
}

#define GRID_STRIDE(i, count)                                                         \
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (count);      \
         i += (size_t)gridDim.x * blockDim.x)

// 16-byte grid-stride copy: the SMs read or write page-locked host memory
// directly through its device mapping
__global__ void copy16_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst, size_t count) {
    GRID_STRIDE(i, count) { dst[i] = src[i]; }
}

__global__ void split_c128_kernel(const double2* src, double* re, double* im, size_t count) {
    GRID_STRIDE(i, count) {
        double2 v = src[i];
        re[i] = v.x;
        im[i] = v.y;
    }
}
__global__ void join_c128_kernel(const double* re, const double* im, double2* dst, size_t count) {
    GRID_STRIDE(i, count) { dst[i] = make_double2(re[i], im[i]); }
}
__global__ void split_c128_f32_kernel(const double2* src, float* re, float* im, size_t count) {
    GRID_STRIDE(i, count) {
        double2 v = src[i];
        re[i] = (float)v.x;
        im[i] = (float)v.y;
    }
}
__global__ void join_c128_f32_kernel(const float* re, const float* im, double2* dst, size_t count) {
    GRID_STRIDE(i, count) { dst[i] = make_double2((double)re[i], (double)im[i]); }
}

struct LinComb {
    const double* m[4];
    double c[4];
    int terms;
    double cid;
};
__global__ void lincomb_kernel(LinComb lc, double* out, unsigned N) {
    size_t count = (size_t)N * N;
    GRID_STRIDE(i, count) {
        double v = 0.0;
        for (int t = 0; t < lc.terms; t++) v += lc.c[t] * lc.m[t][i];
        if ((i / N) == (i % N)) v += lc.cid;
        out[i] = v;
    }
}

__global__ void shift_scale_kernel(const double* H, double mu, double dt, double* B, unsigned N) {
    size_t count = (size_t)N * N;
    GRID_STRIDE(i, count) {
        double h = H[i];
        if ((i / N) == (i % N)) h -= mu;
        B[i] = h * dt;
    }
}

// U = e^{-i phi} (C - i S), symmetrised: U_ij <- (U_ij + U_ji) / 2.
__global__ void expm_finish_kernel(const double* C, const double* S, double pr, double pi,
                                   double2* U, unsigned N) {
    size_t count = (size_t)N * N;
    GRID_STRIDE(e, count) {
        size_t i = e / N, j = e % N;
        size_t t = j * N + i;
        double c = 0.5 * (C[e] + C[t]);
        double s = 0.5 * (S[e] + S[t]);
        // (pr + i pi)(c - i s) = (pr c + pi s) + i (pi c - pr s)
        U[e] = make_double2(pr * c + pi * s, pi * c - pr * s);
    }
}

// per-row sum of |A_ij - mu delta_ij| (A symmetric: equals the column sum); one warp per row
__global__ void row_abs_sum_kernel(const double* A, double mu, unsigned N, double* rows, double* diag) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (unsigned r = warp; r < N; r += nwarps) {
        double acc = 0.0;
        const double* row = A + (size_t)r * N;
        for (unsigned c = lane; c < N; c += 32) {
            double v = row[c];
            if (c == r) v -= mu;
            acc += fabs(v);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            rows[r] = acc;
            diag[r] = row[r];
        }
    }
}

// one block: out[0] = max rows[], out[1] = sum diag[] in a fixed order
__global__ void max_sum_kernel(const double* rows, const double* diag, unsigned N, double* out) {
    __shared__ double smax[1024], ssum[1024];
    double mx = 0.0, sm = 0.0;
    for (unsigned i = threadIdx.x; i < N; i += blockDim.x) {
        mx = fmax(mx, rows[i]);
        sm += diag[i];
    }
    smax[threadIdx.x] = mx;
    ssum[threadIdx.x] = sm;
    __syncthreads();
    for (unsigned w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + w]);
            ssum[threadIdx.x] += ssum[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = smax[0];
        out[1] = ssum[0];
    }
}

}  // namespace

tc_status host_mapping(const void* host, const void** dev) {
    *dev = nullptr;
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, host);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();   // pageable memory on older drivers reports an error: not mapped
        return TC_OK;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return TC_OK;
    if (reinterpret_cast<uintptr_t>(a.devicePointer) & 15u) return TC_OK;
    *dev = a.devicePointer;
    return TC_OK;
}

tc_status copy_by_sms(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15u) || (bytes & 15u))
        return fail(TC_ERR_INVALID_ARG, "copy_by_sms: 16-byte aligned addresses and size required");
    const size_t count = bytes / 16;
    copy16_kernel<<<grid_for(count), 256, 0, s>>>(static_cast<const uint4*>(src), static_cast<uint4*>(dst), count);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

tc_status launch_split_c128(const double* src, double* re, double* im, size_t count, cudaStream_t s) {
    split_c128_kernel<<<grid_for(count), 256, 0, s>>>(reinterpret_cast<const double2*>(src), re, im, count);
    TC_LAUNCH_CHECK();
    return TC_OK;
}
tc_status launch_join_c128(const double* re, const double* im, double* dst, size_t count, cudaStream_t s) {
    join_c128_kernel<<<grid_for(count), 256, 0, s>>>(re, im, reinterpret_cast<double2*>(dst), count);
    TC_LAUNCH_CHECK();
    return TC_OK;
}
tc_status launch_split_c128_f32(const double* src, float* re, float* im, size_t count, cudaStream_t s) {
    split_c128_f32_kernel<<<grid_for(count), 256, 0, s>>>(reinterpret_cast<const double2*>(src), re, im, count);
    TC_LAUNCH_CHECK();
    return TC_OK;
}
tc_status launch_join_c128_f32(const float* re, const float* im, double* dst, size_t count, cudaStream_t s) {
    join_c128_f32_kernel<<<grid_for(count), 256, 0, s>>>(re, im, reinterpret_cast<double2*>(dst), count);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

tc_status launch_lincomb(int N, double c_identity, int terms, const double* const* mats,
                         const double* coef, double* out, cudaStream_t s) {
    if (terms < 0 || terms > 4) return fail(TC_ERR_INVALID_ARG, "lincomb: at most 4 terms");
    LinComb lc{};
    for (int t = 0; t < terms; t++) {
        lc.m[t] = mats[t];
        lc.c[t] = coef[t];
    }
    lc.terms = terms;
    lc.cid = c_identity;
    size_t count = (size_t)N * N;
    lincomb_kernel<<<grid_for(count), 256, 0, s>>>(lc, out, (unsigned)N);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

tc_status launch_shift_scale(int N, const double* H, double mu, double dt, double* B, cudaStream_t s) {
    size_t count = (size_t)N * N;
    shift_scale_kernel<<<grid_for(count), 256, 0, s>>>(H, mu, dt, B, (unsigned)N);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

tc_status launch_expm_finish(int N, const double* Cm, const double* Sm, double phase_re,
                             double phase_im, double* U, cudaStream_t s) {
    size_t count = (size_t)N * N;
    expm_finish_kernel<<<grid_for(count), 256, 0, s>>>(Cm, Sm, phase_re, phase_im,
                                                       reinterpret_cast<double2*>(U), (unsigned)N);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

tc_status matrix_trace_and_norm1(int N, const double* H, double mu_for_norm, double* trace,
                                 double* norm1, double* scratch, cudaStream_t s) {
    double* rows = scratch;
    double* diag = scratch + N;
    double* out = scratch + 2 * (size_t)N;
    row_abs_sum_kernel<<<grid_for((size_t)N * 32), 256, 0, s>>>(H, mu_for_norm, (unsigned)N, rows, diag);
    TC_LAUNCH_CHECK();
    max_sum_kernel<<<1, 1024, 0, s>>>(rows, diag, (unsigned)N, out);
    TC_LAUNCH_CHECK();
    double host[2];
    TC_CUDA(cudaMemcpyAsync(host, out, sizeof(host), cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    *norm1 = host[0];
    *trace = host[1];
    return TC_OK;
}

}  // namespace tc
