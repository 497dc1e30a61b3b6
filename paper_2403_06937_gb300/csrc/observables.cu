// observables.cu -- the observable row of a density matrix (Sec. IV.A, Eq. 13)
// and the FP64 trace renormalisation of the low-precision forms.
//
// Row layout (TC_OBS_STRIDE(n) = 2n + 5 doubles):
//   P_1..P_n, <p>, P(0..n), Tr rho, Tr rho^2, E = Tr(H rho)
// P(m) is the weight of the basis states with popcount(s) = n - m, the
// projector reading of the photon-number states of Eq. 13.
//
// Deterministic two-pass reduction, no floating-point atomics: one warp per
// row (lanes stride the row for the purity sum, lanes < n take the n energy
// pairs of that row), warps fold in a fixed order into per-block partials,
// and a single block sums the partials in block order.  The grid size is a
// function of N only, so reruns are bitwise identical.
#include <mutex>

#include "kernels.cuh"

namespace tc {
namespace {

constexpr int kObsWarps = 8;
constexpr int kMaxStride = 2 * kMaxAtoms + 5;

unsigned obs_grid(int n) {
    unsigned rows = 1u << n;
    unsigned g = (rows + kObsWarps - 1) / kObsWarps;
    return g > 1024 ? 1024 : g;
}

template <int L>
struct Rho {
    const void* a;
    const void* b;
    size_t ld;   // row stride in elements
    __device__ __forceinline__ double re(size_t i) const {
        if (L == kRhoInterleaved) return static_cast<const double*>(a)[2 * i];
        if (L == kRhoPlanarF64) return static_cast<const double*>(a)[i];
        return (double)static_cast<const float*>(a)[i];
    }
    __device__ __forceinline__ double im(size_t i) const {
        if (L == kRhoInterleaved) return static_cast<const double*>(a)[2 * i + 1];
        if (L == kRhoPlanarF64) return static_cast<const double*>(b)[i];
        return (double)static_cast<const float*>(b)[i];
    }
};

template <int L>
__global__ void obs_partial_kernel(Rho<L> rho, Model m, int has_model, int n, double* partials) {
    __shared__ double acc[kObsWarps][kMaxStride];
    const int stride = 2 * n + 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = lane; j < stride; j += 32) acc[warp][j] = 0.0;
    __syncwarp();
    const unsigned N = 1u << n;
    double pur = 0.0, epair = 0.0;
    for (unsigned r = blockIdx.x * kObsWarps + warp; r < N; r += gridDim.x * kObsWarps) {
        const size_t row = (size_t)r * rho.ld;
        // four independent loads per lane in flight, fixed summation order
        double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
        unsigned c = lane;
        if (L == kRhoPlanarF32) {
            // FP32 planes: the squares of a chunk of 16 entries (4 per
            // accumulator) are summed in FP32 and only the chunk sums are
            // carried in FP64; per entry FP64 work (GB300's scarce FP64
            // issue) drops 40-fold, the sum's relative error stays within
            // ~17 FP32 ulps of a chunk's sum
            const float* ra = static_cast<const float*>(rho.a) + row;
            const float* rb = static_cast<const float*>(rho.b) + row;
            for (; c + 480 < N; c += 512) {
                float q0 = 0.f, q1 = 0.f, q2 = 0.f, q3 = 0.f;
#pragma unroll
                for (int h = 0; h < 4; h++) {
                    const unsigned b = c + 128 * h;
                    const float x0 = ra[b], x1 = ra[b + 32], x2 = ra[b + 64], x3 = ra[b + 96];
                    const float y0 = rb[b], y1 = rb[b + 32], y2 = rb[b + 64], y3 = rb[b + 96];
                    q0 = fmaf(x0, x0, fmaf(y0, y0, q0));
                    q1 = fmaf(x1, x1, fmaf(y1, y1, q1));
                    q2 = fmaf(x2, x2, fmaf(y2, y2, q2));
                    q3 = fmaf(x3, x3, fmaf(y3, y3, q3));
                }
                p0 += (double)((q0 + q1) + (q2 + q3));
            }
        }
        for (; c + 96 < N; c += 128) {
            const double x0 = rho.re(row + c), x1 = rho.re(row + c + 32), x2 = rho.re(row + c + 64),
                         x3 = rho.re(row + c + 96);
            const double y0 = rho.im(row + c), y1 = rho.im(row + c + 32), y2 = rho.im(row + c + 64),
                         y3 = rho.im(row + c + 96);
            p0 += x0 * x0 + y0 * y0;
            p1 += x1 * x1 + y1 * y1;
            p2 += x2 * x2 + y2 * y2;
            p3 += x3 * x3 + y3 * y3;
        }
        for (; c < N; c += 32) {
            const double x = rho.re(row + c), y = rho.im(row + c);
            p0 += x * x + y * y;
        }
        pur += (p0 + p1) + (p2 + p3);
        // energy pair of atom `lane` when that atom is excited in r
        if (has_model && lane < n) {
            unsigned bit = 1u << (n - 1 - lane);
            if (r & bit) {
                unsigned sg = r & ~bit;
                double h = m.coupling == TC_COUPLING_QUBIT_PHOTON
                               ? m.g[lane]
                               : m.g[lane] * sqrt((double)(n - __popc(r) + 1));
                epair += h * (rho.re(row + sg) + rho.re((size_t)sg * rho.ld + r));
            }
        }
        if (lane == 0) {
            double d = rho.re(row + r);
            int pc = __popc(r);
            for (int i = 0; i < n; i++)
                if ((r >> (n - 1 - i)) & 1u) acc[warp][i] += d;
            acc[warp][n] += d * (double)(n - pc);
            acc[warp][n + 1 + (n - pc)] += d;
            acc[warp][2 * n + 2] += d;
            if (has_model) acc[warp][2 * n + 4] += (m.omega_c * (double)(n - pc) + m.omega_a * (double)pc) * d;
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
        double s = 0.0;
        for (int w = 0; w < kObsWarps; w++) s += acc[w][j];
        partials[(size_t)blockIdx.x * stride + j] = s;
    }
}

__global__ void obs_final_kernel(const double* partials, int blocks, int stride, double* out) {
    for (int j = threadIdx.x; j < stride; j += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < blocks; b++) s += partials[(size_t)b * stride + j];
        out[j] = s;
    }
}

// trace of the planar diagonal in FP64, one block, fixed order
template <typename T>
__global__ void trace_kernel(const T* re, unsigned N, double* out) {
    __shared__ double s[1024];
    double a = 0.0;
    for (unsigned i = threadIdx.x; i < N; i += blockDim.x) a += (double)re[(size_t)i * N + i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (unsigned w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = s[0];
}

template <typename T>
__global__ void scale_kernel(T* re, T* im, size_t count, const double* trace, unsigned* status) {
    double tr = trace[0];
    if (!(tr > 0.0) || !isfinite(tr)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kStatusNumeric);
        return;
    }
    double inv = 1.0 / tr;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x) {
        re[i] = (T)((double)re[i] * inv);
        im[i] = (T)((double)im[i] * inv);
    }
}

// sum_s O_s Re rho[s][s] of an interleaved complex128 rho; one block, fixed order
__global__ void expectation_diag_kernel(const double* rho, const double* O, unsigned N, double* out) {
    __shared__ double s[1024];
    double a = 0.0;
    for (unsigned i = threadIdx.x; i < N; i += blockDim.x) a += O[i] * rho[2 * ((size_t)i * N + i)];
    s[threadIdx.x] = a;
    __syncthreads();
    for (unsigned w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = s[0];
}

}  // namespace

size_t observables_scratch_bytes(int n) {
    return round256((size_t)obs_grid(n) * (2 * n + 5) * sizeof(double)) + 256;
}

tc_status launch_observables(int layout, const void* a, const void* b, const Model* m, int n,
                             double* out, double* scratch, cudaStream_t s, size_t ld) {
    if (ld == 0) ld = (size_t)1 << n;
    unsigned grid = obs_grid(n);
    Model mm{};
    int has = 0;
    if (m) {
        mm = *m;
        has = 1;
    }
    mm.n = n;
    switch (layout) {
        case kRhoInterleaved:
            obs_partial_kernel<kRhoInterleaved><<<grid, 32 * kObsWarps, 0, s>>>(Rho<kRhoInterleaved>{a, b, ld}, mm, has, n, scratch);
            break;
        case kRhoPlanarF64:
            obs_partial_kernel<kRhoPlanarF64><<<grid, 32 * kObsWarps, 0, s>>>(Rho<kRhoPlanarF64>{a, b, ld}, mm, has, n, scratch);
            break;
        case kRhoPlanarF32:
            obs_partial_kernel<kRhoPlanarF32><<<grid, 32 * kObsWarps, 0, s>>>(Rho<kRhoPlanarF32>{a, b, ld}, mm, has, n, scratch);
            break;
        default:
            return fail(TC_ERR_INVALID_ARG, "observables: unknown layout");
    }
    TC_LAUNCH_CHECK();
    obs_final_kernel<<<1, 64, 0, s>>>(scratch, (int)grid, 2 * n + 5, out);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

tc_status launch_renormalise(int layout, void* re, void* im, int n, double* scratch, cudaStream_t s) {
    unsigned N = 1u << n;
    size_t count = (size_t)N * N;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    unsigned grid = (unsigned)sms * 8;
    if (layout == kRhoPlanarF64) {
        trace_kernel<double><<<1, 1024, 0, s>>>(static_cast<double*>(re), N, scratch);
        TC_LAUNCH_CHECK();
        scale_kernel<double><<<grid, 256, 0, s>>>(static_cast<double*>(re), static_cast<double*>(im), count,
                                                  scratch, device_status_word());
    } else if (layout == kRhoPlanarF32) {
        trace_kernel<float><<<1, 1024, 0, s>>>(static_cast<float*>(re), N, scratch);
        TC_LAUNCH_CHECK();
        scale_kernel<float><<<grid, 256, 0, s>>>(static_cast<float*>(re), static_cast<float*>(im), count,
                                                 scratch, device_status_word());
    } else {
        return fail(TC_ERR_INVALID_ARG, "renormalise: planar layouts only");
    }
    TC_LAUNCH_CHECK();
    return TC_OK;
}

}  // namespace tc

extern "C" TC_API tc_status tc_expectation_diag(const void* rho, int n, const double* O_diag, double* out,
                                                void* stream) {
    using namespace tc;
    if (n < 1 || n > kMaxAtoms) return fail(TC_ERR_INVALID_ARG, "n = %d outside 1..16", n);
    if (!rho || !O_diag || !out) return fail(TC_ERR_INVALID_ARG, "rho, O_diag or out is NULL");
    if ((reinterpret_cast<uintptr_t>(rho) | reinterpret_cast<uintptr_t>(O_diag) | reinterpret_cast<uintptr_t>(out)) &
        7u)
        return fail(TC_ERR_INVALID_ARG, "rho, O_diag and out must be 8-byte aligned");
    TC_TRY(check_device());
    expectation_diag_kernel<<<1, 1024, 0, as_stream(stream)>>>(static_cast<const double*>(rho), O_diag, 1u << n,
                                                               out);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

// ---------------------------------------------------------------------------
// tc_observables_noalloc: the same two kernels with their per-block partial
// sums in a fixed device array instead of a caller-provided work buffer.
//
// The array is sized for the largest grid the observables use (1024 blocks)
// times the widest row (n = 16: 37 doubles), 296 KiB.  It is file-scope
// device memory: every GPU that loads this library holds it until the
// process exits.  All calls share it, so calls that overlap on the GPU
// (different streams, or different host threads on one device) race on it.
// Nothing in it has to start at zero: the first kernel writes every slot the
// second kernel reads, in the same call.
namespace tc {
namespace {
constexpr size_t kNoAllocPartials = 1024 * (2 * kMaxAtoms + 5);
static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64];   // device address of the array, per device
}  // namespace

}  // namespace tc

extern "C" TC_API tc_status tc_observables_noalloc(const void* rho, int n, const tc_params* params, double* out,
                                                   void* stream) {
    using namespace tc;
    if (n < 1 || n > kMaxAtoms) return fail(TC_ERR_INVALID_ARG, "n = %d outside 1..16", n);
    if (!rho || !out) return fail(TC_ERR_INVALID_ARG, "rho or out is NULL");
    if ((reinterpret_cast<uintptr_t>(rho) | reinterpret_cast<uintptr_t>(out)) & 7u)
        return fail(TC_ERR_INVALID_ARG, "rho and out must be 8-byte aligned");
    const size_t need = (size_t)obs_grid(n) * (size_t)(2 * n + 5);
    if (need > kNoAllocPartials)
        return fail(TC_ERR_INVALID_ARG,
                    "tc_observables_noalloc: n = %d needs %zu doubles of scratch, the fixed array holds %zu",
                    n, need, kNoAllocPartials);
    Model m;
    if (params) {
        TC_TRY(make_model(params, &m));
        if (m.n != n) return fail(TC_ERR_INVALID_ARG, "params->n != n");
    }
    TC_TRY(check_device());
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(TC_ERR_UNSUPPORTED_DEVICE, "device index %d out of range", dev);
    double* partials = nullptr;
    {
        // first call on this device: resolve the array's device address with
        // the device current (the array's name in host code is not that address)
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess)
                return fail(TC_ERR_CUDA, "cudaGetSymbolAddress(observables scratch): %s", cudaGetErrorString(e));
            g_noalloc_ptr[dev] = static_cast<double*>(p);
        }
        partials = g_noalloc_ptr[dev];
    }
    return launch_observables(kRhoInterleaved, rho, nullptr, params ? &m : nullptr, n, out, partials,
                              as_stream(stream));
}
