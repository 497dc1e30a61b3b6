// cgemm_tc.cu -- complex GEMM Y = U P^H on the sm_103a tensor cores
// (tcgen05.mma, operands staged by TMA, FP32 accumulators in TMEM) for the
// low-precision forms of the step rho <- U rho U^dag (Sec. III.A, Eqs. 6, 12).
//
// Both products of a step have this one shape, because U is complex symmetric
// (U^T = U, H real symmetric) and rho is Hermitian:
//     X   = U rho   = U rho^H           (P = rho)
//     rho' = X U^dag = (U X^H)^H = U X^H (rho' Hermitian; P = X)
// so a kernel computing Y = U P^H for a row-major P serves both, with P
// read K-major exactly as it is stored.
//
// Tile: one CTA computes the complex 128 x 128 tile Y[I, J].  A operands are
// the row tiles U_r[I], U_i[I] (M = 128); the B operand is the 256-row stack
// [P_r[J]; P_i[J]] (N = 256), shared by both MMAs.  Two FP32 accumulators in
// TMEM (2 x 256 columns):
//     D1 = U_r [P_r; P_i]^T = [U_r P_r^T | U_r P_i^T]
//     D2 = U_i [P_r; P_i]^T = [U_i P_r^T | U_i P_i^T]
// and the epilogue forms Y_r = U_r P_r^T + U_i P_i^T, Y_i = U_i P_r^T - U_r P_i^T.
//
// Increment form: the operand is V = U / c - I (c = Tr U / |Tr U|, a unit
// phase that cancels in U rho U^dag), and the epilogue adds the identity
// term P^H exactly in FP32.  The tensor cores then only accumulate V P^H,
// of size ||V|| |P| (a few hundredths here), so the truncation of their FP32
// accumulation (round toward zero, a systematic shrink of every running sum)
// is scaled down by ||V|| instead of acting on sums of size |P|.
//
// Precision forms: every FP32 (or FP64) operand x is held as S parts
// (BF16x3: three BF16 parts x0 + x1 + x2; TF32: one TF32 part; TF32x3: a
// big and a small TF32 part) and the product of two split operands is the
// sum of the part products whose order is below the FP32 rounding level
// (BF16x3: six products, TF32x3: three).  All S parts of every operand for a
// 32-byte slice of K sit in one pipeline stage, and all part products of the
// stage are issued from it, so each operand byte crosses L2 -> SMEM once.
//
// Roles (192 threads): warp 4 lane 0 issues TMA loads into a ring of STAGES
// stages; warp 5 lane 0 issues tcgen05.mma and commits each stage back to the
// producer; warps 0-3 (one TMEM lane quarter each) run the epilogue.  Every
// wait is bounded: on timeout the CTA records kStatusTimeout, stops issuing,
// waits (bounded) for its own copies and MMAs, frees TMEM and returns.
#include <cuda_bf16.h>

#include <atomic>

#include "cgemm_dev.cuh"
#include "cgemm_tc.cuh"

namespace tc {
namespace {

using namespace sm100;
using namespace cg;

constexpr int kThreads = 192;

template <int KIND, int S, int STAGES, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    cgemm_tc_kernel(const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmP, CgemmEpi ep) {
    constexpr int kStage = 2 * S * kATile + S * kBTile;
    constexpr int kElem = KIND == 0 ? 2 : 4;
    constexpr int kKPerStage = kRowBytes / kElem;   // K elements per stage (one MMA K-step)
    constexpr uint32_t kIdesc = make_idesc(KIND == 0 ? 1u : 2u, 128u, 256u);

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * kStage);
    uint64_t* empty = full + STAGES;
    uint64_t* accum = empty + STAGES;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t lim = ep.wait_ns ? ep.wait_ns : kWaitLimitNs;
    int I, J;
    tile_of_range(MODE, ep.tiles, ep.group, ep.lo, ep.hi > 0 ? ep.hi : ep.tiles, blockIdx.x, I, J);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(saddr(tmem_slot), 512);
        tmem_relinquish();
    }
    if (warp == 4 && lane == 0) {
        prefetch_tmap(&tmU);
        prefetch_tmap(&tmP);
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int KB = ep.Np / kKPerStage;

    if (warp == 4) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            int issued = 0;
            for (int kb = 0; kb < KB; kb++) {
                const int s = kb % STAGES;
                const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
                if (!mbar_wait_bounded(&empty[s], ph ^ 1u, abort, lim, 0)) break;
                if (ep.withhold && kb == 0) continue;   // injected fault: stage 0 is never filled
                mbar_arrive_expect_tx(&full[s], kStage);
                uint8_t* st = smem + s * kStage;
                const uint32_t fb = saddr(&full[s]);
                const int kx = kb * kKPerStage;
#pragma unroll
                for (int part = 0; part < 2; part++)
#pragma unroll
                    for (int a = 0; a < S; a++)
                        tma_load_3d(saddr(st + (part * S + a) * kATile), &tmU, fb, kx, I * 128, part * S + a);
#pragma unroll
                for (int b = 0; b < S; b++) {
                    uint8_t* bt = st + 2 * S * kATile + b * kBTile;
                    tma_load_3d(saddr(bt), &tmP, fb, kx, J * 128, b);                   // P_r part b
                    tma_load_3d(saddr(bt + 128 * kRowBytes), &tmP, fb, kx, J * 128, S + b);   // P_i part b
                }
                issued = kb + 1;
            }
            if (*abort) {
                // let the copies already issued land before the CTA goes away
                for (int kb = issued - STAGES > 0 ? issued - STAGES : 0; kb < issued; kb++)
                    if (!(ep.withhold && kb == 0))
                        (void)mbar_wait_bounded(&full[kb % STAGES], (uint32_t)(kb / STAGES) & 1u, nullptr,
                                                lim, 0);
            }
        }
    } else if (warp == 5) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            for (int kb = 0; kb < KB; kb++) {
                const int s = kb % STAGES;
                const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
                if (!mbar_wait_bounded(&full[s], ph, abort, lim, 0)) break;
                tc_fence_after();
                uint8_t* st = smem + s * kStage;
#pragma unroll
                for (int p = 0; p < Pairs<S>::n; p++) {
                    const uint64_t bd = desc_kmajor_sw32(saddr(st + 2 * S * kATile + Pairs<S>::b(p) * kBTile));
#pragma unroll
                    for (int part = 0; part < 2; part++) {
                        const uint64_t ad = desc_kmajor_sw32(saddr(st + (part * S + Pairs<S>::a(p)) * kATile));
                        umma<KIND>(tmem + part * 256, ad, bd, kIdesc, (kb > 0 || p > 0) ? 1u : 0u);
                    }
                }
                umma_commit(saddr(&empty[s]));
            }
            // always: completes when every MMA issued above has finished
            umma_commit(saddr(accum));
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const bool ok = mbar_wait_bounded(accum, 0u, abort, lim, 128);
        tc_fence_after();
        if (ok && !*abort)
            cg::epilogue_tile<KIND, S, MODE>(tmem, warp, lane, I, J, ep.Np, ep.pr, ep.pi, ep.parts, ep.yr, ep.yi);
        if (!ok || *abort) {
            if (threadIdx.x == 0) atomicOr(ep.status, kStatusTimeout);
        }
    }

    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

template <int KIND, int S, int STAGES>
constexpr int smem_bytes() {
    return STAGES * (2 * S * kATile + S * kBTile) + 1024 /*align*/ + 256 /*barriers*/;
}

template <int KIND, int S, int STAGES, int MODE>
tc_status launch(const CUtensorMap& tmU, const CUtensorMap& tmP, const CgemmEpi& ep, cudaStream_t s) {
    auto k = cgemm_tc_kernel<KIND, S, STAGES, MODE>;
    constexpr int smem = smem_bytes<KIND, S, STAGES>();
    static bool attr_set[64] = {};   // per device; set before the first launch there
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(TC_ERR_UNSUPPORTED_DEVICE, "device index out of range");
    if (!attr_set[dev]) {
        TC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr_set[dev] = true;
    }
    const int T = ep.tiles;
    const int lo = ep.hi > 0 ? ep.lo : 0, hi = ep.hi > 0 ? ep.hi : T;
    const unsigned grid =
        MODE == 0 ? (unsigned)(T * (hi - lo)) : (unsigned)((hi * (hi + 1) - lo * (lo + 1)) / 2);
    k<<<grid, kThreads, smem, s>>>(tmU, tmP, ep);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

}  // namespace

namespace {
std::atomic<int> g_inject_count{0};
std::atomic<unsigned long long> g_inject_wait{0};
}  // namespace

void cgemm_inject_timeout(int count, unsigned long long wait_ns) {
    g_inject_wait.store(wait_ns);
    g_inject_count.store(count);
}

int cgemm_default_stages(int precision) { return precision == TC_BF16X3 ? 4 : precision == TC_TF32X3 ? 6 : 8; }
int cgemm_alt_stages(int precision) { return precision == TC_BF16X3 ? 3 : precision == TC_TF32X3 ? 3 : 4; }

tc_status cgemm_tc(int precision, int mode, const CUtensorMap& tmU, const CUtensorMap& tmP, const CgemmEpi& ep_in,
                   cudaStream_t s, int stages) {
    CgemmEpi ep = ep_in;
    if (g_inject_count.load() > 0 && g_inject_count.fetch_sub(1) > 0) {
        ep.withhold = 1;
        ep.wait_ns = g_inject_wait.load();
    }
    if (ep.Np < 128 || ep.Np % 128 != 0 || ep.tiles * 128 != ep.Np)
        return fail(TC_ERR_INVALID_ARG, "cgemm_tc: padded dimension must be a multiple of 128");
    if (mode != 0 && mode != 1) return fail(TC_ERR_INVALID_ARG, "cgemm_tc: mode");
    if (ep.hi > 0) {
        const int G = ep.group < 1 ? 1 : ep.group;
        if (ep.lo < 0 || ep.lo >= ep.hi || ep.hi > ep.tiles)
            return fail(TC_ERR_INVALID_ARG, "cgemm_tc: tile range [%d, %d) outside [0, %d)", ep.lo, ep.hi, ep.tiles);
        if (mode == 1 && (ep.lo % G != 0 || (ep.hi % G != 0 && ep.hi != ep.tiles)))
            return fail(TC_ERR_INVALID_ARG, "cgemm_tc: row range [%d, %d) not aligned to the group %d", ep.lo,
                        ep.hi, G);
    }
    if (stages == 0) stages = cgemm_default_stages(precision);
    const bool alt = stages == cgemm_alt_stages(precision);
    if (!alt && stages != cgemm_default_stages(precision))
        return fail(TC_ERR_INVALID_ARG, "cgemm_tc: %d stages not built for precision %d", stages, precision);
    switch (precision) {
        case TC_BF16X3:
            if (alt) return mode == 0 ? launch<0, 3, 3, 0>(tmU, tmP, ep, s) : launch<0, 3, 3, 1>(tmU, tmP, ep, s);
            return mode == 0 ? launch<0, 3, 4, 0>(tmU, tmP, ep, s) : launch<0, 3, 4, 1>(tmU, tmP, ep, s);
        case TC_TF32:
            if (alt) return mode == 0 ? launch<1, 1, 4, 0>(tmU, tmP, ep, s) : launch<1, 1, 4, 1>(tmU, tmP, ep, s);
            return mode == 0 ? launch<1, 1, 8, 0>(tmU, tmP, ep, s) : launch<1, 1, 8, 1>(tmU, tmP, ep, s);
        case TC_TF32X3:
            if (alt) return mode == 0 ? launch<1, 2, 3, 0>(tmU, tmP, ep, s) : launch<1, 2, 3, 1>(tmU, tmP, ep, s);
            return mode == 0 ? launch<1, 2, 6, 0>(tmU, tmP, ep, s) : launch<1, 2, 6, 1>(tmU, tmP, ep, s);
        default:
            return fail(TC_ERR_INVALID_ARG, "cgemm_tc: precision %d has no tensor-core form", precision);
    }
}

int cgemm_parts(int precision) {
    return precision == TC_BF16X3 ? 3 : precision == TC_TF32X3 ? 2 : 1;
}

int cgemm_products(int precision) {
    return precision == TC_BF16X3 ? 6 : precision == TC_TF32X3 ? 3 : 1;
}

size_t cgemm_elem_bytes(int precision) { return precision == TC_BF16X3 ? 2 : 4; }

}  // namespace tc
