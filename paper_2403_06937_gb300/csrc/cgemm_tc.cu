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
#include <cstdlib>

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


// ---------------------------------------------------------------------------
// CTA pairs on the 2-SM MMA (cta_group::2).  The two CTAs of a cluster take
// the row tiles I = 2p and 2p + 1 of one column tile J.  Each loads into its
// own shared memory all S parts of its own U_r and U_i rows and one half of
// every B part (P_r parts in the even CTA, P_i parts in the odd one): a stage
// is 12 S KB instead of 16 S KB, and each CTA's tensor core reads 8 KB of
// shared memory per MMA instead of 12.  The even CTA arms its full barrier
// of each stage for both CTAs' bytes; the odd CTA's copies (cta_group::2
// copies) complete their bytes on it.  The even CTA's MMA thread issues
// M = 256 pair MMAs into both CTAs' TMEM; the MMA completions release the
// stages of both CTAs (commits to each CTA's barrier by address).  Each
// CTA's copies land in its own shared memory only.  Each CTA's epilogue
// writes its own tile exactly as the
// single-CTA kernel does; in the Hermitian launch the tile (2p, 2p + 1)
// above the diagonal is computed and not written (its lower partner writes
// both).  Every wait is bounded; a timeout raises the abort flag of both
// CTAs, the copies in flight land (the even CTA waits for its armed stages,
// the odd one a fixed 1 ms), the MMA thread waits for its MMAs, and both
// meet at a cluster barrier before TMEM is freed.
// RB: bytes of K per operand row in a stage (32, 64 or 128, with the matching
// TMA swizzle): a stage is 3 S tiles of 128 RB bytes and RB / 32 MMA K steps
// (split_pair_stages, cgemm_dev.cuh).

template <int KIND, int S, int RB, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    cgemm_tc_pair_kernel(const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmP,
                         CgemmEpi ep) {
    constexpr int STAGES = split_pair_stages<S, RB>();
    static_assert(STAGES >= 2, "ring too small for this row width");
    constexpr int kTile = 128 * RB;          // one 128-row operand tile
    constexpr int kStage = 3 * S * kTile;    // own U_r, U_i parts + own half of each B part
    constexpr int kElem = KIND == 0 ? 2 : 4;
    constexpr int kKPerStage = RB / kElem;
    constexpr int kSteps = RB / 32;          // MMA K steps per stage
    constexpr uint32_t kIdesc = make_idesc(KIND == 0 ? 1u : 2u, 256u, 256u);

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * kStage);
    uint64_t* empty = full + STAGES;
    uint64_t* accum = empty + STAGES;
    uint64_t* drain = accum + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t lim = ep.wait_ns ? ep.wait_ns : kWaitLimitNs;
    const uint32_t rank = cluster_ctarank();
    int I, J;
    pair_tile_rows_range(MODE, ep.tiles, ep.group > 1 ? ep.group / 2 : 1, ep.hi > 0 ? ep.lo : 0,
                         ep.hi > 0 ? ep.hi : ep.tiles, (int)(blockIdx.x >> 1), (int)rank, I, J);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        mbar_init(drain, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc_pair(saddr(tmem_slot), 512);
        tmem_relinquish_pair();
    }
    if (warp == 4 && lane == 0) {
        prefetch_tmap(&tmU);
        prefetch_tmap(&tmP);
    }
    __syncthreads();
    cluster_sync();   // both CTAs' barriers exist before either arrives on the other's
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t peer_abort = cluster_addr(saddr(const_cast<int*>(abort)), rank ^ 1u);
    const int KB = ep.Np / kKPerStage;

    if (warp == 4) {
        // ---------------------------------------------------------- producer (both CTAs)
        if (lane == 0) {
            const uint32_t lead_full = cluster_addr(saddr(&full[0]), 0u);
            int issued = 0;
            bool ok = true;
            for (int kb = 0; kb < KB; kb++) {
                const int s = kb % STAGES;
                const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
                if (!mbar_wait_bounded(&empty[s], ph ^ 1u, abort, lim, 0)) {
                    ok = false;
                    break;
                }
                issued = kb + 1;
                if (ep.withhold && kb == 0) continue;   // injected fault: stage 0 is never filled
                uint8_t* st = smem + s * kStage;
                const int kx = kb * kKPerStage;
                if (rank == 0) {
                    mbar_arrive_expect_tx(&full[s], 2 * kStage);   // both CTAs' bytes
                    const uint32_t fb = saddr(&full[s]);
#pragma unroll
                    for (int part = 0; part < 2; part++)
#pragma unroll
                        for (int a = 0; a < S; a++)
                            tma_load_3d(saddr(st + (part * S + a) * kTile), &tmU, fb, kx, I * 128, part * S + a);
#pragma unroll
                    for (int b = 0; b < S; b++)   // P_r part b
                        tma_load_3d(saddr(st + (2 * S + b) * kTile), &tmP, fb, kx, J * 128, b);
                } else {
                    const uint32_t fb = lead_full + 8u * (uint32_t)s;
#pragma unroll
                    for (int part = 0; part < 2; part++)
#pragma unroll
                        for (int a = 0; a < S; a++)
                            tma_load_3d_pair(saddr(st + (part * S + a) * kTile), &tmU, fb, kx, I * 128,
                                             part * S + a);
#pragma unroll
                    for (int b = 0; b < S; b++)   // P_i part b
                        tma_load_3d_pair(saddr(st + (2 * S + b) * kTile), &tmP, fb, kx, J * 128, S + b);
                }
            }
            const int from = issued - STAGES > 0 ? issued - STAGES : 0;
            if (!ok || *abort) {
                *abort = 1;
                st_cluster_u32(peer_abort, 1u);
                // the copies in flight land before the CTAs go away
                if (rank == 0) {
                    for (int kb = from; kb < issued; kb++)
                        if (!(ep.withhold && kb == 0))
                            (void)mbar_wait_bounded(&full[kb % STAGES], (uint32_t)(kb / STAGES) & 1u, nullptr,
                                                    10000000ull, 0);
                } else {
                    spin_ns(1000000ull);
                }
            } else {
                // the last releases of this CTA's stages have arrived
                for (int kb = from; kb < issued; kb++)
                    (void)mbar_wait_bounded(&empty[kb % STAGES], (uint32_t)(kb / STAGES) & 1u, abort, lim, 0);
            }
        }
    } else if (warp == 5) {
        if (lane == 0 && rank == 0) {
            // ------------------------------------------------------ MMA issuer (even CTA)
            const uint32_t peer_empty = cluster_addr(saddr(&empty[0]), 1u);
            for (int kb = 0; kb < KB; kb++) {
                const int s = kb % STAGES;
                const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
                if (!mbar_wait_bounded_cluster(&full[s], ph, abort, lim, 0)) break;
                tc_fence_after();
                uint8_t* st = smem + s * kStage;
#pragma unroll
                for (int ks = 0; ks < kSteps; ks++) {
                    const uint64_t off = 2u * (uint64_t)ks;   // 32 bytes of K further in each row
#pragma unroll
                    for (int p = 0; p < Pairs<S>::n; p++) {
                        const uint64_t bd = desc_kmajor<RB>(saddr(st + (2 * S + Pairs<S>::b(p)) * kTile)) + off;
#pragma unroll
                        for (int part = 0; part < 2; part++) {
                            const uint64_t ad =
                                desc_kmajor<RB>(saddr(st + (part * S + Pairs<S>::a(p)) * kTile)) + off;
                            umma_pair(tmem + part * 256, ad, bd, kIdesc, (kb > 0 || ks > 0 || p > 0) ? 1u : 0u);
                        }
                    }
                }
                umma_commit_pair(saddr(&empty[s]));
                umma_commit_pair(peer_empty + 8u * (uint32_t)s);
            }
            // always: complete when every pair MMA issued above has finished
            umma_commit_pair(saddr(accum));
            umma_commit_pair(cluster_addr(saddr(accum), 1u));
            umma_commit_pair(saddr(drain));
            (void)mbar_wait_bounded(drain, 0u, nullptr, lim, 0);
            if (*abort) st_cluster_u32(peer_abort, 1u);
        }
    } else {
        // ---------------------------------------------------------- epilogue (both CTAs, own tile)
        const bool ok = mbar_wait_bounded_cluster(accum, 0u, abort, lim, 128);
        tc_fence_after();
        if (ok && !*abort && !(MODE == 1 && J > I))
            cg::epilogue_tile<KIND, S, MODE>(tmem, warp, lane, I, J, ep.Np, ep.pr, ep.pi, ep.parts, ep.yr, ep.yi);
        if (!ok || *abort) {
            if (threadIdx.x == 0) {
                atomicOr(ep.status, kStatusTimeout);
                st_cluster_u32(peer_abort, 1u);
            }
        }
    }

    __syncwarp();
    tc_fence_before();
    __syncthreads();
    cluster_sync();   // neither CTA frees TMEM or leaves while the other may still use it
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, 512);
    }
}

template <int KIND, int S, int RB, int MODE>
tc_status launch_pair(const CUtensorMap& tmU, const CUtensorMap& tmP, const CgemmEpi& ep, cudaStream_t s) {
    auto k = cgemm_tc_pair_kernel<KIND, S, RB, MODE>;
    constexpr int smem = split_pair_smem<S, RB>();
    static bool attr_set[64] = {};
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(TC_ERR_UNSUPPORTED_DEVICE, "device index out of range");
    if (!attr_set[dev]) {
        TC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr_set[dev] = true;
    }
    const int lo = ep.hi > 0 ? ep.lo : 0, hi = ep.hi > 0 ? ep.hi : ep.tiles;
    const unsigned pairs = (unsigned)pair_count(MODE, ep.tiles, lo, hi);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(2 * pairs);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    TC_CUDA(cudaLaunchKernelEx(&cfg, k, tmU, tmP, ep));
    TC_LAUNCH_CHECK();
    return TC_OK;
}
}  // namespace

namespace {
std::atomic<int> g_inject_count{0};
std::atomic<unsigned long long> g_inject_wait{0};
// -1: not read yet; else TC_GEMM_PAIRS from the environment (0: kShapeAuto
// resolves to single CTAs; anything else, or unset: to CTA pairs)
std::atomic<int> g_pairs{-1};
}  // namespace

int cgemm_resolve_shape(int shape) {
    if (shape == kShapeSingle || shape == kShapePair32 || shape == kShapePairWide) return shape;
    int v = g_pairs.load();
    if (v < 0) {
        const char* e = std::getenv("TC_GEMM_PAIRS");
        v = e && std::atoi(e) == 0 ? 0 : 1;
        g_pairs.store(v);
    }
    return v == 0 ? kShapeSingle : kShapePairWide;
}

bool cgemm_use_pairs(int tiles, int mode, int lo, int hi) {
    if (tiles < 2 || tiles % 2 != 0) return false;
    // a Hermitian launch over a row band needs whole row pairs
    return !(mode == 1 && hi > 0 && (lo % 2 != 0 || hi % 2 != 0));
}

void cgemm_inject_timeout(int count, unsigned long long wait_ns) {
    g_inject_wait.store(wait_ns);
    g_inject_count.store(count);
}

int cgemm_default_stages(int precision) { return precision == TC_BF16X3 ? 4 : precision == TC_TF32X3 ? 6 : 8; }
int cgemm_alt_stages(int precision) { return precision == TC_BF16X3 ? 3 : precision == TC_TF32X3 ? 3 : 4; }

int cgemm_pair_rows(int precision) {
    static std::atomic<int> forced{-1};
    int f = forced.load();
    if (f < 0) {
        const char* e = std::getenv("TC_GEMM_ROWS");
        f = e ? std::atoi(e) : 0;
        if (f != 32 && f != 64 && f != 128) f = 0;
        forced.store(f);
    }
    const int dflt = precision == TC_TF32 ? 128 : 64;
    if (f == 128 && precision == TC_BF16X3) return 64;   // one 144 KB stage would not double-buffer
    return f ? f : dflt;
}

tc_status cgemm_tc(int precision, int mode, const CUtensorMap& tmU, const CUtensorMap& tmP, const CgemmEpi& ep_in,
                   cudaStream_t s, int stages, const CUtensorMap* tmU_w, const CUtensorMap* tmP_w) {
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
    if (ep.shape < kShapeAuto || ep.shape > kShapePairWide)
        return fail(TC_ERR_INVALID_ARG, "cgemm_tc: tile shape %d", ep.shape);
    const int shape = cgemm_resolve_shape(ep.shape);
    if (shape != kShapeSingle && cgemm_use_pairs(ep.tiles, mode, ep.lo, ep.hi)) {
        // CTA pairs: rows of cgemm_pair_rows() bytes when wide and the caller gave maps of that width,
        // else of 32 bytes
        const bool wide = shape == kShapePairWide && tmU_w && tmP_w && cgemm_pair_rows(precision) != 32;
        const CUtensorMap& u = wide ? *tmU_w : tmU;
        const CUtensorMap& p = wide ? *tmP_w : tmP;
        const int rb = wide ? cgemm_pair_rows(precision) : 32;
#define TC_PAIR(K, S_, RB_) \
    return mode == 0 ? launch_pair<K, S_, RB_, 0>(u, p, ep, s) : launch_pair<K, S_, RB_, 1>(u, p, ep, s)
        switch (precision) {
            case TC_BF16X3:
                if (rb == 64) TC_PAIR(0, 3, 64);
                TC_PAIR(0, 3, 32);
            case TC_TF32:
                if (rb == 128) TC_PAIR(1, 1, 128);
                if (rb == 64) TC_PAIR(1, 1, 64);
                TC_PAIR(1, 1, 32);
            case TC_TF32X3:
                if (rb == 128) TC_PAIR(1, 2, 128);
                if (rb == 64) TC_PAIR(1, 2, 64);
                TC_PAIR(1, 2, 32);
            default:
                return fail(TC_ERR_INVALID_ARG, "cgemm_tc: precision %d has no tensor-core form", precision);
        }
#undef TC_PAIR
    }
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
