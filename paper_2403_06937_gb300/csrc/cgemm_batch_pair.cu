// cgemm_batch_pair.cu -- the batched tensor-core complex GEMM of the step on
// CTA pairs (the 2-SM MMA, cta_group::2): one persistent launch per product
// over the units of every system of a batch.
//
// A unit is one column tile J of one row pair (2p, 2p + 1) of one system
// (pair_unit, tile_order.cuh): the even CTA of a cluster takes row tile 2p,
// the odd one 2p + 1; for an odd tile count T the odd CTA of the last row
// pair has no rows (its U loads read the zeros past the end of the map, its
// tile is not written).  The unit list runs system by system in the caller's
// order (largest first), each system's units in groups of G row pairs,
// column by column; cluster q of C takes units q, q + C, q + 2C, ... (static
// round-robin: no waits between clusters).
//
// Each stage holds, in each CTA, its own S parts of U_r and U_i rows and one
// half of every B part (P_r parts in the even CTA, P_i parts in the odd one)
// for RB bytes of K per row; the even CTA arms its full barrier for both
// CTAs' bytes and the odd CTA's copies (cta_group::2) complete on it; the
// even CTA's MMA thread issues the part products as M = 256 pair MMAs into
// both CTAs' TMEM and commits each stage back to both CTAs.  Each CTA's
// copies land in its own shared memory only.  TMEM (two 128 x 256 FP32
// accumulators per CTA) holds one unit:
// after each unit both epilogues read their own tile and arrive on the even
// CTA's tmem_empty (count 2) before the next unit's MMAs start; the TMA ring
// runs on across units.  Each output element is accumulated in the order of
// the single-CTA kernels (K slice by K slice, the part products in one fixed
// order), so the results are bitwise those of cgemm_tc and cgemm_batch.
//
// Every wait is bounded: a timeout raises the abort flag of both CTAs, the
// copies in flight land (the even CTA waits for its armed stages, the odd
// one a fixed 1 ms), the MMA thread waits for its MMAs, and both CTAs meet at
// a cluster barrier before TMEM is freed.
#include "cgemm_batch.cuh"
#include "cgemm_dev.cuh"

namespace tc {
namespace {

using namespace sm100;
using namespace cg;

constexpr int kThreads = 192;

struct UnitRef {
    int b, I, J;
};

// unit u of the list -> (system, own row tile, column tile); `hint` is the
// system of the caller's previous unit
__device__ __forceinline__ UnitRef unit_at(const BatchSys* sys, int nsys, int mode, int u, int group,
                                           uint32_t rank, int& hint) {
    int b = hint;
    while (b + 1 < nsys && u >= sys[b + 1].unit_begin[mode]) b++;
    while (b > 0 && u < sys[b].unit_begin[mode]) b--;
    hint = b;
    UnitRef r;
    r.b = b;
    pair_unit(mode, sys[b].tiles, group, u - sys[b].unit_begin[mode], (int)rank, r.I, r.J);
    return r;
}

template <int RB>
__device__ __forceinline__ const CUtensorMap* map_of(const CUtensorMap& narrow, const CUtensorMap& wide) {
    return RB == 32 ? &narrow : &wide;
}

template <int KIND, int S, int RB, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    cgemm_batch_pair_kernel(const BatchSys* __restrict__ sys, int nsys, int nunits, int group, unsigned* status) {
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
    uint64_t* accum = empty + STAGES;       // MMA -> both epilogues, once per unit
    uint64_t* tmem_empty = accum + 1;       // both epilogues -> MMA (even CTA, count 2), once per unit
    uint64_t* drain = tmem_empty + 1;       // MMA issuer's own completion wait at teardown
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const int cluster = (int)(blockIdx.x >> 1), clusters = (int)(gridDim.x >> 1);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        mbar_init(tmem_empty, 2);
        mbar_init(drain, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc_pair(saddr(tmem_slot), 512);
        tmem_relinquish_pair();
    }
    __syncthreads();
    cluster_sync();   // both CTAs' barriers exist before either arrives on the other's
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t peer_abort = cluster_addr(saddr(const_cast<int*>(abort)), rank ^ 1u);

    if (warp == 4) {
        // ---------------------------------------------------------- producer (both CTAs)
        if (lane == 0) {
            const uint32_t lead_full = cluster_addr(saddr(&full[0]), 0u);
            uint32_t it = 0;   // stages issued so far
            int hint = 0;
            bool ok = true;
            for (int u = cluster; u < nunits && ok && !*abort; u += clusters) {
                const UnitRef r = unit_at(sys, nsys, MODE, u, group, rank, hint);
                const BatchSys& d = sys[r.b];
                const CUtensorMap* mu = map_of<RB>(d.tmU, d.tmU_w);
                const CUtensorMap* mp = MODE == 0 ? map_of<RB>(d.tmR, d.tmR_w) : map_of<RB>(d.tmX, d.tmX_w);
                const int KB = d.Np / kKPerStage;
                for (int kb = 0; kb < KB; kb++, it++) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1u;
                    if (!mbar_wait_bounded(&empty[s], ph ^ 1u, abort, kWaitLimitNs, 0)) {
                        ok = false;
                        break;
                    }
                    uint8_t* st = smem + s * kStage;
                    const int kx = kb * kKPerStage;
                    if (rank == 0) {
                        mbar_arrive_expect_tx(&full[s], 2 * kStage);   // both CTAs' bytes
                        const uint32_t fb = saddr(&full[s]);
#pragma unroll
                        for (int part = 0; part < 2; part++)
#pragma unroll
                            for (int a = 0; a < S; a++)
                                tma_load_3d(saddr(st + (part * S + a) * kTile), mu, fb, kx, r.I * 128, part * S + a);
#pragma unroll
                        for (int b = 0; b < S; b++)   // P_r part b
                            tma_load_3d(saddr(st + (2 * S + b) * kTile), mp, fb, kx, r.J * 128, b);
                    } else {
                        const uint32_t fb = lead_full + 8u * (uint32_t)s;
#pragma unroll
                        for (int part = 0; part < 2; part++)
#pragma unroll
                            for (int a = 0; a < S; a++)
                                tma_load_3d_pair(saddr(st + (part * S + a) * kTile), mu, fb, kx, r.I * 128,
                                                 part * S + a);
#pragma unroll
                        for (int b = 0; b < S; b++)   // P_i part b
                            tma_load_3d_pair(saddr(st + (2 * S + b) * kTile), mp, fb, kx, r.J * 128, S + b);
                    }
                }
            }
            const uint32_t from = it > (uint32_t)STAGES ? it - STAGES : 0u;
            if (!ok || *abort) {
                *abort = 1;
                st_cluster_u32(peer_abort, 1u);
                // the copies in flight land before the CTAs go away
                if (rank == 0) {
                    for (uint32_t k = from; k < it; k++)
                        (void)mbar_wait_bounded(&full[k % STAGES], (k / STAGES) & 1u, nullptr, 10000000ull, 0);
                } else {
                    spin_ns(1000000ull);
                }
            } else {
                // the last releases of this CTA's stages have arrived (no commit of the
                // pair's MMAs is still on its way to this CTA's barriers)
                for (uint32_t k = from; k < it; k++)
                    (void)mbar_wait_bounded(&empty[k % STAGES], (k / STAGES) & 1u, abort, kWaitLimitNs, 0);
            }
        }
    } else if (warp == 5) {
        if (lane == 0 && rank == 0) {
            // ------------------------------------------------------ MMA issuer (even CTA)
            const uint32_t peer_empty = cluster_addr(saddr(&empty[0]), 1u);
            const uint32_t peer_accum = cluster_addr(saddr(accum), 1u);
            uint32_t it = 0;
            int tl = 0, hint = 0;
            bool ok = true;
            for (int u = cluster; u < nunits && ok; u += clusters, tl++) {
                const UnitRef r = unit_at(sys, nsys, MODE, u, group, 0u, hint);
                const int KB = sys[r.b].Np / kKPerStage;
                if (tl > 0 && !mbar_wait_bounded_cluster(tmem_empty, (uint32_t)(tl - 1) & 1u, abort, kWaitLimitNs, 0))
                    break;
                tc_fence_after();
                for (int kb = 0; kb < KB; kb++, it++) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1u;
                    if (!mbar_wait_bounded_cluster(&full[s], ph, abort, kWaitLimitNs, 0)) {
                        ok = false;
                        break;
                    }
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
                if (!ok) break;
                umma_commit_pair(saddr(accum));
                umma_commit_pair(peer_accum);
            }
            // the pair MMAs (into both CTAs' TMEM) complete before either frees it
            umma_commit_pair(saddr(drain));
            (void)mbar_wait_bounded(drain, 0u, nullptr, kWaitLimitNs, 0);
            if (*abort) st_cluster_u32(peer_abort, 1u);
        }
    } else {
        // ---------------------------------------------------------- epilogue (both CTAs, own tile)
        const uint32_t lead_tmem_empty = cluster_addr(saddr(tmem_empty), 0u);
        int tl = 0, hint = 0;
        for (int u = cluster; u < nunits; u += clusters, tl++) {
            const UnitRef r = unit_at(sys, nsys, MODE, u, group, rank, hint);
            const BatchSys& d = sys[r.b];
            const bool ok = mbar_wait_bounded_cluster(accum, (uint32_t)tl & 1u, abort, kWaitLimitNs, 128);
            tc_fence_after();
            // the four epilogue warps leave together or not at all (barrier 1 below)
            uint32_t bad = (!ok || *abort) ? 1u : 0u, any;
            asm volatile(
                "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
                "bar.red.or.pred q, 1, 128, p;\n\tselp.u32 %0, 1, 0, q;\n}"
                : "=r"(any)
                : "r"(bad)
                : "memory");
            if (any) {
                if (threadIdx.x == 0) {
                    *abort = 1;
                    st_cluster_u32(peer_abort, 1u);
                }
                break;
            }
            // rows past an odd T, and the tile above the diagonal of the Hermitian product, are not written
            if (r.I < d.tiles && !(MODE == 1 && r.J > r.I)) {
                if (MODE == 0)
                    epilogue_tile<KIND, S, 0>(tmem, warp, lane, r.I, r.J, d.Np, d.Rr, d.Ri, d.Xparts, d.Xr, d.Xi);
                else
                    epilogue_tile<KIND, S, 1>(tmem, warp, lane, r.I, r.J, d.Np, d.Xr, d.Xi, d.Rparts, d.Rr, d.Ri);
            }
            tc_fence_before();
            asm volatile("bar.sync 1, 128;" ::: "memory");   // all four epilogue warps have read TMEM
            if (threadIdx.x == 0) {
                if (rank == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(tmem_empty)) : "memory");
                else
                    mbar_arrive_cluster(lead_tmem_empty);
            }
        }
        if (*abort && threadIdx.x == 0) atomicOr(status, kStatusTimeout);
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
tc_status launch(const BatchSys* sys, int nsys, int nunits, int group, unsigned* status, cudaStream_t s) {
    auto k = cgemm_batch_pair_kernel<KIND, S, RB, MODE>;
    constexpr int smem = split_pair_smem<S, RB>();
    static bool attr_set[64] = {};
    int dev = 0, sms = 0;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(TC_ERR_UNSUPPORTED_DEVICE, "device index out of range");
    TC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (!attr_set[dev]) {
        TC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr_set[dev] = true;
    }
    const int clusters = nunits < sms / 2 ? nunits : sms / 2;
    if (clusters <= 0) return TC_OK;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(2 * clusters);
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
    TC_CUDA(cudaLaunchKernelEx(&cfg, k, sys, nsys, nunits, group, status));
    TC_LAUNCH_CHECK();
    return TC_OK;
}

}  // namespace

tc_status cgemm_batch_pairs(int precision, int mode, int rb, const BatchSys* sys_dev, int nsys, int nunits,
                            int group, unsigned* status, cudaStream_t s) {
#define TC_BP(K, S_, RB_) \
    return mode == 0 ? launch<K, S_, RB_, 0>(sys_dev, nsys, nunits, group, status, s) \
                     : launch<K, S_, RB_, 1>(sys_dev, nsys, nunits, group, status, s)
    switch (precision) {
        case TC_BF16X3:
            if (rb == 64) TC_BP(0, 3, 64);
            if (rb == 32) TC_BP(0, 3, 32);
            break;
        case TC_TF32:
            if (rb == 128) TC_BP(1, 1, 128);
            if (rb == 64) TC_BP(1, 1, 64);
            if (rb == 32) TC_BP(1, 1, 32);
            break;
        case TC_TF32X3:
            if (rb == 128) TC_BP(1, 2, 128);
            if (rb == 64) TC_BP(1, 2, 64);
            if (rb == 32) TC_BP(1, 2, 32);
            break;
        default:
            return fail(TC_ERR_INVALID_ARG, "cgemm_batch: precision %d has no tensor-core form", precision);
    }
#undef TC_BP
    return fail(TC_ERR_INVALID_ARG, "cgemm_batch: %d-byte rows not built for precision %d", rb, precision);
}

}  // namespace tc
