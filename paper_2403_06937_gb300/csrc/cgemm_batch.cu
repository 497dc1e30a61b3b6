// cgemm_batch.cu -- the tensor-core complex GEMM of the step for a batch of
// independent systems of uneven size, in one persistent launch per product.
//
// Every system b contributes the tiles of its own product (T_b^2 tiles of
// X_b = U_b rho_b, or T_b (T_b + 1) / 2 block-lower tiles of rho_b'), with
// its own TMA descriptors (kept in global memory, in the caller's workspace)
// and its own dimension Np_b.  The tile list is ordered by decreasing K
// (systems sorted by size), and CTA c of a grid of G = #SMs takes tiles
// c, c + G, c + 2G, ... (static round-robin: no inter-CTA waits), so the
// longest tiles start first and the short ones fill the tail.
//
// One CTA keeps its TMEM (512 columns: the two 128 x 256 accumulators) and its
// barriers for all its tiles.  The TMA ring and the MMA issue run continuously
// across tile boundaries; the MMA issuer waits for the epilogue to release
// TMEM (tmem_empty) before it starts the next tile's accumulation.
//
// This file holds the single-CTA shape (128 x 128 tiles, 32-byte K rows) and
// the dispatch; the CTA-pair shapes are in cgemm_batch_pair.cu.  The shape
// and the raster group come from the autotuner's choice for the batch's
// largest n (batch_plan).
#include "cgemm_batch.cuh"
#include "cgemm_dev.cuh"
#include "cgemm_tc.cuh"
#include "kernels.cuh"

namespace tc {
namespace {

using namespace sm100;
using namespace cg;

constexpr int kThreads = 192;

struct TileRef {
    int b, I, J;
};

// tile t of the list -> (system, I, J); `hint` is the system of the caller's previous tile
__device__ __forceinline__ TileRef tile_at(const BatchSys* sys, int nsys, int mode, int t, int& hint) {
    int b = hint;
    while (b + 1 < nsys && t >= sys[b + 1].tile_begin[mode]) b++;
    while (b > 0 && t < sys[b].tile_begin[mode]) b--;
    hint = b;
    const int T = sys[b].tiles;
    const int local = t - sys[b].tile_begin[mode];
    TileRef r;
    r.b = b;
    if (mode == 0) {
        r.I = local / T;
        r.J = local % T;
    } else {
        int i = (int)((sqrt(8.0 * (double)local + 1.0) - 1.0) * 0.5);
        while ((i + 1) * (i + 2) / 2 <= local) ++i;
        while (i * (i + 1) / 2 > local) --i;
        r.I = i;
        r.J = local - i * (i + 1) / 2;
    }
    return r;
}

template <int KIND, int S, int STAGES, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    cgemm_batch_kernel(const BatchSys* __restrict__ sys, int nsys, int ntiles, unsigned* status) {
    constexpr int kStage = 2 * S * kATile + S * kBTile;
    constexpr int kElem = KIND == 0 ? 2 : 4;
    constexpr int kKPerStage = kRowBytes / kElem;
    constexpr uint32_t kIdesc = make_idesc(KIND == 0 ? 1u : 2u, 128u, 256u);

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * kStage);
    uint64_t* empty = full + STAGES;
    uint64_t* accum = empty + STAGES;       // MMA -> epilogue, once per tile
    uint64_t* tmem_empty = accum + 1;       // epilogue -> MMA, once per tile
    uint64_t* drain = tmem_empty + 1;       // MMA issuer's own completion wait at teardown
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        mbar_init(tmem_empty, 1);
        mbar_init(drain, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(saddr(tmem_slot), 512);
        tmem_relinquish();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 4) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            uint32_t it = 0;   // stages issued so far
            int hint = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
                const TileRef r = tile_at(sys, nsys, MODE, t, hint);
                const BatchSys& d = sys[r.b];
                const CUtensorMap* mu = &d.tmU;
                const CUtensorMap* mp = MODE == 0 ? &d.tmR : &d.tmX;
                const int KB = d.Np / kKPerStage;
                for (int kb = 0; kb < KB; kb++, it++) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1u;
                    if (!mbar_wait_bounded(&empty[s], ph ^ 1u, abort, kWaitLimitNs, 0)) break;
                    mbar_arrive_expect_tx(&full[s], kStage);
                    uint8_t* st = smem + s * kStage;
                    const uint32_t fb = saddr(&full[s]);
                    const int kx = kb * kKPerStage;
#pragma unroll
                    for (int part = 0; part < 2; part++)
#pragma unroll
                        for (int a = 0; a < S; a++)
                            tma_load_3d(saddr(st + (part * S + a) * kATile), mu, fb, kx, r.I * 128, part * S + a);
#pragma unroll
                    for (int b = 0; b < S; b++) {
                        uint8_t* bt = st + 2 * S * kATile + b * kBTile;
                        tma_load_3d(saddr(bt), mp, fb, kx, r.J * 128, b);
                        tma_load_3d(saddr(bt + 128 * kRowBytes), mp, fb, kx, r.J * 128, S + b);
                    }
                }
            }
            if (*abort) {
                for (uint32_t k = it > (uint32_t)STAGES ? it - STAGES : 0u; k < it; k++)
                    (void)mbar_wait_bounded(&full[k % STAGES], (k / STAGES) & 1u, nullptr, kWaitLimitNs, 0);
            }
        }
    } else if (warp == 5) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            uint32_t it = 0;
            int tl = 0, hint = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x, tl++) {
                const TileRef r = tile_at(sys, nsys, MODE, t, hint);
                const int KB = sys[r.b].Np / kKPerStage;
                if (tl > 0 && !mbar_wait_bounded(tmem_empty, (uint32_t)(tl - 1) & 1u, abort, kWaitLimitNs, 0))
                    break;
                tc_fence_after();
                bool ok = true;
                for (int kb = 0; kb < KB; kb++, it++) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1u;
                    if (!mbar_wait_bounded(&full[s], ph, abort, kWaitLimitNs, 0)) {
                        ok = false;
                        break;
                    }
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
                umma_commit(saddr(accum));
                if (!ok) break;
            }
            // own MMAs complete before the CTA frees TMEM
            umma_commit(saddr(drain));
            (void)mbar_wait_bounded(drain, 0u, nullptr, kWaitLimitNs, 0);
        }
    } else {
        // ---------------------------------------------------------- epilogue
        int tl = 0, hint = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, tl++) {
            const TileRef r = tile_at(sys, nsys, MODE, t, hint);
            const BatchSys& d = sys[r.b];
            const bool ok = mbar_wait_bounded(accum, (uint32_t)tl & 1u, abort, kWaitLimitNs, 128);
            tc_fence_after();
            // the four epilogue warps leave together or not at all (barrier 1 below)
            uint32_t bad = (!ok || *abort) ? 1u : 0u, any;
            asm volatile(
                "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
                "bar.red.or.pred q, 1, 128, p;\n\tselp.u32 %0, 1, 0, q;\n}"
                : "=r"(any)
                : "r"(bad)
                : "memory");
            if (any) break;
            if (MODE == 0)
                epilogue_tile<KIND, S, 0>(tmem, warp, lane, r.I, r.J, d.Np, d.Rr, d.Ri, d.Xparts, d.Xr, d.Xi);
            else
                epilogue_tile<KIND, S, 1>(tmem, warp, lane, r.I, r.J, d.Np, d.Xr, d.Xi, d.Rparts, d.Rr, d.Ri);
            tc_fence_before();
            asm volatile("bar.sync 1, 128;" ::: "memory");   // all four epilogue warps have read TMEM
            if (threadIdx.x == 0) {
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(tmem_empty)) : "memory");
            }
        }
        if (*abort && threadIdx.x == 0) atomicOr(status, kStatusTimeout);
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
    return STAGES * (2 * S * kATile + S * kBTile) + 1024 + 256;
}

template <int KIND, int S, int STAGES, int MODE>
tc_status launch(const BatchSys* sys, int nsys, int ntiles, unsigned* status, cudaStream_t s) {
    auto k = cgemm_batch_kernel<KIND, S, STAGES, MODE>;
    constexpr int smem = smem_bytes<KIND, S, STAGES>();
    static bool attr_set[64] = {};
    int dev = 0, sms = 0;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(TC_ERR_UNSUPPORTED_DEVICE, "device index out of range");
    TC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (!attr_set[dev]) {
        TC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr_set[dev] = true;
    }
    const int grid = ntiles < sms ? ntiles : sms;
    if (grid <= 0) return TC_OK;
    k<<<grid, kThreads, smem, s>>>(sys, nsys, ntiles, status);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

}  // namespace

BatchPlan batch_plan(int precision, int n) {
    const TuneChoice c = tune_lookup(n, precision);
    BatchPlan p{};
    p.shape = cgemm_resolve_shape(c.tc_shape);
    p.group = c.tc_group;
    p.rb = p.shape == kShapePairWide ? cgemm_pair_rows(precision) : 32;
    return p;
}

tc_status batch_plan_add(BatchPlan& plan, BatchSys& h, int precision, int Np, const void* Uparts,
                         const void* Rparts, const void* Xparts) {
    if (Np < 128 || Np % 128 != 0) return fail(TC_ERR_INVALID_ARG, "batch: padded dimension %d", Np);
    const int planes = 2 * cgemm_parts(precision);
    TC_TRY(make_part_map(&h.tmU, Uparts, Np, planes, precision));
    TC_TRY(make_part_map(&h.tmR, Rparts, Np, planes, precision));
    TC_TRY(make_part_map(&h.tmX, Xparts, Np, planes, precision));
    const int rb = plan.rb == 32 ? cgemm_pair_rows(precision) : plan.rb;   // maps unused at 32 bytes
    TC_TRY(make_part_map_rows(&h.tmU_w, Uparts, Np, planes, precision, rb));
    TC_TRY(make_part_map_rows(&h.tmR_w, Rparts, Np, planes, precision, rb));
    TC_TRY(make_part_map_rows(&h.tmX_w, Xparts, Np, planes, precision, rb));
    h.Np = Np;
    h.tiles = Np / 128;
    for (int mode = 0; mode < 2; mode++) {
        h.tile_begin[mode] = plan.tiles[mode];
        h.unit_begin[mode] = plan.units[mode];
    }
    plan.tiles[0] += h.tiles * h.tiles;
    plan.tiles[1] += h.tiles * (h.tiles + 1) / 2;
    plan.units[0] += (int)pair_units(0, h.tiles);
    plan.units[1] += (int)pair_units(1, h.tiles);
    return TC_OK;
}

tc_status cgemm_batch(int precision, int mode, const BatchSys* sys_dev, int nsys, const BatchPlan& plan,
                      unsigned* status, cudaStream_t s) {
    if (mode != 0 && mode != 1) return fail(TC_ERR_INVALID_ARG, "cgemm_batch: mode");
    if (plan.shape == kShapePair32 || plan.shape == kShapePairWide) {
        const int G = plan.group > 1 ? plan.group / 2 : 1;
        return cgemm_batch_pairs(precision, mode, plan.rb, sys_dev, nsys, plan.units[mode], G, status, s);
    }
    const int ntiles = plan.tiles[mode];
    switch (precision) {
        case TC_BF16X3:
            return mode == 0 ? launch<0, 3, 4, 0>(sys_dev, nsys, ntiles, status, s)
                             : launch<0, 3, 4, 1>(sys_dev, nsys, ntiles, status, s);
        case TC_TF32:
            return mode == 0 ? launch<1, 1, 8, 0>(sys_dev, nsys, ntiles, status, s)
                             : launch<1, 1, 8, 1>(sys_dev, nsys, ntiles, status, s);
        case TC_TF32X3:
            return mode == 0 ? launch<1, 2, 6, 0>(sys_dev, nsys, ntiles, status, s)
                             : launch<1, 2, 6, 1>(sys_dev, nsys, ntiles, status, s);
        default:
            return fail(TC_ERR_INVALID_ARG, "cgemm_batch: precision %d has no tensor-core form", precision);
    }
}

}  // namespace tc
