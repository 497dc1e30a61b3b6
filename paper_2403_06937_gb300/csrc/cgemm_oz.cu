// cgemm_oz.cu -- FP64-accurate complex GEMM Y = U P^H on the BF16 tensor
// cores by exact integer slices (the Ozaki splitting), for the step
// rho <- U rho U^dag (Sec. III.A, Eqs. 6, 12) at FP64 accuracy.
//
// Slicing.  Every row r of an operand (both planes together) gets an
// exponent e_r with max |x| < 2^(e_r - 1); with S digits of b bits
// (oz_digits: b = 6, 7 or 8 as K allows, bS = 54 or 56), x 2^(bS - e_r) is
// rounded to an integer below 2^(bS - 1) and written in balanced base-2^b
// digits,
//     x = 2^e_r sum_{t=0..S-1} d_t 2^(-b(t+1)),   d_t integers, |d_t| <= 2^(b-1),
// each digit stored as an exact BF16 value (slice t).
//
// Products.  For slices t of U and u of P, sum_k d_t(U) d_u(P) is a sum of
// integers of size <= 2^(2b-2); over K <= 2^(26-2b) terms it stays within
// 2^24, so the FP32 accumulation of the tensor cores is exact (no rounding,
// hence no truncation).  One pass of the K loop per slice pair (t, u) with
// t + u <= S - 1 (S(S+1)/2 pairs; the first dropped level is below 2^-52 of
// the row and column scales) accumulates that pair in TMEM; the epilogue
// accumulates the exact integer results in int64 with the level weights as
// shifts and the last pass writes Y = sum 2^(e_i + f_j - b(t + u + 2))
// (integer) in FP64.  With 6-bit digits, K above 16384 is cut into chunks of
// 16384, one pass each.
//
// Tile and roles as the split-BF16 kernel (cgemm_tc.cu): one CTA per 128 x 128
// complex tile, A = slice t of U_r and U_i (M = 128), B = slice u of
// [P_r; P_i] (N = 256), two FP32 accumulators (512 TMEM columns); a stage is
// one K step of one pair (16 KB), 12 stages.  Warp 4 issues TMA, warp 5 the
// MMAs, warps 0-3 the epilogue; the MMA issuer starts a pass only after the
// epilogue has read the previous one out of TMEM.  Every wait is bounded.
//   mode 0: all tiles (X = U rho).
//   mode 1: block-lower tiles (rho' = U X^H); oz_mirror fills the upper half.
#include <cuda_bf16.h>

#include <atomic>
#include <cstdlib>

#include "cgemm_dev.cuh"
#include "cgemm_oz.cuh"
#include "cgemm_tc.cuh"

namespace tc {
namespace {

using namespace sm100;
using namespace cg;

constexpr int kThreads = 192;
constexpr int kStages = 12;
constexpr int kStage = 2 * kATile + kBTile;   // 16 KB
constexpr int kKPerStage = kRowBytes / 2;     // 16 BF16 values of K
constexpr int kZeroExp = -100000;             // exponent of an all-zero row

// pair q -> (t, u) with t + u <= S - 1, t-major: (0,0), (0,1), ..., (0,S-1),
// (1,0), ..., (S-1,0).  Consecutive passes of a tile reuse the U slice t,
// which the CTAs of a wave (a few row tiles) keep in L2 while the P slices
// stream.
__device__ __forceinline__ void oz_pair(int q, int S, int& t, int& u) {
    int tt = 0, base = 0;
    while (base + (S - tt) <= q) {
        base += S - tt;
        tt++;
    }
    t = tt;
    u = q - base;
}

__device__ __forceinline__ double pow2(int e) {
    if (e < -1022) return 0.0;
    if (e > 1023) e = 1023;
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// Epilogue of one pass (slice pair of level L = t + u).  The pass's sums are
// exact integers below 2^24; Y_r = U_r P_r^T + U_i P_i^T and
// Y_i = U_i P_r^T - U_r P_i^T are formed exactly in int32 and accumulated
// exactly in int64, with the level's weight as a shift: levels 0-3 into
// `hi` (shift b(3 - L), unit 2^(e_i + f_j - 5b), kept in the FP64 output
// planes until the last pass), levels 4..S-1 into `lo` (shift b(S - 1 - L),
// unit 2^(e_i + f_j - b(S + 1))).  Bounds (a level holds at most L + 1 pair
// sums of magnitude 2^25 per K chunk): b = 6, hi <= chunks 2^25 2^18 1.2 and
// lo <= chunks 5 2^25 2^24 1.1, within int64 for up to 2^8 K chunks; b = 7
// and 8 (one chunk), hi <= 2^25 2^24 1.1, lo <= 5 2^25 2^21 1.1.  The last
// pass (level S - 1) writes
//     Y = hi 2^(e_i + f_j - 5b) + lo 2^(e_i + f_j - b(S + 1))
// in FP64.  Integer work only, except that final combination.
__device__ __forceinline__ void oz_epilogue(uint32_t tmem, int warp, int lane, int I, int J, const OzEpi& ep, int L,
                                            bool first_hi, bool first_lo, bool last) {
    const int row = warp * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    const size_t Np = (size_t)ep.Np;
    const size_t gi = (size_t)I * 128 + row;
    const int b = ep.bits;
    const bool to_hi = L <= 3;
    const int shift = to_hi ? b * (3 - L) : b * (ep.slices - 1 - L);
    const int e_hi = 5 * b, e_lo = b * (ep.slices + 1);
    const bool first = to_hi ? first_hi : first_lo;
    const int ei = ep.eU[gi];
#pragma unroll 1
    for (int c = 0; c < 128; c += 16) {
        float d1r[16], d1i[16], d2r[16], d2i[16];
        tmem_ld16(tl + c, d1r);            // U_r P_r^T
        tmem_ld16(tl + 128 + c, d1i);      // U_r P_i^T
        tmem_ld16(tl + 256 + c, d2r);      // U_i P_r^T
        tmem_ld16(tl + 384 + c, d2i);      // U_i P_i^T
        const size_t o = gi * Np + (size_t)J * 128 + c;
        long long* ar = to_hi ? reinterpret_cast<long long*>(ep.yr) + o : ep.lo_r + o;
        long long* ai = to_hi ? reinterpret_cast<long long*>(ep.yi) + o : ep.lo_i + o;
        longlong2* vr2 = reinterpret_cast<longlong2*>(ar);
        longlong2* vi2 = reinterpret_cast<longlong2*>(ai);
        // The exact pass sums as int64 pairs, two columns per entry of x.
        auto sums = [&](int h, longlong2& xr, longlong2& xi) {
            const int q = 2 * h;
            xr.x = (long long)(__float2int_rn(d1r[q]) + __float2int_rn(d2i[q])) << shift;
            xr.y = (long long)(__float2int_rn(d1r[q + 1]) + __float2int_rn(d2i[q + 1])) << shift;
            xi.x = (long long)(__float2int_rn(d2r[q]) - __float2int_rn(d1i[q])) << shift;
            xi.y = (long long)(__float2int_rn(d2r[q + 1]) - __float2int_rn(d1i[q + 1])) << shift;
        };
        // Every load of a batch is issued before its first store (the planes
        // are separate buffers, which the compiler cannot see), so a chunk
        // waits for one memory round trip, not one per pair of columns.
        if (!last) {
            longlong2 pr[8], pi[8];
            if (!first) {
#pragma unroll
                for (int h = 0; h < 8; h++) {
                    pr[h] = vr2[h];
                    pi[h] = vi2[h];
                }
            }
            tmem_wait_ld();
#pragma unroll
            for (int h = 0; h < 8; h++) {
                longlong2 xr, xi;
                sums(h, xr, xi);
                if (!first) {
                    xr.x += pr[h].x;
                    xr.y += pr[h].y;
                    xi.x += pi[h].x;
                    xi.y += pi[h].y;
                }
                vr2[h] = xr;
                vi2[h] = xi;
            }
        } else {
            // the last pass is of level S - 1 (lo): combine with hi into FP64,
            // eight columns per batch
            tmem_wait_ld();
            const longlong2* hr2 = reinterpret_cast<const longlong2*>(ep.yr + o);
            const longlong2* hi2 = reinterpret_cast<const longlong2*>(ep.yi + o);
#pragma unroll
            for (int g = 0; g < 8; g += 4) {
                longlong2 pr[4], pi[4], hr[4], hi[4];
                int ej[8];
#pragma unroll
                for (int h = 0; h < 4; h++) {
                    pr[h] = first ? make_longlong2(0, 0) : vr2[g + h];
                    pi[h] = first ? make_longlong2(0, 0) : vi2[g + h];
                    hr[h] = hr2[g + h];
                    hi[h] = hi2[g + h];
                    ej[2 * h] = ep.eP[(size_t)J * 128 + c + 2 * (g + h)];
                    ej[2 * h + 1] = ep.eP[(size_t)J * 128 + c + 2 * (g + h) + 1];
                }
#pragma unroll
                for (int h = 0; h < 4; h++) {
                    longlong2 xr, xi;
                    sums(g + h, xr, xi);
                    const long long lr[2] = {xr.x + pr[h].x, xr.y + pr[h].y};
                    const long long li[2] = {xi.x + pi[h].x, xi.y + pi[h].y};
                    const long long hr_[2] = {hr[h].x, hr[h].y}, hii[2] = {hi[h].x, hi[h].y};
                    double yr[2], yi[2];
#pragma unroll
                    for (int w = 0; w < 2; w++) {
                        const double s_hi = pow2(ei + ej[2 * h + w] - e_hi), s_lo = pow2(ei + ej[2 * h + w] - e_lo);
                        yr[w] = (double)hr_[w] * s_hi + (double)lr[w] * s_lo;
                        yi[w] = (double)hii[w] * s_hi + (double)li[w] * s_lo;
                    }
                    reinterpret_cast<double2*>(ep.yr + o)[g + h] = make_double2(yr[0], yr[1]);
                    reinterpret_cast<double2*>(ep.yi + o)[g + h] = make_double2(yi[0], yi[1]);
                }
            }
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    cgemm_oz_kernel(const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmP, OzEpi ep) {
    constexpr uint32_t kIdesc = make_idesc(1u, 128u, 256u);   // BF16 x BF16 -> FP32, M 128, N 256

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStage);
    uint64_t* empty = full + kStages;
    uint64_t* accum = empty + kStages;      // MMA -> epilogue, once per pass
    uint64_t* tmem_empty = accum + 1;       // epilogue -> MMA, once per pass
    uint64_t* drain = tmem_empty + 1;       // MMA issuer's own completion wait at teardown
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t lim = ep.wait_ns ? ep.wait_ns : kWaitLimitNs;
    int I, J;
    tile_of(MODE, ep.tiles, ep.group, blockIdx.x, I, J);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
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
    if (warp == 4 && lane == 0) {
        prefetch_tmap(&tmU);
        prefetch_tmap(&tmP);
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int S = ep.slices;
    const int kmax = 1 << (26 - 2 * ep.bits);
    const int Kc = ep.Np < kmax ? ep.Np : kmax;
    const int chunks = ep.Np / Kc;
    const int KBc = Kc / kKPerStage;
    const int passes = S * (S + 1) / 2 * chunks;

    if (warp == 4) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            // U slices are kept in L2 across the consecutive passes that reuse them
            const uint64_t keep = l2_policy_evict_last();
            uint32_t it = 0;
            bool ok = true;
            for (int p = 0; p < passes && ok; p++) {
                int t, u;
                oz_pair(p / chunks, S, t, u);
                const int c = p % chunks;
                for (int kb = 0; kb < KBc; kb++, it++) {
                    const int s = it % kStages;
                    const uint32_t ph = (it / kStages) & 1u;
                    if (!mbar_wait_bounded(&empty[s], ph ^ 1u, abort, lim, 0)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[s], kStage);
                    uint8_t* st = smem + s * kStage;
                    const uint32_t fb = saddr(&full[s]);
                    const int kx = c * Kc + kb * kKPerStage;
                    tma_load_3d_hint(saddr(st), &tmU, fb, kx, I * 128, t, keep);                       // U_r
                    tma_load_3d_hint(saddr(st + kATile), &tmU, fb, kx, I * 128, S + t, keep);          // U_i
                    tma_load_3d(saddr(st + 2 * kATile), &tmP, fb, kx, J * 128, u);                     // P_r slice u
                    tma_load_3d(saddr(st + 2 * kATile + 128 * kRowBytes), &tmP, fb, kx, J * 128,
                                S + u);                                                                // P_i slice u
                }
            }
            if (*abort) {
                // let the copies already issued land before the CTA goes away
                for (uint32_t k = it > (uint32_t)kStages ? it - kStages : 0u; k < it; k++)
                    (void)mbar_wait_bounded(&full[k % kStages], (k / kStages) & 1u, nullptr, lim, 0);
            }
        }
    } else if (warp == 5) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int p = 0; p < passes && ok; p++) {
                if (p > 0 && !mbar_wait_bounded(tmem_empty, (uint32_t)(p - 1) & 1u, abort, lim, 0)) break;
                tc_fence_after();
                for (int kb = 0; kb < KBc; kb++, it++) {
                    const int s = it % kStages;
                    const uint32_t ph = (it / kStages) & 1u;
                    if (!mbar_wait_bounded(&full[s], ph, abort, lim, 0)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    uint8_t* st = smem + s * kStage;
                    const uint64_t bd = desc_kmajor_sw32(saddr(st + 2 * kATile));
                    umma<0>(tmem, desc_kmajor_sw32(saddr(st)), bd, kIdesc, kb > 0 ? 1u : 0u);
                    umma<0>(tmem + 256, desc_kmajor_sw32(saddr(st + kATile)), bd, kIdesc, kb > 0 ? 1u : 0u);
                    umma_commit(saddr(&empty[s]));
                }
                umma_commit(saddr(accum));
            }
            // own MMAs complete before the CTA frees TMEM
            umma_commit(saddr(drain));
            (void)mbar_wait_bounded(drain, 0u, nullptr, lim, 0);
        }
    } else {
        // ---------------------------------------------------------- epilogue
        for (int p = 0; p < passes; p++) {
            const bool ok = mbar_wait_bounded(accum, (uint32_t)p & 1u, abort, lim, 128);
            tc_fence_after();
            // the four epilogue warps leave together or not at all
            uint32_t bad = (!ok || *abort) ? 1u : 0u, any;
            asm volatile(
                "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
                "bar.red.or.pred q, 1, 128, p;\n\tselp.u32 %0, 1, 0, q;\n}"
                : "=r"(any)
                : "r"(bad)
                : "memory");
            if (any) {
                if (threadIdx.x == 0) *abort = 1;
                break;
            }
            int t, u;
            oz_pair(p / chunks, S, t, u);
            // first pass into hi: pair (0, 0); into lo: pair (0, 4); the last pass, pair (S - 1, 0), is into lo
            oz_epilogue(tmem, warp, lane, I, J, ep, t + u, p == 0, p == 4 * chunks, p == passes - 1);
            tc_fence_before();
            asm volatile("bar.sync 1, 128;" ::: "memory");   // all four epilogue warps have read TMEM
            if (threadIdx.x == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(tmem_empty)) : "memory");
        }
        if (*abort && threadIdx.x == 0) atomicOr(ep.status, kStatusTimeout);
    }

    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

constexpr int kSmem = kStages * kStage + 1024 /*align*/ + 256 /*barriers*/;

// ---------------------------------------------------------------------------
// CTA pairs on the 2-SM MMA (cta_group::2).  The two CTAs of a cluster take
// the row tiles I = 2p and 2p + 1 of one column tile J.  Each loads into its
// own shared memory the slice-t panels of its own U_r and U_i rows and one
// half of the B stack: P_r slice u in the even CTA, P_i slice u in the odd
// one (12 KB a stage; no operand is loaded twice, and each CTA's copies land
// in its own shared memory only).
// The even CTA's MMA thread issues M = 256 pair MMAs (its A rows and the odd
// CTA's, B from both halves) into both CTAs' TMEM, so each CTA's tensor core
// reads 8 KB of shared memory per MMA instead of 12.  Coordination:
//   full[s]        (even CTA) stage s of both CTAs landed: the even CTA arms
//                  it for both CTAs' bytes, the odd CTA's copies complete
//                  their bytes on it (cta_group::2 copies);
//   empty[s]       each CTA's stage s released: the MMA thread commits to the
//                  even CTA's barrier and, by its cluster address, the odd one's;
//   accum          (both) a pass's accumulators are complete (two commits);
//   tmem_empty     (even CTA, count 2) both epilogues have read a pass.
// Every wait is bounded; a timeout raises the abort flag of both CTAs, the
// copies in flight land (the even CTA waits for its armed stages, the odd
// one, whose copies complete on the even CTA's barriers, waits a fixed
// 1 ms), the MMA thread waits for its MMAs, and both meet at a cluster
// barrier before TMEM is freed and either CTA exits.
constexpr int kPairRing = 192 * 1024;    // bytes of the TMA ring per CTA
constexpr int kPairGroup = 6;            // row pairs per raster group (a wave: ~12 row x 12 column tiles)

// RB: bytes of K per operand row in a stage (32, 64 or 128, with the matching
// TMA swizzle).  A stage holds the CTA's U_r, U_i slice rows and its half of
// the B stack, 3 x 128 RB bytes, RB / 32 MMA K steps (two pair MMAs each);
// wider rows move each operand byte in fewer, larger TMA requests and give
// the barrier and issue overhead of a stage more MMAs.
template <int RB>
struct PairRing {
    static constexpr int kTile = 128 * RB;                  // one 128-row operand tile
    static constexpr int kStage = 3 * kTile;
    static constexpr int kStages = kPairRing / kStage;     // 16, 8 or 4
    static constexpr int kKPer = RB / 2;                    // BF16 K values per stage
    static constexpr int kSteps = RB / 32;                  // MMA K steps per stage
};

template <int MODE, int RB>
__global__ void __launch_bounds__(kThreads, 1)
    cgemm_oz_pair_kernel(const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmP, OzEpi ep) {
    constexpr uint32_t kIdesc = make_idesc(1u, 256u, 256u);   // BF16 x BF16 -> FP32, M 256 (128 per CTA), N 256
    using R = PairRing<RB>;
    constexpr int kPairStages = R::kStages;
    constexpr int kPairStage = R::kStage;

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kPairStages * kPairStage);
    uint64_t* empty = full + kPairStages;
    uint64_t* accum = empty + kPairStages;
    uint64_t* tmem_empty = accum + 1;
    uint64_t* drain = tmem_empty + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t lim = ep.wait_ns ? ep.wait_ns : kWaitLimitNs;
    const uint32_t rank = cluster_ctarank();
    int I, J;
    pair_unit(MODE, ep.tiles, kPairGroup, (int)(blockIdx.x >> 1), (int)rank, I, J);
    const bool own_rows = I < ep.tiles;   // false for the odd CTA of the last row pair of an odd T

    if (threadIdx.x == 0) {
        for (int s = 0; s < kPairStages; s++) {
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
    if (warp == 4 && lane == 0) {
        prefetch_tmap(&tmU);
        prefetch_tmap(&tmP);
    }
    __syncthreads();
    cluster_sync();   // both CTAs' barriers exist before either arrives on the other's
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t peer_abort = cluster_addr(saddr(const_cast<int*>(abort)), rank ^ 1u);
    const int S = ep.slices;
    const int kmax = 1 << (26 - 2 * ep.bits);
    const int Kc = ep.Np < kmax ? ep.Np : kmax;
    const int chunks = ep.Np / Kc;
    const int KBc = Kc / R::kKPer;
    const int passes = S * (S + 1) / 2 * chunks;

    if (warp == 4) {
        // ---------------------------------------------------------- producer (both CTAs)
        if (lane == 0) {
            const uint64_t keep = l2_policy_evict_last();
            const uint32_t lead_full = cluster_addr(saddr(&full[0]), 0u);
            uint32_t it = 0;
            bool ok = true;
            for (int p = 0; p < passes && ok; p++) {
                int t, u;
                oz_pair(p / chunks, S, t, u);
                const int c = p % chunks;
                for (int kb = 0; kb < KBc; kb++, it++) {
                    const int s = it % kPairStages;
                    const uint32_t ph = (it / kPairStages) & 1u;
                    if (!mbar_wait_bounded(&empty[s], ph ^ 1u, abort, lim, 0)) {
                        ok = false;
                        break;
                    }
                    uint8_t* st = smem + s * kPairStage;
                    const int kx = c * Kc + kb * R::kKPer;
                    if (rank == 0) {
                        mbar_arrive_expect_tx(&full[s], 2 * kPairStage);   // both CTAs' bytes
                        const uint32_t fb = saddr(&full[s]);
                        tma_load_3d_hint(saddr(st), &tmU, fb, kx, I * 128, t, keep);                  // U_r slice t
                        tma_load_3d_hint(saddr(st + R::kTile), &tmU, fb, kx, I * 128, S + t, keep);   // U_i slice t
                        tma_load_3d(saddr(st + 2 * R::kTile), &tmP, fb, kx, J * 128, u);              // P_r slice u
                    } else {
                        const uint32_t fb = lead_full + 8u * (uint32_t)s;
                        tma_load_3d_pair_hint(saddr(st), &tmU, fb, kx, I * 128, t, keep);
                        tma_load_3d_pair_hint(saddr(st + R::kTile), &tmU, fb, kx, I * 128, S + t, keep);
                        tma_load_3d_pair(saddr(st + 2 * R::kTile), &tmP, fb, kx, J * 128, S + u);     // P_i slice u
                    }
                }
            }
            const uint32_t from = it > (uint32_t)kPairStages ? it - kPairStages : 0u;
            if (!ok || *abort) {
                *abort = 1;
                st_cluster_u32(peer_abort, 1u);
                // the copies in flight land before the CTAs go away
                if (rank == 0) {
                    for (uint32_t k = from; k < it; k++)
                        (void)mbar_wait_bounded(&full[k % kPairStages], (k / kPairStages) & 1u, nullptr,
                                                10000000ull, 0);
                } else {
                    spin_ns(1000000ull);
                }
            } else {
                // the last releases of this CTA's stages have arrived (no commit of the
                // pair's MMAs is still on its way to this CTA's barriers)
                for (uint32_t k = from; k < it; k++)
                    (void)mbar_wait_bounded(&empty[k % kPairStages], (k / kPairStages) & 1u, abort, lim, 0);
            }
        }
    } else if (warp == 5) {
        if (lane == 0 && rank == 0) {
            // ------------------------------------------------------ MMA issuer (even CTA)
            const uint32_t peer_empty = cluster_addr(saddr(&empty[0]), 1u);
            const uint32_t peer_accum = cluster_addr(saddr(accum), 1u);
            uint32_t it = 0;
            bool ok = true;
            for (int p = 0; p < passes && ok; p++) {
                if (p > 0 && !mbar_wait_bounded_cluster(tmem_empty, (uint32_t)(p - 1) & 1u, abort, lim, 0)) break;
                tc_fence_after();
                for (int kb = 0; kb < KBc; kb++, it++) {
                    const int s = it % kPairStages;
                    const uint32_t ph = (it / kPairStages) & 1u;
                    if (!mbar_wait_bounded_cluster(&full[s], ph, abort, lim, 0)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    uint8_t* st = smem + s * kPairStage;
                    const uint64_t ar = desc_kmajor<RB>(saddr(st));
                    const uint64_t ai = desc_kmajor<RB>(saddr(st + R::kTile));
                    const uint64_t bd = desc_kmajor<RB>(saddr(st + 2 * R::kTile));
#pragma unroll
                    for (int ks = 0; ks < R::kSteps; ks++) {
                        const uint32_t acc = (kb > 0 || ks > 0) ? 1u : 0u;
                        const uint64_t off = 2u * (uint64_t)ks;   // 32 bytes of K further in each row
                        umma_pair(tmem, ar + off, bd + off, kIdesc, acc);
                        umma_pair(tmem + 256, ai + off, bd + off, kIdesc, acc);
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
            (void)mbar_wait_bounded(drain, 0u, nullptr, lim, 0);
            if (*abort) st_cluster_u32(peer_abort, 1u);
        }
    } else {
        // ---------------------------------------------------------- epilogue (both CTAs, own rows)
        const uint32_t lead_tmem_empty = cluster_addr(saddr(tmem_empty), 0u);
        for (int p = 0; p < passes; p++) {
            const bool ok = mbar_wait_bounded_cluster(accum, (uint32_t)p & 1u, abort, lim, 128);
            tc_fence_after();
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
            int t, u;
            oz_pair(p / chunks, S, t, u);
            if (own_rows)   // rows past an odd T: loads read zeros, nothing is written
                oz_epilogue(tmem, warp, lane, I, J, ep, t + u, p == 0, p == 4 * chunks, p == passes - 1);
            tc_fence_before();
            asm volatile("bar.sync 1, 128;" ::: "memory");   // all four epilogue warps have read TMEM
            if (threadIdx.x == 0) {
                if (rank == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(tmem_empty)) : "memory");
                else
                    mbar_arrive_cluster(lead_tmem_empty);
            }
        }
        if (*abort && threadIdx.x == 0) atomicOr(ep.status, kStatusTimeout);
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

constexpr int kPairSmem = kPairRing + 1024 /*align*/ + 512 /*barriers*/;

// One warp per row r < Np: the row exponent over both planes, then the S
// balanced base-2^b digits of every entry (zero beyond the valid N x N block).
// INTERLEAVED: re/im interleaved complex128 with row stride ld (complex
// elements); else planar FP64 planes re, im with row stride ld.
template <bool INTERLEAVED>
__global__ void oz_slice_kernel(const double* __restrict__ re, const double* __restrict__ im, int N, size_t ld,
                                int Np, double im_sign, int bits, int S, __nv_bfloat16* __restrict__ slices,
                                int* __restrict__ ex) {
    const int warps = (int)(gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    const size_t plane = (size_t)Np * Np;
    for (int r = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); r < Np; r += warps) {
        auto at = [&](int c, double& xr, double& xi) {
            if (r < N && c < N) {
                if (INTERLEAVED) {
                    xr = re[2 * ((size_t)r * ld + c)];
                    xi = re[2 * ((size_t)r * ld + c) + 1];
                } else {
                    xr = re[(size_t)r * ld + c];
                    xi = im[(size_t)r * ld + c];
                }
            } else {
                xr = 0.0;
                xi = 0.0;
            }
        };
        double m = 0.0;
        for (int c = lane; c < (r < N ? N : 0); c += 32) {
            double xr, xi;
            at(c, xr, xi);
            m = fmax(m, fmax(fabs(xr), fabs(xi)));
        }
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        const int e = m > 0.0 ? ilogb(m) + 2 : kZeroExp;   // max |x| < 2^(e - 1)
        if (lane == 0) ex[r] = e;
        // x 2^(bS - e) as two exact power-of-two factors (bS - e exceeds the
        // FP64 exponent range for rows below 2^-969)
        const int sh = bits * S - e;
        const long long half = 1ll << (bits - 1), mask = (1ll << bits) - 1;
        const double sc1 = m > 0.0 ? pow2(sh < 1000 ? sh : 1000) : 0.0;
        const double sc2 = m > 0.0 ? pow2(sh < 1000 ? 0 : sh - 1000) : 0.0;
        for (int c = lane; c < Np; c += 32) {
            double xv[2];
            at(c, xv[0], xv[1]);
            xv[1] *= im_sign;
#pragma unroll
            for (int part = 0; part < 2; part++) {
                long long v = __double2ll_rn(xv[part] * sc1 * sc2);   // |v| < 2^(bS - 1)
                __nv_bfloat16* dst = slices + (size_t)part * S * plane + (size_t)r * Np + c;
                for (int t = S - 1; t >= 1; t--) {
                    const long long d = ((v + half) & mask) - half;   // balanced digit in [-2^(b-1), 2^(b-1))
                    v = (v - d) >> bits;
                    dst[(size_t)t * plane] = __float2bfloat16_rn((float)d);
                }
                dst[0] = __float2bfloat16_rn((float)v);   // |v| <= 2^(b-1)
            }
        }
    }
}

// Upper triangle of a Hermitian result from its lower triangle; real diagonal.
__global__ void oz_mirror_kernel(double* __restrict__ yr, double* __restrict__ yi, int Np) {
    const size_t count = (size_t)Np * Np;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = e / Np, j = e % Np;
        if (i == j) {
            yi[e] = 0.0;
        } else if (i < j) {
            yr[e] = yr[j * Np + i];
            yi[e] = -yi[j * Np + i];
        }
    }
}

unsigned grid_for(size_t work) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t want = (work + 255) / 256;
    size_t cap = (size_t)sms * 16;
    return (unsigned)(want < cap ? (want ? want : 1) : cap);
}

template <int MODE>
tc_status launch(const CUtensorMap& tmU, const CUtensorMap& tmP, const OzEpi& ep, cudaStream_t s) {
    auto k = cgemm_oz_kernel<MODE>;
    static bool attr_set[64] = {};
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(TC_ERR_UNSUPPORTED_DEVICE, "device index out of range");
    if (!attr_set[dev]) {
        TC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
        attr_set[dev] = true;
    }
    const int T = ep.tiles;
    const unsigned grid = MODE == 0 ? (unsigned)(T * T) : (unsigned)(T * (T + 1) / 2);
    k<<<grid, kThreads, kSmem, s>>>(tmU, tmP, ep);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

// Pairs of CTAs (clusters of 2) on the 2-SM MMA: T even; mode 0 T * T / 2
// pairs, mode 1 sum over row pairs p of (2p + 2).
template <int MODE, int RB>
tc_status launch_pair(const CUtensorMap& tmU, const CUtensorMap& tmP, const OzEpi& ep, cudaStream_t s) {
    auto k = cgemm_oz_pair_kernel<MODE, RB>;
    static bool attr_set[64] = {};
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(TC_ERR_UNSUPPORTED_DEVICE, "device index out of range");
    if (!attr_set[dev]) {
        TC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kPairSmem));
        attr_set[dev] = true;
    }
    const unsigned pairs = (unsigned)pair_units(MODE, ep.tiles);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(2 * pairs);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kPairSmem;
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

// -1: not read yet; else TC_OZ_PAIRS from the environment (0: single CTAs at
// every size; anything else, or unset: CTA pairs from two tiles a side; an
// odd tile count leaves the odd CTA of the last row pair without rows).
// Both arrangements give the same bits.
std::atomic<int> g_oz_pairs{-1};

// -1: not chosen yet (TC_OZ_BITS=6 in the environment: 6-bit digits at every
// size; else the widest digits K allows)
std::atomic<int> g_oz_narrow{-1};

}  // namespace

bool oz_use_pairs(int tiles) {
    int v = g_oz_pairs.load();
    if (v < 0) {
        const char* e = std::getenv("TC_OZ_PAIRS");
        v = e && std::atoi(e) == 0 ? 0 : 1;
        g_oz_pairs.store(v);
    }
    return v != 0 && tiles >= 2;
}

OzDigits oz_digits(int Np) {
    int narrow = g_oz_narrow.load();
    if (narrow < 0) {
        const char* e = std::getenv("TC_OZ_BITS");
        narrow = e && std::atoi(e) == 6 ? 1 : 0;
        g_oz_narrow.store(narrow);
    }
    if (!narrow && Np <= 1024) return OzDigits{8, 7, 28, 1024};
    if (!narrow && Np <= 4096) return OzDigits{7, 8, 36, 4096};
    return OzDigits{6, 9, 45, 16384};
}

tc_status oz_slice(const double* re, const double* im, bool interleaved, bool conj, int N, size_t ld, int Np,
                   const OzDigits& dg, void* slices, int* ex, cudaStream_t s) {
    const unsigned blocks = (unsigned)(((size_t)Np * 32 + 255) / 256);
    const unsigned g = blocks < grid_for((size_t)Np * 32) ? blocks : grid_for((size_t)Np * 32);
    const double sign = conj ? -1.0 : 1.0;
    auto* out = static_cast<__nv_bfloat16*>(slices);
    if (interleaved)
        oz_slice_kernel<true><<<g, 256, 0, s>>>(re, im, N, ld, Np, sign, dg.bits, dg.slices, out, ex);
    else
        oz_slice_kernel<false><<<g, 256, 0, s>>>(re, im, N, ld, Np, sign, dg.bits, dg.slices, out, ex);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

tc_status oz_mirror(double* yr, double* yi, int Np, cudaStream_t s) {
    oz_mirror_kernel<<<grid_for((size_t)Np * Np), 256, 0, s>>>(yr, yi, Np);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

int oz_pair_rows() {
    static std::atomic<int> rows{0};
    int v = rows.load();
    if (v == 0) {
        const char* e = std::getenv("TC_OZ_ROWS");
        v = e ? std::atoi(e) : 128;
        if (v != 32 && v != 64 && v != 128) v = 128;
        rows.store(v);
    }
    return v;
}

tc_status cgemm_oz(int mode, const CUtensorMap& tmU, const CUtensorMap& tmP, const CUtensorMap& tmU_w,
                   const CUtensorMap& tmP_w, const OzEpi& ep, cudaStream_t s) {
    if (ep.Np < 128 || ep.Np % 128 != 0 || ep.tiles * 128 != ep.Np)
        return fail(TC_ERR_INVALID_ARG, "cgemm_oz: padded dimension must be a multiple of 128");
    const OzDigits dg = oz_digits(ep.Np);
    if (ep.bits != dg.bits || ep.slices != dg.slices)
        return fail(TC_ERR_INVALID_ARG, "cgemm_oz: digit width does not match the dimension");
    if (ep.Np > dg.kmax && ep.Np % dg.kmax != 0)
        return fail(TC_ERR_INVALID_ARG, "cgemm_oz: dimension above %d must be a multiple of it", dg.kmax);
    if (oz_use_pairs(ep.tiles)) {
        if (mode != 0 && mode != 1) return fail(TC_ERR_INVALID_ARG, "cgemm_oz: mode");
        switch (oz_pair_rows()) {
            case 32:
                return mode == 0 ? launch_pair<0, 32>(tmU_w, tmP_w, ep, s) : launch_pair<1, 32>(tmU_w, tmP_w, ep, s);
            case 64:
                return mode == 0 ? launch_pair<0, 64>(tmU_w, tmP_w, ep, s) : launch_pair<1, 64>(tmU_w, tmP_w, ep, s);
            default:
                return mode == 0 ? launch_pair<0, 128>(tmU_w, tmP_w, ep, s) : launch_pair<1, 128>(tmU_w, tmP_w, ep, s);
        }
    }
    if (mode == 0) return launch<0>(tmU, tmP, ep, s);
    if (mode == 1) return launch<1>(tmU, tmP, ep, s);
    return fail(TC_ERR_INVALID_ARG, "cgemm_oz: mode");
}

size_t oz_slice_bytes(int Np) {
    return round256((size_t)2 * oz_digits(Np).slices * Np * Np * sizeof(__nv_bfloat16));
}

size_t oz_mat_bytes(int Np) { return oz_slice_bytes(Np) + round256((size_t)Np * sizeof(int)); }

tc_status oz_mat_init(OzMat& m, Arena& ar, int Np) {
    m.Np = Np;
    m.dg = oz_digits(Np);
    m.slices = ar.take<uint8_t>(oz_slice_bytes(Np));
    m.ex = ar.take<int>((size_t)Np);
    if (!m.ex) return fail(TC_ERR_WORKSPACE, "FP64 emulation: workspace too small");
    TC_TRY(make_part_map_rows(&m.map_w, m.slices, Np, 2 * m.dg.slices, TC_BF16X3, oz_pair_rows()));
    return make_part_map(&m.map, m.slices, Np, 2 * m.dg.slices, TC_BF16X3);
}

tc_status oz_mat_view(OzMat& view, const OzMat& base, int Np) {
    if (Np > base.Np || oz_slice_bytes(Np) > oz_slice_bytes(base.Np))
        return fail(TC_ERR_INVALID_ARG, "FP64 emulation: operand view larger than its buffers");
    view = base;
    view.Np = Np;
    view.dg = oz_digits(Np);
    TC_TRY(make_part_map_rows(&view.map_w, base.slices, Np, 2 * view.dg.slices, TC_BF16X3, oz_pair_rows()));
    return make_part_map(&view.map, base.slices, Np, 2 * view.dg.slices, TC_BF16X3);
}

tc_status oz_mat_load(OzMat& m, const double* re, const double* im, bool interleaved, bool conj, int N, size_t ld,
                      cudaStream_t s) {
    return oz_slice(re, im, interleaved, conj, N, ld, m.Np, m.dg, m.slices, m.ex, s);
}

tc_status oz_product(int mode, const OzMat& A, const OzMat& B, const OzOut& out, int group, cudaStream_t s) {
    if (A.Np != B.Np || A.dg.bits != B.dg.bits)
        return fail(TC_ERR_INVALID_ARG, "FP64 emulation: operands of different sizes");
    OzEpi ep{};
    ep.Np = A.Np;
    ep.tiles = A.Np / 128;
    ep.group = group;
    ep.eU = A.ex;
    ep.eP = B.ex;
    ep.yr = out.yr;
    ep.yi = out.yi;
    ep.lo_r = out.lo_r;
    ep.lo_i = out.lo_i;
    ep.bits = A.dg.bits;
    ep.slices = A.dg.slices;
    ep.status = device_status_word();
    TC_TRY(cgemm_oz(mode, A.map, B.map, A.map_w, B.map_w, ep, s));
    if (mode == 1) TC_TRY(oz_mirror(out.yr, out.yi, A.Np, s));
    return TC_OK;
}

}  // namespace tc
