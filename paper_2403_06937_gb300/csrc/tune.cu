// tune.cu -- the autotuner of the step products.
//
// For one (n, precision) it times every built configuration of the kernels a
// step launches, on synthetic operands laid out exactly as tc_evolve lays
// them out in the caller's workspace, and keeps the fastest (tensor cores:
// the mean over windows of 8 back-to-back steps, at least 150 ms and at
// most 1.2 s, in two passes, so that the clock each configuration holds
// under the power cap counts):
//   FP64:         the DMMA GEMM tile (32 x 32 or 64 x 64 complex elements);
//   tensor cores: the tile shape (single CTAs on 128 x 128 tiles; CTA
//                 pairs on the 2-SM MMA, 256 x 128 per pair, with 32-byte
//                 or wide K rows a stage), the raster group G (the X = U rho
//                 launch takes G row tiles at a time, the Hermitian launch
//                 G x G super-blocks, so concurrent CTAs share operand panels
//                 in L2: 4, 8, 12, 16) and, for single CTAs, the depth of the
//                 TMA ring (two per precision).  tc_batch_evolve takes the
//                 shape and group chosen for its largest n.
// The choice lives in a process-wide table that tc_evolve, tc_expm and
// tc_evolve_backward consult, and is appended as one JSON object per line to
// the file named by TC_AUTOTUNE_CACHE (read back on the first lookup), keyed
// by the device architecture, n and the precision.  Every configuration
// computes every output element in the same order, so the choice changes
// speed, not results.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <cuda_bf16.h>

#include "cgemm_batch.cuh"
#include "cgemm_tc.cuh"
#include "lowp.cuh"
#include "paths.cuh"

namespace tc {
namespace {

struct Key {
    int arch, n, precision;
    bool operator<(const Key& o) const {
        if (arch != o.arch) return arch < o.arch;
        if (n != o.n) return n < o.n;
        return precision < o.precision;
    }
};
std::mutex g_mu;
std::map<Key, TuneChoice> g_table;
bool g_loaded = false;

// a batch by its composition: FNV-1a over the sorted n values (the order of
// the systems does not change the launches, which sort them)
struct BatchKey {
    int arch, precision;
    unsigned long long hash;
    bool operator<(const BatchKey& o) const {
        if (arch != o.arch) return arch < o.arch;
        if (precision != o.precision) return precision < o.precision;
        return hash < o.hash;
    }
};
std::map<BatchKey, TuneChoice> g_batch;

unsigned long long batch_hash(int count, const int* n) {
    std::vector<int> v(n, n + count);
    std::sort(v.begin(), v.end());
    unsigned long long h = 1469598103934665603ull;
    for (int x : v) {
        h ^= (unsigned long long)(unsigned)x;
        h *= 1099511628211ull;
    }
    return h;
}

int current_arch() {
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    return major * 10 + minor;
}

TuneChoice default_choice(int n, int precision) {
    TuneChoice c;
    c.f64_tile = gemm_f64_default_tile(1 << n);
    c.tc_group = 8;
    c.tc_stages = precision == TC_FP64 ? 0 : cgemm_default_stages(precision);
    c.tc_shape = kShapeAuto;
    return c;
}

void load_cache_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const char* path = std::getenv("TC_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char line[512];
    while (std::fgets(line, sizeof(line), f)) {
        int arch = 0, n = 0, prec = 0, tile = 0, group = 0, stages = 0;
        unsigned long long hash = 0;
        int shape = 0;
        if (std::sscanf(line, " {\"arch\": %d, \"batch\": \"%llx\", \"precision\": %d, \"tc_group\": %d, "
                              "\"tc_shape\": %d",
                        &arch, &hash, &prec, &group, &shape) == 5) {
            if (shape < kShapeAuto || shape > kShapePairWide) shape = kShapeAuto;
            g_batch[BatchKey{arch, prec, hash}] = TuneChoice{0, group, cgemm_default_stages(prec), shape};
            continue;
        }
        if (std::sscanf(line,
                        " {\"arch\": %d, \"n\": %d, \"precision\": %d, \"f64_tile\": %d, \"tc_group\": %d, "
                        "\"tc_stages\": %d",
                        &arch, &n, &prec, &tile, &group, &stages) == 6) {
            int shape = kShapeAuto;
            const char* sh = std::strstr(line, "\"tc_shape\":");
            if (sh) std::sscanf(sh, "\"tc_shape\": %d", &shape);
            if (shape < kShapeAuto || shape > kShapePairWide) shape = kShapeAuto;
            TuneChoice c{tile, group, stages, shape};
            g_table[Key{arch, n, prec}] = c;
        }
    }
    std::fclose(f);
}

void save_entry(int arch, int n, int prec, const TuneChoice& c, double ms) {
    const char* path = std::getenv("TC_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"arch\": %d, \"n\": %d, \"precision\": %d, \"f64_tile\": %d, \"tc_group\": %d, "
                 "\"tc_stages\": %d, \"tc_shape\": %d, \"ms\": %.6f}\n",
                 arch, n, prec, c.f64_tile, c.tc_group, c.tc_stages, c.tc_shape, ms);
    std::fclose(f);
}

void save_batch_entry(int arch, unsigned long long hash, int prec, const TuneChoice& c, double ms) {
    const char* path = std::getenv("TC_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "{\"arch\": %d, \"batch\": \"%016llx\", \"precision\": %d, \"tc_group\": %d, \"tc_shape\": %d, "
                    "\"ms\": %.6f}\n",
                 arch, hash, prec, c.tc_group, c.tc_shape, ms);
    std::fclose(f);
}

// counter-based pattern in [-0.005, 0.005): realistic magnitudes, no NaN/Inf
__device__ __forceinline__ float pattern(size_t i, uint32_t seed) {
    uint32_t h = (uint32_t)(i * 2654435761u) ^ seed;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    return ((float)(h & 0xFFFFu) / 65536.0f - 0.5f) * 0.01f;
}
__global__ void fill_f64(double* p, size_t n, uint32_t seed) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = (double)pattern(i, seed);
}
__global__ void fill_f32(float* p, size_t n, uint32_t seed) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = pattern(i, seed);
}
__global__ void fill_bf16(__nv_bfloat16* p, size_t n, uint32_t seed) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = __float2bfloat16_rn(pattern(i, seed));
}

// synthetic operands in the buffers of one system: V parts, rho parts and FP32 planes
tc_status fill_operands(const LowpBufs& b, cudaStream_t s) {
    const unsigned blocks = 152 * 8;
    const size_t planes = (size_t)2 * b.S * b.Np * b.Np;
    if (b.E == 2) {
        fill_bf16<<<blocks, 256, 0, s>>>(static_cast<__nv_bfloat16*>(b.Uparts), planes, 3u);
        fill_bf16<<<blocks, 256, 0, s>>>(static_cast<__nv_bfloat16*>(b.Rparts), planes, 5u);
    } else {
        fill_f32<<<blocks, 256, 0, s>>>(static_cast<float*>(b.Uparts), planes, 3u);
        fill_f32<<<blocks, 256, 0, s>>>(static_cast<float*>(b.Rparts), planes, 5u);
    }
    TC_LAUNCH_CHECK();
    fill_f32<<<blocks, 256, 0, s>>>(b.Rr, (size_t)b.Np * b.Np, 7u);
    fill_f32<<<blocks, 256, 0, s>>>(b.Ri, (size_t)b.Np * b.Np, 9u);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

template <typename F>
tc_status time_ms(cudaStream_t s, int reps, F launch, double* best) {
    cudaEvent_t a, b;
    TC_CUDA(cudaEventCreate(&a));
    TC_CUDA(cudaEventCreate(&b));
    tc_status st = launch();   // warm-up
    *best = 1e30;
    for (int r = 0; r < reps && st == TC_OK; r++) {
        cudaEventRecord(a, s);
        st = launch();
        cudaEventRecord(b, s);
        if (st != TC_OK) break;
        if (cudaEventSynchronize(b) != cudaSuccess) {
            st = fail(TC_ERR_CUDA, "autotune: event wait failed");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < *best) *best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

// Sustained timing: launches back to back over at least `window_ms` of device
// time, mean per launch.  Under the GPU's power cap a configuration's clock
// depends on the power it draws (its shared-memory and L2 bytes per FLOP
// above all), which a few launches from an idle GPU do not show.
template <typename F>
tc_status time_window(cudaStream_t s, double window_ms, F launch, double* mean) {
    double one = 0.0;
    TC_TRY(time_ms(s, 1, launch, &one));
    const int reps = one > 0.0 && one < window_ms ? (int)(window_ms / one) + 1 : 1;
    cudaEvent_t a, b;
    TC_CUDA(cudaEventCreate(&a));
    TC_CUDA(cudaEventCreate(&b));
    tc_status st = TC_OK;
    cudaEventRecord(a, s);
    for (int r = 0; r < reps && st == TC_OK; r++) st = launch();
    cudaEventRecord(b, s);
    if (st == TC_OK && cudaEventSynchronize(b) != cudaSuccess) st = fail(TC_ERR_CUDA, "autotune: event wait failed");
    float ms = 0.f;
    if (st == TC_OK) cudaEventElapsedTime(&ms, a, b);
    *mean = (double)ms / reps;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

// Scores of `count` configurations (the mean step time of each over two
// passes).  The window of a timing is 8 steps of the first configuration,
// within [150 ms, 1.2 s]: long enough that the clock settles to what the
// configuration draws under the power cap.  The GPU first runs the last
// configuration for a window; the second pass takes the configurations in
// reverse order, so a slow drift of the clock weighs on all of them alike.
template <typename F>
tc_status score_configs(cudaStream_t s, int count, F step, std::vector<double>& score) {
    double one = 0.0;
    TC_TRY(time_ms(s, 1, [&]() { return step(0); }, &one));
    double window = 8.0 * one;
    window = window < 150.0 ? 150.0 : window > 1200.0 ? 1200.0 : window;
    double ms = 0.0;
    TC_TRY(time_window(s, window, [&]() { return step(count - 1); }, &ms));
    score.assign(count, 0.0);
    for (int pass = 0; pass < 2; pass++)
        for (int i = 0; i < count; i++) {
            const int c = pass == 0 ? i : count - 1 - i;
            TC_TRY(time_window(s, window, [&]() { return step(c); }, &ms));
            score[c] += 0.5 * ms;
        }
    return TC_OK;
}

}  // namespace

TuneChoice tune_lookup(int n, int precision) {
    const int arch = current_arch();
    std::lock_guard<std::mutex> lk(g_mu);
    load_cache_locked();
    auto it = g_table.find(Key{arch, n, precision});
    if (it != g_table.end()) return it->second;
    return default_choice(n, precision);
}

bool tune_batch_lookup(int count, const int* n, int precision, TuneChoice* c) {
    const int arch = current_arch();
    std::lock_guard<std::mutex> lk(g_mu);
    load_cache_locked();
    auto it = g_batch.find(BatchKey{arch, precision, batch_hash(count, n)});
    if (it == g_batch.end()) return false;
    *c = it->second;
    return true;
}

int tuned_f64_tile(int N) {
    int n = 0;
    while ((1 << n) < N && n < 30) n++;
    return tune_lookup(n, TC_FP64).f64_tile;
}

}  // namespace tc

using namespace tc;

extern "C" {

TC_API tc_status tc_autotune_lookup(int n, int precision, int* choice) {
    if (n < 1 || n > kMaxAtoms || !choice) return fail(TC_ERR_INVALID_ARG, "tc_autotune_lookup: bad argument");
    if (precision < TC_FP64 || precision > TC_TF32X3) return fail(TC_ERR_INVALID_ARG, "unknown precision");
    const TuneChoice c = tune_lookup(n, precision);
    choice[0] = c.f64_tile;
    choice[1] = c.tc_group;
    choice[2] = c.tc_stages;
    choice[3] = c.tc_shape;
    return TC_OK;
}

TC_API tc_status tc_autotune_set(int n, int precision, const int* choice) {
    if (n < 1 || n > kMaxAtoms || !choice) return fail(TC_ERR_INVALID_ARG, "tc_autotune_set: bad argument");
    if (precision < TC_FP64 || precision > TC_TF32X3) return fail(TC_ERR_INVALID_ARG, "unknown precision");
    if (choice[0] != 32 && choice[0] != 64) return fail(TC_ERR_INVALID_ARG, "f64 tile must be 32 or 64");
    if (choice[1] < 1 || choice[1] > 128) return fail(TC_ERR_INVALID_ARG, "raster group must be 1..128");
    if (precision != TC_FP64 && choice[2] != cgemm_default_stages(precision) && choice[2] != cgemm_alt_stages(precision))
        return fail(TC_ERR_INVALID_ARG, "ring depth %d not built for precision %d", choice[2], precision);
    if (choice[3] < kShapeAuto || choice[3] > kShapePairWide)
        return fail(TC_ERR_INVALID_ARG, "tile shape %d: 0 (automatic), 1, 2 or 3", choice[3]);
    const int arch = current_arch();
    std::lock_guard<std::mutex> lk(g_mu);
    load_cache_locked();
    g_table[Key{arch, n, precision}] =
        TuneChoice{choice[0], choice[1], precision == TC_FP64 ? 0 : choice[2], precision == TC_FP64 ? 0 : choice[3]};
    return TC_OK;
}

TC_API tc_status tc_autotune(int n, int precision, void* work, size_t work_bytes, void* stream, int* choice) {
    if (n < 1 || n > kMaxAtoms) return fail(TC_ERR_INVALID_ARG, "n = %d outside 1..16", n);
    if (precision < TC_FP64 || precision > TC_TF32X3) return fail(TC_ERR_INVALID_ARG, "unknown precision");
    const size_t need = tc_workspace_size(n, precision, TC_OP_EVOLVE, 0, 0);
    if (!work) return fail(TC_ERR_WORKSPACE, "work is NULL (need %zu bytes)", need);
    if (reinterpret_cast<uintptr_t>(work) & 255u) return fail(TC_ERR_WORKSPACE, "work is not 256-byte aligned");
    if (work_bytes < need) return fail(TC_ERR_WORKSPACE, "work has %zu bytes, need %zu", work_bytes, need);
    TC_TRY(check_device());
    cudaStream_t s = as_stream(stream);
    const int N = 1 << n;
    const size_t NN = (size_t)N * N;
    const unsigned blocks = 152 * 8;
    Arena ar{static_cast<char*>(work), work_bytes, 0};
    TuneChoice best_c = default_choice(n, precision);
    double best_ms = 1e30;

    if (precision == TC_FP64) {
        double* pl[6];
        for (int k = 0; k < 6; k++) {
            pl[k] = ar.take<double>(NN);
            fill_f64<<<blocks, 256, 0, s>>>(pl[k], NN, 17u + k);
            TC_LAUNCH_CHECK();
        }
        // X = U rho over a K slice (FP64 at full K takes tens of seconds at n = 14)
        const int K = N < 1024 ? N : 1024;
        for (int tile : {32, 64}) {
            GemmF64 g{};
            g.M = g.N = N;
            g.K = K;
            g.Ar = pl[0]; g.Ai = pl[1]; g.lda = N;
            g.Br = pl[2]; g.Bi = pl[3]; g.ldb = N;
            g.Cr = pl[4]; g.Ci = pl[5]; g.ldc = N;
            g.alpha = 1.0;
            g.cplx = 1;
            g.tile = tile;
            double ms = 0.0;
            TC_TRY(time_ms(s, 2, [&]() { return gemm_f64(g, s); }, &ms));
            if (ms < best_ms) {
                best_ms = ms;
                best_c.f64_tile = tile;
            }
        }
    } else {
        LowpBufs b{};
        TC_TRY(lowp_carve(n, precision, ar, b));
        TC_TRY(fill_operands(b, s));
        CUtensorMap tmU, tmR, tmX;
        TC_TRY(make_part_map(&tmU, b.Uparts, b.Np, 2 * b.S, precision));
        TC_TRY(make_part_map(&tmR, b.Rparts, b.Np, 2 * b.S, precision));
        TC_TRY(make_part_map(&tmX, b.Xparts, b.Np, 2 * b.S, precision));
        CUtensorMap wU, wR, wX;   // the CTA-pair kernel's wider rows
        const int rows = cgemm_pair_rows(precision);
        TC_TRY(make_part_map_rows(&wU, b.Uparts, b.Np, 2 * b.S, precision, rows));
        TC_TRY(make_part_map_rows(&wR, b.Rparts, b.Np, 2 * b.S, precision, rows));
        TC_TRY(make_part_map_rows(&wX, b.Xparts, b.Np, 2 * b.S, precision, rows));
        CgemmEpi e{};   // X = rho^H + V rho^H
        e.Np = b.Np;
        e.tiles = b.Np / 128;
        e.pr = b.Rr;
        e.pi = b.Ri;
        e.parts = b.Xparts;
        e.yr = b.Xr;
        e.yi = b.Xi;
        e.status = device_status_word();
        CgemmEpi e2 = e;  // rho' = X^H + V X^H
        e2.pr = b.Xr;
        e2.pi = b.Xi;
        e2.parts = b.Rparts;
        e2.yr = b.Rr;
        e2.yi = b.Ri;
        // one whole step (both launches) per configuration: single CTAs with either ring depth, then the
        // CTA-pair shapes (their ring depth is fixed by the shared memory); the single-system pair kernel
        // needs an even tile count
        struct Cand {
            int shape, stages, group;
            double ms;
        };
        std::vector<Cand> cands;
        std::vector<std::pair<int, int>> shapes = {{kShapeSingle, cgemm_default_stages(precision)},
                                                   {kShapeSingle, cgemm_alt_stages(precision)}};
        if (cgemm_use_pairs(e.tiles, 0, 0, 0)) {
            shapes.push_back({kShapePair32, cgemm_default_stages(precision)});
            if (cgemm_pair_rows(precision) != 32) shapes.push_back({kShapePairWide, cgemm_default_stages(precision)});
        }
        for (const auto& sh : shapes)
            for (int group : {4, 8, 12, 16}) cands.push_back({sh.first, sh.second, group, 1e30});
        auto step = [&](const Cand& cd) {
            e.group = e2.group = cd.group;
            e.shape = e2.shape = cd.shape;
            tc_status st = cgemm_tc(precision, 0, tmU, tmR, e, s, cd.stages, &wU, &wR);
            return st == TC_OK ? cgemm_tc(precision, 1, tmU, tmX, e2, s, cd.stages, &wU, &wX) : st;
        };
        std::vector<double> score;
        TC_TRY(score_configs(s, (int)cands.size(), [&](int i) { return step(cands[i]); }, score));
        for (size_t i = 0; i < cands.size(); i++) cands[i].ms = score[i];
        for (const Cand& cd : cands)
            if (cd.ms < best_ms) {
                best_ms = cd.ms;
                best_c.tc_group = cd.group;
                best_c.tc_stages = cd.stages;
                best_c.tc_shape = cd.shape;
            }
    }
    TC_CUDA(cudaStreamSynchronize(s));
    const int arch = current_arch();
    {
        std::lock_guard<std::mutex> lk(g_mu);
        load_cache_locked();
        g_table[Key{arch, n, precision}] = best_c;
    }
    save_entry(arch, n, precision, best_c, best_ms);
    if (choice) {
        choice[0] = best_c.f64_tile;
        choice[1] = best_c.tc_group;
        choice[2] = best_c.tc_stages;
        choice[3] = best_c.tc_shape;
    }
    return TC_OK;
}

TC_API tc_status tc_batch_autotune_lookup(int count, const int* n, int precision, int* choice, int* found) {
    if (count < 1 || !n || !choice || !found) return fail(TC_ERR_INVALID_ARG, "tc_batch_autotune_lookup: bad argument");
    if (precision != TC_BF16X3 && precision != TC_TF32 && precision != TC_TF32X3)
        return fail(TC_ERR_INVALID_ARG, "batch tuning applies to the tensor-core forms (precision %d)", precision);
    TuneChoice c{};
    *found = tune_batch_lookup(count, n, precision, &c) ? 1 : 0;
    choice[0] = *found ? c.tc_group : 0;
    choice[1] = *found ? c.tc_shape : 0;
    return TC_OK;
}

TC_API tc_status tc_batch_autotune_set(int count, const int* n, int precision, const int* choice) {
    if (count < 1 || !n || !choice) return fail(TC_ERR_INVALID_ARG, "tc_batch_autotune_set: bad argument");
    if (precision != TC_BF16X3 && precision != TC_TF32 && precision != TC_TF32X3)
        return fail(TC_ERR_INVALID_ARG, "batch tuning applies to the tensor-core forms (precision %d)", precision);
    if (choice[0] < 1 || choice[0] > 128) return fail(TC_ERR_INVALID_ARG, "raster group must be 1..128");
    if (choice[1] < kShapeAuto || choice[1] > kShapePairWide)
        return fail(TC_ERR_INVALID_ARG, "tile shape %d: 0 (automatic), 1, 2 or 3", choice[1]);
    const int arch = current_arch();
    std::lock_guard<std::mutex> lk(g_mu);
    load_cache_locked();
    g_batch[BatchKey{arch, precision, batch_hash(count, n)}] =
        TuneChoice{0, choice[0], cgemm_default_stages(precision), choice[1]};
    return TC_OK;
}

TC_API tc_status tc_batch_autotune(int count, const int* n, int precision, void* work, size_t work_bytes,
                                   void* stream, int* choice) {
    if (count < 1 || !n) return fail(TC_ERR_INVALID_ARG, "count or n missing");
    if (precision != TC_BF16X3 && precision != TC_TF32 && precision != TC_TF32X3)
        return fail(TC_ERR_INVALID_ARG, "batch tuning applies to the tensor-core forms (precision %d)", precision);
    for (int b = 0; b < count; b++)
        if (n[b] < 1 || n[b] > kMaxAtoms) return fail(TC_ERR_INVALID_ARG, "system %d: n = %d outside 1..16", b, n[b]);
    const size_t need = batch_bytes(count, n, precision);
    if (!work) return fail(TC_ERR_WORKSPACE, "work is NULL (need %zu bytes)", need);
    if (reinterpret_cast<uintptr_t>(work) & 255u) return fail(TC_ERR_WORKSPACE, "work is not 256-byte aligned");
    if (work_bytes < need) return fail(TC_ERR_WORKSPACE, "work has %zu bytes, need %zu", work_bytes, need);
    TC_TRY(check_device());
    cudaStream_t s = as_stream(stream);
    // the batch's buffers as tc_batch_evolve carves them (systems in decreasing size), synthetic operands
    std::vector<int> order(n, n + count);
    std::sort(order.begin(), order.end(), [](int a, int b) { return a > b; });
    Arena ar{static_cast<char*>(work), work_bytes, 0};
    BatchSys* sys_dev = ar.take<BatchSys>((size_t)count);
    std::vector<BatchSys> host(count);
    BatchPlan plan = batch_plan(precision, order[0]);
    for (int k = 0; k < count; k++) {
        LowpBufs b{};
        TC_TRY(lowp_carve(order[k], precision, ar, b));
        TC_TRY(fill_operands(b, s));
        BatchSys& h = host[k];
        std::memset(&h, 0, sizeof(h));
        TC_TRY(batch_plan_add(plan, h, precision, b.Np, b.Uparts, b.Rparts, b.Xparts));
        h.Rr = b.Rr; h.Ri = b.Ri; h.Rparts = b.Rparts;
        h.Xr = b.Xr; h.Xi = b.Xi; h.Xparts = b.Xparts;
    }
    TC_CUDA(cudaMemcpyAsync(sys_dev, host.data(), sizeof(BatchSys) * count, cudaMemcpyHostToDevice, s));
    TC_CUDA(cudaStreamSynchronize(s));
    unsigned* status = device_status_word();
    // one batch step (both launches) per (shape, raster group), sustained windows, two passes
    struct Cand {
        int shape, group;
        double ms;
    };
    std::vector<Cand> cands;
    for (int shape : {kShapeSingle, kShapePair32, kShapePairWide})
        for (int group : {4, 8, 12, 16}) cands.push_back({shape, group, 1e30});
    auto step = [&](const Cand& cd) {
        BatchPlan p = plan;
        p.shape = cd.shape;
        p.group = cd.group;
        p.rb = cd.shape == kShapePairWide ? cgemm_pair_rows(precision) : 32;
        tc_status st = cgemm_batch(precision, 0, sys_dev, count, p, status, s);
        return st == TC_OK ? cgemm_batch(precision, 1, sys_dev, count, p, status, s) : st;
    };
    std::vector<double> score;
    TC_TRY(score_configs(s, (int)cands.size(), [&](int i) { return step(cands[i]); }, score));
    for (size_t i = 0; i < cands.size(); i++) cands[i].ms = score[i];
    TC_CUDA(cudaStreamSynchronize(s));
    TuneChoice best{0, 8, cgemm_default_stages(precision), kShapeAuto};
    double best_ms = 1e30;
    for (const Cand& cd : cands)
        if (cd.ms < best_ms) {
            best_ms = cd.ms;
            best.tc_group = cd.group;
            best.tc_shape = cd.shape;
        }
    const int arch = current_arch();
    const unsigned long long hash = batch_hash(count, n);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        load_cache_locked();
        g_batch[BatchKey{arch, precision, hash}] = best;
    }
    save_batch_entry(arch, hash, precision, best, best_ms);
    if (choice) {
        choice[0] = best.tc_group;
        choice[1] = best.tc_shape;
    }
    return TC_OK;
}

}  // extern "C"
