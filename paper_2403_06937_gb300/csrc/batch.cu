// batch.cu -- many independent systems of uneven size stepped together
// (tc_batch_evolve).  The tensor-core forms run each product of a step as one
// persistent launch over the tiles of every system (cgemm_batch.cu; single
// CTAs or CTA pairs, the autotuner's tile shape); the FP64 form runs the
// systems' DMMA products one after another, the FP64-emulated form each
// system's step loop on one of eight concurrent lanes.  The whole step loop
// is captured into one CUDA graph on a library stream and launched once.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "cgemm_batch.cuh"
#include "cgemm_oz.cuh"
#include "graph.cuh"
#include "cgemm_tc.cuh"
#include "lowp.cuh"
#include "paths.cuh"
#include "timing.cuh"

namespace tc {
namespace {

size_t f64_system_bytes(int n) {
    const size_t cm = 2 * round256(sizeof(double) << (2 * n));
    return 3 * cm + observables_scratch_bytes(n) + 256;   // U, rho, X planar
}

// one split-K scratch shared by the systems' products (they run one after another)
size_t f64_shared_bytes(const int* n, int count) {
    for (int b = 0; b < count; b++)
        if ((1 << n[b]) <= kSplitMaxDim) return gemm_f64_splitk_bytes();
    return 0;
}

struct F64Sys {
    int n, N;
    double *Ur, *Ui, *Rr, *Ri, *Xr, *Xi, *scratch;
};

// Streams on which the systems of an FP64-emulated batch run side by side
// (one pool per device, created on first use), with a fork event and one join
// event per lane.
constexpr int kOzLanes = 8;
struct OzLanes {
    cudaStream_t s[kOzLanes] = {};
    cudaEvent_t join[kOzLanes] = {};
    cudaEvent_t fork = nullptr;
};
std::mutex g_lanes_mu;
OzLanes g_lanes[64];

tc_status oz_lanes(OzLanes** out) {
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(TC_ERR_UNSUPPORTED_DEVICE, "device index out of range");
    std::lock_guard<std::mutex> lk(g_lanes_mu);
    OzLanes& l = g_lanes[dev];
    if (!l.fork) {
        for (int i = 0; i < kOzLanes; i++) {
            TC_CUDA(cudaStreamCreateWithFlags(&l.s[i], cudaStreamNonBlocking));
            TC_CUDA(cudaEventCreateWithFlags(&l.join[i], cudaEventDisableTiming));
        }
        TC_CUDA(cudaEventCreateWithFlags(&l.fork, cudaEventDisableTiming));
    }
    *out = &l;
    return TC_OK;
}

// FP64 emulated on the BF16 tensor cores: every system with its own buffers;
// the step loops run on up to kOzLanes concurrent lanes (systems assigned
// largest first to the lane with the least work, N^3 each), captured into
// one graph (fork from the capture stream, join back before its end), so
// the small systems' launches fill the SMs the large products leave idle.
// Each system's launches keep their order, so its results are bitwise those
// of tc_evolve on it alone.
tc_status batch_oz(int count, const int* n, const void* const* U, void* const* rho, int steps, int renorm_every,
                   const Model* models, double* const* obs, void* work, size_t work_bytes, cudaStream_t us) {
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
    Arena ar{static_cast<char*>(work), work_bytes, 0};
    std::vector<OzSystem> z(count);
    for (int b : order) TC_TRY(z[b].carve(n[b], ar));
    const int L = count < kOzLanes ? count : kOzLanes;
    std::vector<std::vector<int>> lane(L);
    std::vector<double> load(L, 0.0);
    for (int b : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lane[l].push_back(b);
        load[l] += std::pow(2.0, 3.0 * n[b]);
    }
    OzLanes* ls = nullptr;
    TC_TRY(oz_lanes(&ls));
    auto first = [&](cudaStream_t cs) -> tc_status {
        for (int b : order)
            TC_TRY(z[b].first(static_cast<const double*>(U[b]), static_cast<const double*>(rho[b]),
                              models ? &models[b] : nullptr, obs ? obs[b] : nullptr, renorm_every, cs));
        return TC_OK;
    };
    auto rest = [&](cudaStream_t cs) -> tc_status {
        TC_CUDA(cudaEventRecord(ls->fork, cs));
        for (int l = 0; l < L; l++) TC_CUDA(cudaStreamWaitEvent(ls->s[l], ls->fork, 0));
        tc_status st = TC_OK;
        for (int l = 0; l < L && st == TC_OK; l++)
            for (int b : lane[l])
                for (int k = 1; k <= steps && st == TC_OK; k++) st = z[b].step(k, ls->s[l]);
        // every lane joins back, also after a failure (a capture ends only with its streams joined)
        for (int l = 0; l < L; l++) {
            cudaEventRecord(ls->join[l], ls->s[l]);
            cudaStreamWaitEvent(cs, ls->join[l], 0);
        }
        return st;
    };
    auto tail = [&](cudaStream_t cs) -> tc_status {
        for (int b : order) TC_TRY(z[b].tail(static_cast<double*>(rho[b]), cs));
        return TC_OK;
    };
    return run_captured(us, first, rest, tail, steps >= 1 && !timing_enabled());
}

}  // namespace

size_t batch_bytes(int count, const int* n, int precision) {
    if (precision == TC_FP64_OZAKI) {
        // each system has its own buffers (the systems run side by side)
        size_t total = 256;
        for (int b = 0; b < count; b++) {
            if (n[b] < 1 || n[b] > kMaxAtoms) return 0;
            total += evolve_oz_bytes(n[b]);
        }
        return total;
    }
    size_t total = 256 + round256(sizeof(BatchSys) * (size_t)count) + 64;
    for (int b = 0; b < count; b++) {
        if (n[b] < 1 || n[b] > kMaxAtoms) return 0;
        total += precision == TC_FP64 ? f64_system_bytes(n[b]) : lowp_system_bytes(n[b], precision) + 512;
    }
    if (precision == TC_FP64) total += f64_shared_bytes(n, count);
    return total;
}

}  // namespace tc

using namespace tc;

extern "C" {

TC_API size_t tc_batch_workspace_size(int count, const int* n, int precision) {
    if (count < 1 || !n) return 0;
    if (precision < TC_FP64 || precision > TC_FP64_OZAKI) return 0;
    return batch_bytes(count, n, precision);
}

TC_API tc_status tc_batch_evolve(int count, const int* n, const void* const* U, void* const* rho, int steps,
                                 int precision, int renorm_every, const tc_params* params, double* const* obs,
                                 void* work, size_t work_bytes, void* stream) {
    if (count < 1 || !n || !U || !rho) return fail(TC_ERR_INVALID_ARG, "count, n, U or rho missing");
    if (steps < 0 || renorm_every < 0) return fail(TC_ERR_INVALID_ARG, "steps / renorm_every < 0");
    if (precision < TC_FP64 || precision > TC_FP64_OZAKI)
        return fail(TC_ERR_INVALID_ARG, "unknown precision %d", precision);
    std::vector<Model> models(count);
    for (int b = 0; b < count; b++) {
        if (n[b] < 1 || n[b] > kMaxAtoms) return fail(TC_ERR_INVALID_ARG, "system %d: n = %d outside 1..16", b, n[b]);
        if (!U[b] || !rho[b]) return fail(TC_ERR_INVALID_ARG, "system %d: U or rho is NULL", b);
        if ((reinterpret_cast<uintptr_t>(U[b]) | reinterpret_cast<uintptr_t>(rho[b])) & 15u)
            return fail(TC_ERR_INVALID_ARG, "system %d: U and rho must be 16-byte aligned", b);
        if (params) {
            TC_TRY(make_model(&params[b], &models[b]));
            if (models[b].n != n[b]) return fail(TC_ERR_INVALID_ARG, "system %d: params.n != n", b);
        }
    }
    const size_t need = batch_bytes(count, n, precision);
    if (!work) return fail(TC_ERR_WORKSPACE, "work is NULL (need %zu bytes)", need);
    if (reinterpret_cast<uintptr_t>(work) & 255u) return fail(TC_ERR_WORKSPACE, "work is not 256-byte aligned");
    if (work_bytes < need) return fail(TC_ERR_WORKSPACE, "work has %zu bytes, need %zu", work_bytes, need);
    TC_TRY(check_device());
    cudaStream_t us = as_stream(stream);
    if (precision == TC_FP64_OZAKI) return batch_oz(count, n, U, rho, steps, renorm_every, params ? models.data() : nullptr,
                                                    obs, work, work_bytes, us);

    // systems in decreasing size: the longest tiles first in the persistent schedule
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });

    Arena ar{static_cast<char*>(work), work_bytes, 0};
    BatchSys* sys_dev = ar.take<BatchSys>((size_t)count);
    cudaStream_t s = us;   // rebound to the capture stream inside run_captured

    std::vector<LowpBufs> lb(count);
    std::vector<F64Sys> fb(count);
    double* f64_partial = nullptr;   // split-K scratch shared by the FP64 products
    std::vector<BatchSys> host(count);
    // tile shape and raster group: tc_batch_autotune's choice for a batch of this composition, else the
    // autotuner's choice for the largest system (most of the work)
    BatchPlan plan = batch_plan(precision, n[order[0]]);
    TuneChoice tuned{};
    if (precision != TC_FP64 && tune_batch_lookup(count, n, precision, &tuned)) {
        plan.shape = cgemm_resolve_shape(tuned.tc_shape);
        plan.group = tuned.tc_group;
        plan.rb = plan.shape == kShapePairWide ? cgemm_pair_rows(precision) : 32;
    }
    auto observe = [&](int k, int row) -> tc_status {
        const int b = order[k];
        if (!obs || !obs[b]) return TC_OK;
        const int stride = TC_OBS_STRIDE(n[b]);
        const Model* mp = params ? &models[b] : nullptr;
        if (precision == TC_FP64)
            return launch_observables(kRhoPlanarF64, fb[k].Rr, fb[k].Ri, mp, n[b], obs[b] + (size_t)row * stride,
                                      fb[k].scratch, s);
        return launch_observables(kRhoPlanarF32, lb[k].Rr, lb[k].Ri, mp, n[b], obs[b] + (size_t)row * stride,
                                  lb[k].scratch, s, (size_t)lb[k].Np);
    };
    // one step of every system, enqueued on s
    unsigned* status = device_status_word();
    auto one_step = [&](int step) -> tc_status {
        if (precision == TC_FP64) {
            for (int k = 0; k < count; k++) {
                F64Sys& f = fb[k];
                GemmF64 g1{};
                g1.M = g1.N = g1.K = f.N;
                g1.Ar = f.Ur; g1.Ai = f.Ui; g1.lda = f.N;
                g1.Br = f.Rr; g1.Bi = f.Ri; g1.ldb = f.N;
                g1.Cr = f.Xr; g1.Ci = f.Xi; g1.ldc = f.N;
                g1.alpha = 1.0; g1.cplx = 1;
                g1.partial = f64_partial;
                GemmF64 g2 = g1;
                g2.Ar = f.Xr; g2.Ai = f.Xi;
                g2.Br = f.Ur; g2.Bi = f.Ui; g2.conjB = 1;
                g2.Cr = f.Rr; g2.Ci = f.Ri;
                g2.herm_lower = 1;
                TC_TRY(gemm_f64(g1, s));
                TC_TRY(gemm_f64(g2, s));
                if (renorm_every > 0 && step % renorm_every == 0)
                    TC_TRY(launch_renormalise(kRhoPlanarF64, f.Rr, f.Ri, f.n, f.scratch, s));
            }
        } else {
            TC_TRY(cgemm_batch(precision, 0, sys_dev, count, plan, status, s));
            TC_TRY(cgemm_batch(precision, 1, sys_dev, count, plan, status, s));
            if (renorm_every > 0 && step % renorm_every == 0)
                for (int k = 0; k < count; k++) TC_TRY(lowp_renorm(precision, lb[k], s));
        }
        for (int k = 0; k < count; k++) TC_TRY(observe(k, step));
        return TC_OK;
    };


    auto first = [&](cudaStream_t cs) -> tc_status {
        s = cs;
        if (precision == TC_FP64) {
            for (int k = 0; k < count; k++) {
                const int b = order[k];
                F64Sys& f = fb[k];
                f.n = n[b];
                f.N = 1 << n[b];
                const size_t NN = (size_t)f.N * f.N;
                f.Ur = ar.take<double>(NN); f.Ui = ar.take<double>(NN);
                f.Rr = ar.take<double>(NN); f.Ri = ar.take<double>(NN);
                f.Xr = ar.take<double>(NN); f.Xi = ar.take<double>(NN);
                f.scratch = ar.take<double>(observables_scratch_bytes(n[b]) / sizeof(double));
                if (!f.scratch) return fail(TC_ERR_WORKSPACE, "batch: workspace too small");
                TC_TRY(launch_split_c128(static_cast<const double*>(U[b]), f.Ur, f.Ui, NN, s));
                TC_TRY(launch_split_c128(static_cast<const double*>(rho[b]), f.Rr, f.Ri, NN, s));
            }
            if (f64_shared_bytes(n, count)) {
                f64_partial = ar.take<double>(f64_shared_bytes(n, count) / sizeof(double));
                if (!f64_partial) return fail(TC_ERR_WORKSPACE, "batch: workspace too small");
            }
        } else {
            for (int k = 0; k < count; k++) {
                const int b = order[k];
                TC_TRY(lowp_carve(n[b], precision, ar, lb[k]));
                TC_TRY(lowp_prep(precision, static_cast<const double*>(U[b]), static_cast<const double*>(rho[b]), lb[k], s));
                BatchSys& h = host[k];
                std::memset(&h, 0, sizeof(h));
                TC_TRY(batch_plan_add(plan, h, precision, lb[k].Np, lb[k].Uparts, lb[k].Rparts, lb[k].Xparts));
                h.Rr = lb[k].Rr; h.Ri = lb[k].Ri; h.Rparts = lb[k].Rparts;
                h.Xr = lb[k].Xr; h.Xi = lb[k].Xi; h.Xparts = lb[k].Xparts;
            }
            TC_CUDA(cudaMemcpyAsync(sys_dev, host.data(), sizeof(BatchSys) * count, cudaMemcpyHostToDevice, s));
            TC_CUDA(cudaStreamSynchronize(s));   // host copy of the descriptors may go
        }


        for (int k = 0; k < count; k++) TC_TRY(observe(k, 0));
        if (steps > 0) TC_TRY(one_step(1));
        return TC_OK;
    };
    auto rest = [&](cudaStream_t cs) -> tc_status {
        s = cs;
        for (int k = 2; k <= steps; k++) TC_TRY(one_step(k));
        return TC_OK;
    };
    auto tail = [&](cudaStream_t cs) -> tc_status {
        s = cs;
        // results back to the callers' rho
        for (int k = 0; k < count; k++) {
            const int b = order[k];
            if (precision == TC_FP64) {
                const size_t NN = (size_t)fb[k].N * fb[k].N;
                TC_TRY(launch_join_c128(fb[k].Rr, fb[k].Ri, static_cast<double*>(rho[b]), NN, s));
            } else {
                TC_TRY(lowp_finish(lb[k], static_cast<double*>(rho[b]), s));
            }
        }

        return TC_OK;
    };
    return run_captured(us, first, rest, tail, steps > 1);
}

}  // extern "C"
