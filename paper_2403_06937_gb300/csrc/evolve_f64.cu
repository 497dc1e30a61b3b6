// evolve_f64.cu -- the plain FP64 form of the step loop: rho <- U rho U^dag
// (Sec. III.A, Eq. 6), evaluated as the two products of Eq. 12 on the DMMA
// GEMM:  X = U rho (full), then rho' = X conj(U) (U complex symmetric, so
// conj(U) = U^dag), of which only the block-lower triangle is computed and
// mirrored, keeping rho exactly Hermitian.  Steps 2..K are captured into one
// CUDA graph (unless kernel timing is on).
#include "graph.cuh"
#include "paths.cuh"
#include "timing.cuh"

namespace tc {

tc_status evolve_f64(const double* U, double* rho, int n, int steps, int renorm_every, const Model* m,
                     double* obs, Arena& ar, cudaStream_t s) {
    const int N = 1 << n;
    const size_t NN = (size_t)N * N;
    double* Ur = ar.take<double>(NN);
    double* Ui = ar.take<double>(NN);
    double* Rr = ar.take<double>(NN);
    double* Ri = ar.take<double>(NN);
    double* Xr = ar.take<double>(NN);
    double* Xi = ar.take<double>(NN);
    double* scratch = ar.take<double>(observables_scratch_bytes(n) / sizeof(double));
    double* partial = N <= kSplitMaxDim ? ar.take<double>(gemm_f64_splitk_bytes() / sizeof(double)) : nullptr;
    if (!scratch || (N <= kSplitMaxDim && !partial)) return fail(TC_ERR_WORKSPACE, "evolve: workspace too small");
    const int stride = TC_OBS_STRIDE(n);

    GemmF64 g1{};
    g1.M = g1.N = g1.K = N;
    g1.Ar = Ur; g1.Ai = Ui; g1.lda = N;
    g1.Br = Rr; g1.Bi = Ri; g1.ldb = N;
    g1.Cr = Xr; g1.Ci = Xi; g1.ldc = N;
    g1.alpha = 1.0; g1.beta = 0.0;
    g1.cplx = 1;
    g1.partial = partial;
    GemmF64 g2 = g1;
    g2.Ar = Xr; g2.Ai = Xi;
    g2.Br = Ur; g2.Bi = Ui; g2.conjB = 1;
    g2.Cr = Rr; g2.Ci = Ri;
    g2.herm_lower = 1;

    auto one_step = [&](int k, cudaStream_t cs) -> tc_status {
        {
            ProductTimer t(8.0 * (double)N * N * N, cs);   // X = U rho: 8 N^3
            TC_TRY(gemm_f64(g1, cs));
        }
        {
            ProductTimer t(4.0 * (double)N * N * N, cs);   // rho' = X U^dag, Hermitian half: 4 N^3
            TC_TRY(gemm_f64(g2, cs));
        }
        if (renorm_every > 0 && k % renorm_every == 0)
            TC_TRY(launch_renormalise(kRhoPlanarF64, Rr, Ri, n, scratch, cs));
        if (obs) TC_TRY(launch_observables(kRhoPlanarF64, Rr, Ri, m, n, obs + (size_t)k * stride, scratch, cs));
        return TC_OK;
    };
    auto first = [&](cudaStream_t cs) -> tc_status {
        TC_TRY(launch_split_c128(U, Ur, Ui, NN, cs));
        TC_TRY(launch_split_c128(rho, Rr, Ri, NN, cs));
        if (obs) TC_TRY(launch_observables(kRhoPlanarF64, Rr, Ri, m, n, obs, scratch, cs));
        if (steps >= 1) TC_TRY(one_step(1, cs));
        return TC_OK;
    };
    auto rest = [&](cudaStream_t cs) -> tc_status {
        for (int k = 2; k <= steps; k++) TC_TRY(one_step(k, cs));
        return TC_OK;
    };
    auto tail = [&](cudaStream_t cs) -> tc_status { return launch_join_c128(Rr, Ri, rho, NN, cs); };
    return run_captured(s, first, rest, tail, steps > 2 && !timing_enabled());
}

}  // namespace tc
