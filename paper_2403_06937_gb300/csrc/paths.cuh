// paths.cuh -- the multi-kernel paths behind the C-ABI calls.
#pragma once

#include "kernels.cuh"

namespace tc {

// e^{-iHdt} into U (interleaved c128) using the arena for scratch.
tc_status expm_impl(const double* H, int n, double dt, const tc_expm_opts* opts, double* U, Arena& ar,
                    cudaStream_t s, int* used_degree, int* used_squarings);

// One excitation block of the model: the atom strings basis[0..d) (popcount
// at most k, sorted by popcount) with photon count k - popcount(s); pos is
// the inverse permutation over all 2^n strings.  order == pos == nullptr is
// the closed model (k = n, d = 2^n, identity order).
struct ExcitationBlock {
    int k;
    int d;
    const int* order;   // device
    const int* pos;     // device
};

// e^{-iHdt} from the model by Horner's rule with H applied as a stencil.
size_t expm_model_bytes(int n);
size_t expm_block_bytes(size_t d);
tc_status expm_block_impl(const Model& m, const ExcitationBlock& blk, const int* host_order, double dt,
                          const tc_expm_opts* opts, double* U, Arena& ar, cudaStream_t s, int* used_degree,
                          int* used_squarings);
tc_status expm_model_impl(const Model& m, double dt, const tc_expm_opts* opts, double* U, Arena& ar,
                          cudaStream_t s, int* used_degree, int* used_squarings);

// FP64 step loop (DMMA products).
tc_status evolve_f64(const double* U, double* rho, int n, int steps, int renorm_every, const Model* m,
                     double* obs, Arena& ar, cudaStream_t s);

// FP64-accurate step loop on the BF16 tensor cores (exact integer slices).
size_t evolve_oz_bytes(int n);
tc_status evolve_oz(const double* U, double* rho, int n, int steps, int renorm_every, const Model* m, double* obs,
                    Arena& ar, cudaStream_t s);

// Low-precision step loop (tcgen05 products).
size_t evolve_lowp_bytes(int n, int precision);
tc_status evolve_lowp(const double* U, double* rho, int n, int steps, int precision, int renorm_every,
                      const Model* m, double* obs, Arena& ar, cudaStream_t s);
// tc_evolve_host for the tensor-core forms: rho_host copied in by row blocks
// (the first product starts on the column blocks whose rows have arrived) and
// out by row bands (the last second product runs bottom-up, each band's
// finished entries converted and copied while the rows above are computed),
// on a copy stream of its own; rho_dev is the N x N complex128 staging.
// Sizes without group-aligned blocks, or N < 2048, copy whole around the loop.
tc_status evolve_lowp_host(const double* U, double* rho_host, double* rho_dev, int n, int steps, int precision,
                           int renorm_every, const Model* m, double* obs, Arena& ar, cudaStream_t s);
int lowp_host_chunks(int n, int precision);   // row blocks in (4, 2 or 1)
int lowp_host_bands(int n, int precision);    // row bands out (8, 4, 2 or 1)

// Open-system form (packed excitation blocks).
size_t lindblad_bytes(int n, int precision);

// Reverse-mode gradient.
size_t backward_bytes(int n, int steps, int ckpt_every, int precision);

}  // namespace tc
