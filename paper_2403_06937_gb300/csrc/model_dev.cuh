// model_dev.cuh -- device formulas of the Hamiltonian of Eq. 4 (Sec. II)
// for one excitation block: in block k the photon count of atom string s is
// k - popcount(s) (the closed model of Eq. 2 is k = n).  Every element is
// one fixed sequence of correctly rounded operations (no FMA contraction).
#pragma once

#include "common.cuh"

namespace tc {

__device__ __forceinline__ double h_diag(const Model& m, int k, unsigned s) {
    const int pc = __popc(s);
    return __dadd_rn(__dmul_rn(m.omega_c, (double)(k - pc)), __dmul_rn(m.omega_a, (double)pc));
}

// coupling between s and s ^ 2^bit (atom n - bit): g sqrt(p_e + 1) with p_e
// the photon count of the side where that atom is excited
__device__ __forceinline__ double h_pair(const Model& m, int k, unsigned s, int bit) {
    const unsigned se = s | (1u << bit);
    const int atom0 = m.n - 1 - bit;
    if (m.coupling == TC_COUPLING_QUBIT_PHOTON) return m.g[atom0];
    return __dmul_rn(m.g[atom0], __dsqrt_rn((double)(k - __popc(se) + 1)));
}

}  // namespace tc
