// backward.cu -- reverse-mode gradient (placeholder until the adjoint lands).
#include "paths.cuh"

namespace tc {
size_t backward_bytes(int n, int steps, int ckpt_every) { (void)n; (void)steps; (void)ckpt_every; return 0; }
}  // namespace tc

extern "C" TC_API tc_status tc_evolve_backward(const tc_params*, double, int, const void*, const void*, int,
                                               const double*, double*, double*, void*, size_t, void*) {
    return tc::fail(TC_ERR_INVALID_ARG, "tc_evolve_backward is not built yet");
}
