// timing.cuh -- launch counting and optional event timing of product kernels.
#pragma once

#include "common.cuh"

namespace tc {

// True while tc_timing_enable(1) is in effect (the step loops then launch
// directly instead of through a CUDA graph, so each launch is bracketed).
bool timing_enabled();

// RAII: when timing is enabled, records an event pair around the enclosed
// product-kernel launch(es) on stream `s`, credited with `flops`.
class ProductTimer {
  public:
    ProductTimer(double flops, cudaStream_t s);
    ~ProductTimer();
    ProductTimer(const ProductTimer&) = delete;
    ProductTimer& operator=(const ProductTimer&) = delete;

  private:
    double flops_;
    cudaStream_t s_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};

// When phase marks are enabled (tc_phases_enable), records a timing event on
// stream `s` named `name` (copied, at most 15 characters); tc_phases_read
// returns the marks' times relative to the first one.  A no-op otherwise.
void phase_mark(const char* name, cudaStream_t s);

}  // namespace tc
