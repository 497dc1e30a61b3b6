// graph.cuh -- capture of a step loop into one CUDA graph on a library stream.
#pragma once

#include <functional>

#include "common.cuh"

namespace tc {

// Runs `first` on a library stream ordered after `user`, then captures
// `rest` on that stream into a CUDA graph, instantiates and launches it (the
// call does not wait for it), and orders `user` after it.  `first` may set kernel attributes and
// do host work that capture forbids.  With capture == false `rest` is simply
// enqueued.  `tail` runs after the graph (on the same stream).
tc_status run_captured(cudaStream_t user, const std::function<tc_status(cudaStream_t)>& first,
                       const std::function<tc_status(cudaStream_t)>& rest,
                       const std::function<tc_status(cudaStream_t)>& tail, bool capture);

}  // namespace tc
