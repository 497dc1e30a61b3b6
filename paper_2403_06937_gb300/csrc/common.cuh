// common.cuh -- internal helpers of libtc: error reporting, device check,
// workspace carving and the model-parameter block passed to kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstddef>
#include <cstdint>
#include <cstdio>

#include "tc.h"

namespace tc {

// Thread-local message for tc_last_error(); returns `s` for chaining.
tc_status fail(tc_status s, const char* fmt, ...);

// Records `s` with the message of the failing CUDA call.
#define TC_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess)                                                     \
            return ::tc::fail(TC_ERR_CUDA, "%s failed: %s (%s:%d)", #call,         \
                              cudaGetErrorString(e_), __FILE__, __LINE__);         \
    } while (0)

// Every kernel launch is followed by this: it counts the launch and reports
// a launch error as TC_ERR_CUDA.
void count_launch(int k);
#define TC_LAUNCH_CHECK()                                                          \
    do {                                                                           \
        ::tc::count_launch(1);                                                     \
        TC_CUDA(cudaPeekAtLastError());                                            \
    } while (0)

#define TC_TRY(expr)                                                               \
    do {                                                                           \
        tc_status s_ = (expr);                                                     \
        if (s_ != TC_OK) return s_;                                                \
    } while (0)

// TC_OK if the current device is sm_103 (the only target compiled).
tc_status check_device();

// TC_OK if `work` is non-null, 256-byte aligned and holds `need` bytes.
tc_status check_work(void* work, size_t have, size_t need);

// Device status word: kernels OR in these bits; tc_sync_status reads them.
enum : unsigned { kStatusTimeout = 1u, kStatusNumeric = 2u };
unsigned* device_status_word();   // device address of the word (per device)

constexpr int kMaxAtoms = 16;

// Model parameters by value (fits in a kernel parameter block).
struct Model {
    int n;
    int coupling;     // tc_coupling
    double omega_a;
    double omega_c;
    double g[kMaxAtoms];
};

tc_status make_model(const tc_params* p, Model* m);

// Bump allocator over the caller's work buffer (256-byte aligned slices).
struct Arena {
    char* base;
    size_t size;
    size_t used;
    template <typename T>
    T* take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        if (used + bytes > size) return nullptr;
        T* p = reinterpret_cast<T*>(base + used);
        used += bytes;
        return p;
    }
};

inline size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace tc
