// timing.cu -- measurement support: a count of every kernel this library
// launched, and optional CUDA-event pairs around the product (GEMM) kernels,
// recorded on the stream those kernels are launched on.
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "timing.cuh"

namespace tc {
namespace {
std::atomic<long long> g_launches{0};
std::atomic<int> g_timing_on{0};
std::mutex g_mu;
struct Pair {
    cudaEvent_t a, b;
    double flops;
};
std::vector<Pair> g_pairs;
std::vector<cudaEvent_t> g_free;
std::atomic<int> g_phases_on{0};
struct Mark {
    char name[16];
    cudaEvent_t e;
};
std::vector<Mark> g_marks;

cudaEvent_t take_event() {
    if (!g_free.empty()) {
        cudaEvent_t e = g_free.back();
        g_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

bool timing_enabled() { return g_timing_on.load() != 0; }

ProductTimer::ProductTimer(double flops, cudaStream_t s) : flops_(flops), s_(s) {
    if (!g_timing_on.load()) return;
    std::lock_guard<std::mutex> lk(g_mu);
    a_ = take_event();
    b_ = take_event();
    if (a_ && b_) cudaEventRecord(a_, s_);
}

ProductTimer::~ProductTimer() {
    if (!a_ || !b_) return;
    cudaEventRecord(b_, s_);
    std::lock_guard<std::mutex> lk(g_mu);
    g_pairs.push_back({a_, b_, flops_});
}

void phase_mark(const char* name, cudaStream_t s) {
    if (!g_phases_on.load()) return;
    std::lock_guard<std::mutex> lk(g_mu);
    Mark m{};
    std::strncpy(m.name, name, sizeof(m.name) - 1);
    m.e = take_event();
    if (!m.e) return;
    if (cudaEventRecord(m.e, s) != cudaSuccess) {
        g_free.push_back(m.e);
        return;
    }
    g_marks.push_back(m);
}

}  // namespace tc

using namespace tc;

extern "C" {

TC_API long long tc_launch_count(void) { return g_launches.load(); }

TC_API tc_status tc_timing_enable(int on) {
    g_timing_on.store(on ? 1 : 0);
    return TC_OK;
}

TC_API tc_status tc_timing_read(long long* launches, double* ms, double* flops) {
    std::lock_guard<std::mutex> lk(g_mu);
    long long n = 0;
    double t = 0.0, f = 0.0;
    tc_status st = TC_OK;
    for (auto& p : g_pairs) {
        float e = 0.f;
        if (cudaEventSynchronize(p.b) != cudaSuccess || cudaEventElapsedTime(&e, p.a, p.b) != cudaSuccess)
            st = fail(TC_ERR_CUDA, "timing: event query failed");
        t += e;
        f += p.flops;
        n++;
        g_free.push_back(p.a);
        g_free.push_back(p.b);
    }
    g_pairs.clear();
    if (launches) *launches = n;
    if (ms) *ms = t;
    if (flops) *flops = f;
    return st;
}

TC_API tc_status tc_phases_enable(int on) {
    g_phases_on.store(on ? 1 : 0);
    return TC_OK;
}

TC_API tc_status tc_phases_read(double* ms, char* names, size_t names_bytes, int max, int* count) {
    std::lock_guard<std::mutex> lk(g_mu);
    tc_status st = TC_OK;
    size_t used = 0;
    if (names && names_bytes) names[0] = '\0';
    for (size_t i = 0; i < g_marks.size(); i++) {
        float e = 0.f;
        if (cudaEventSynchronize(g_marks[i].e) != cudaSuccess ||
            (i > 0 && cudaEventElapsedTime(&e, g_marks[0].e, g_marks[i].e) != cudaSuccess))
            st = fail(TC_ERR_CUDA, "phases: event query failed");
        if ((int)i < max) {
            if (ms) ms[i] = e;
            const size_t len = std::strlen(g_marks[i].name);
            if (names && used + len + 2 <= names_bytes) {
                std::memcpy(names + used, g_marks[i].name, len);
                used += len;
                names[used++] = '\n';
                names[used] = '\0';
            }
        }
    }
    if (count) *count = (int)g_marks.size();
    for (auto& m : g_marks) g_free.push_back(m.e);
    g_marks.clear();
    return st;
}

}  // extern "C"
