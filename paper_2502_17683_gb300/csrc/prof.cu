#include <atomic>
#include <mutex>
#include <vector>

#include "prof.cuh"
#include "thc_cpd.h"

namespace thc {
namespace {
std::atomic<long> g_launches{0};
std::atomic<int> g_prof{0};
struct Rec {
    int cls;
    cudaEvent_t a, b;
    double flops, bytes;
};
std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event() {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
bool prof_on() { return g_prof.load(std::memory_order_relaxed) != 0; }

ProfScope::ProfScope(cudaStream_t s, int c, double f, double b) : cls(c), st(s), flops(f), bytes(b) {
    if (prof_on()) {
        e0 = get_event();
        cudaEventRecord(e0, st);
    }
}

ProfScope::~ProfScope() {
    if (!e0) return;
    cudaEvent_t e1 = get_event();
    cudaEventRecord(e1, st);
    std::lock_guard<std::mutex> lk(g_mu);
    g_recs.push_back({cls, e0, e1, flops, bytes});
}

}  // namespace thc

extern "C" {

long thc_cpd_launch_count(void) { return thc::g_launches.load(); }

void thc_cpd_profile(int enable) {
    using namespace thc;
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    g_prof.store(enable ? 1 : 0);
}

int thc_cpd_profile_read(thc_cpd_kstat* out, int max_classes) {
    using namespace thc;
    std::lock_guard<std::mutex> lk(g_mu);
    const int n = max_classes < KC_N ? max_classes : KC_N;
    for (int c = 0; c < n; ++c) out[c] = thc_cpd_kstat{0.0, 0.0, 0.0, 0};
    for (auto& r : g_recs) {
        if (r.cls >= n) continue;
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess) return -1;
        cudaEventElapsedTime(&ms, r.a, r.b);
        out[r.cls].ms += ms;
        out[r.cls].flops += r.flops;
        out[r.cls].bytes += r.bytes;
        out[r.cls].groups += 1;
    }
    return n;
}

}  // extern "C"
