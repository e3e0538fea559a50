// Launch accounting and optional per-kernel-class CUDA-event timing (for roofline
// reporting). Timing is off unless thc_cpd_profile(1) was called.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace thc {

enum KClass { KC_DGEMM = 0, KC_CHOL = 1, KC_BSOLVE = 2, KC_AUX = 3, KC_TC = 4, KC_OZ = 5, KC_TCZ = 6, KC_N = 7 };

void count_launch(int n = 1);
bool prof_on();
// Bracket a group of launches of one class on `st`; flops/bytes are the group's
// algorithmic work.
struct ProfScope {
    int cls;
    cudaStream_t st;
    double flops, bytes;
    cudaEvent_t e0 = nullptr;
    ProfScope(cudaStream_t s, int c, double f, double b = 0.0);
    ~ProfScope();
};

// A named range on the host timeline (NVTX v3, header-only): shown by profilers that record
// NVTX (nsys timelines, ncu's --nvtx-include filters), a no-op when none is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace thc
