// Shared host/device helpers for the THC-CPD library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <string>

namespace thc {

// SMs of the current device (GB300: 152), queried once per device: grids of persistent and
// grid-stride kernels follow the part they run on.
inline int num_sms() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 152;
        cache[dev] = n;
    }
    return cache[dev];
}

// Blocks of the fixed-order reductions (loss, norms): a constant, so that the order of the
// sums, and with it the result's bits, is the same on every device.
constexpr int kReduceBlocks = 304;

// Device-side scalars of one ALS run (one struct per problem).
struct DevScalars {
    double normG2;     // ||G||^2
    double loss;       // loss after the last evaluated sweep
    double fit;        // fit after the last evaluated sweep
    double inner;      // <G, Gt>
    double cpdn2;      // ||Gt||^2
    double prev_fit;   // fit of the previous evaluated sweep (NaN before the first)
    double maxdiag;    // max_i H_ii of the current normal matrix
    double pad0;
    int fail_mask;     // bit k: Cholesky pivot failure in mode k of this sweep
    int done;          // convergence reached
    int nonfinite;     // a loss/fit came out non-finite
    int pad1;
};

// Bump allocator over one cudaMallocAsync block; every carve is 256-byte aligned.
struct Arena {
    char* base = nullptr;
    size_t cap = 0, off = 0;
    template <class T>
    T* take(size_t n) {
        size_t bytes = (n * sizeof(T) + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base + off);
        off += bytes;
        return p;
    }
    template <class T>
    static size_t need(size_t n) { return (n * sizeof(T) + 255) & ~size_t(255); }
};

inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

// Record the message returned by thc_cpd_last_error() for this host thread; returns s.
int set_error(int s, const char* msg);

// The argument checks of thc_cpd_mttkrp (shapes, null pointers, mode), shared by every
// MTTKRP entry point so that they accept and reject the same arguments with the same
// messages. Returns a thc_cpd_status; the message is set on failure.
int check_mttkrp_args(int o, int v, int Rt, int R, const double* Xo, const double* Xv,
                      const double* Z, const double* const* A, int mode, const double* M);
// The shape and pointer checks alone (THC factors and the four CP factors).
int check_problem_args(int o, int v, int Rt, int R, const double* Xo, const double* Xv,
                       const double* Z, const double* const* A);

}  // namespace thc
