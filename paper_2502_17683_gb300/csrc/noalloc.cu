// thc_cpd_mttkrp_noalloc: the FP64 matrix-free MTTKRP with every piece of scratch
// memory taken from one fixed array in the library's own device memory, so that a call
// never allocates.
//
// Who needs it: callers that may not allocate device memory while they run. Examples are
// a host that hands all device memory to its own pool allocator and forbids any other
// allocation, code that enqueues work from a context where a cudaMalloc (which can
// synchronise the device) is not allowed, and real-time loops that must not touch the
// allocator at all. They pass inputs and outputs as usual; the scratch comes from here.
//
// Where the 32 MiB come from: the array lives in this file's own device module. Under
// CUDA's default lazy module loading that module, and so the array, is created on a device
// by the first call there (its address lookup loads the module); with
// CUDA_MODULE_LOADING=EAGER it is created when the process first initialises the device.
// Either way the reservation happens once, before any work of that call is enqueued: a
// caller whose own pool will claim the device should make one call first. If the device
// has no room left at that moment the call fails with THC_CPD_ERR_CUDA and says so.
//
// Set-up: the first call on a device (with that device current) looks up the device
// address of the array with cudaGetSymbolAddress and caches it per device ordinal; make
// that first call before any stream capture begins. The cached address belongs to the
// device's primary context and stays valid for the life of the process; a caller that
// resets the device (cudaDeviceReset) or drives the library from another context must not
// use this entry point afterwards.
//
// Sharing: all calls on a device use the same array and it keeps the contents of the
// last call. Calls whose GPU work overlaps (different streams, or different host threads
// on one device) race on it and must be serialised by the caller. Nothing in it has to
// start at zero: every buffer carved from it is written completely before it is read.
#include <stdio.h>

#include <mutex>

#include "f64.cuh"
#include "thc_cpd.h"

namespace {

// 32 MiB: holds the four R_thc x R_cp buffers of problems up to R_thc * R_cp of about
// one million (for example R_thc = 960 with R_cp = 1080), plus split-K partials.
constexpr size_t kScratchBytes = size_t(32) << 20;
constexpr size_t kScratchDoubles = kScratchBytes / sizeof(double);

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {};

size_t round256(size_t doubles) { return (doubles + 31) & ~size_t(31); }

}  // namespace

extern "C" thc_cpd_status thc_cpd_mttkrp_noalloc(int o, int v, int Rt, int R, const double* Xo,
                                                 const double* Xv, const double* Z,
                                                 const double* const A[4], int mode, double* M,
                                                 const thc_cpd_opts* opts) {
    using namespace thc;
    char msg[256];
    // the same checks, in the same order and with the same messages, as thc_cpd_mttkrp
    const int chk = check_mttkrp_args(o, v, Rt, R, Xo, Xv, Z, A, mode, M);
    if (chk != THC_CPD_OK) return (thc_cpd_status)chk;
    if (opts && opts->precision != THC_CPD_FP64)
        return (thc_cpd_status)set_error(THC_CPD_ERR_UNSUPPORTED, "the allocation-free MTTKRP is FP64 only");
    const size_t RtR = round256((size_t)Rt * R);
    const size_t need = 4 * RtR;  // three projections W_k and the Z product Y
    if (need > kScratchDoubles) {
        snprintf(msg, sizeof msg,
                 "R_thc * R_cp = %d * %d needs %zu bytes of scratch; the allocation-free "
                 "MTTKRP has %zu (use thc_cpd_mttkrp)",
                 Rt, R, need * sizeof(double), kScratchBytes);
        return (thc_cpd_status)set_error(THC_CPD_ERR_SHAPE, msg);
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return (thc_cpd_status)set_error(THC_CPD_ERR_CUDA, "no current CUDA device");
    double* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e == cudaErrorMemoryAllocation) {
                cudaGetLastError();
                snprintf(msg, sizeof msg,
                         "the 32 MiB scratch array could not be created on device %d (its module "
                         "is loaded by the first call there): no device memory left; make the "
                         "first call before another allocator claims the device",
                         dev);
                return (thc_cpd_status)set_error(THC_CPD_ERR_CUDA, msg);
            }
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                snprintf(msg, sizeof msg, "cudaGetSymbolAddress of the scratch array failed: %s",
                         cudaGetErrorString(e));
                return (thc_cpd_status)set_error(THC_CPD_ERR_CUDA, msg);
            }
            g_scratch_ptr[dev] = (double*)p;
        }
        base = g_scratch_ptr[dev];
    }
    cudaStream_t st = opts ? (cudaStream_t)opts->stream : (cudaStream_t)0;
    const int n[4] = {o, v, o, v};
    const double* X[4] = {Xo, Xv, Xo, Xv};
    double* W[4];
    for (int k = 0; k < 4; ++k) W[k] = base + k * RtR;  // W[mode] is used as Y
    double* Y = W[mode];
    double* part = base + 4 * RtR;
    const size_t part_cap = kScratchDoubles - 4 * RtR;  // split-K partials (may be 0)

    for (int k = 0; k < 4; ++k)
        if (k != mode)
            dgemm(st, true, Rt, R, n[k], X[k], Rt, A[k], nullptr, R, W[k], R, nullptr, false, part,
                  part_cap);
    if (mode < 2)
        dgemm(st, false, Rt, R, Rt, Z, Rt, W[2], W[3], R, Y, R, nullptr, false, part, part_cap);
    else
        dgemm(st, true, Rt, R, Rt, Z, Rt, W[0], W[1], R, Y, R, nullptr, false, part, part_cap);
    const int partner = mode == 0 ? 1 : mode == 1 ? 0 : mode == 2 ? 3 : 2;
    dgemm(st, false, n[mode], R, Rt, X[mode], Rt, W[partner], Y, R, M, R, nullptr, false, part,
          part_cap);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "launch failed: %s", cudaGetErrorString(e));
        return (thc_cpd_status)set_error(THC_CPD_ERR_CUDA, msg);
    }
    return THC_CPD_OK;
}
