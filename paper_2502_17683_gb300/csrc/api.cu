// C ABI of the THC-CPD library: argument checks, workspace, and the host-side order of
// the kernels of one ALS sweep (textbook CP-ALS on Eq. lossF, Sec. 2.1).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <memory>
#include <string>
#include <vector>

#include "thc_cpd.h"
#include "f64.cuh"
#include "mixed.cuh"
#include "oz.cuh"
#include "prof.cuh"

namespace {

using namespace thc;

thread_local std::string g_err;

thc_cpd_status set_err(thc_cpd_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CK(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return set_err(THC_CPD_ERR_CUDA, "%s failed at %s:%d: %s", #call, __FILE__,     \
                           __LINE__, cudaGetErrorString(e_));                               \
    } while (0)

#define CKS(expr)                              \
    do {                                       \
        thc_cpd_status s_ = (expr);            \
        if (s_ != THC_CPD_OK) return s_;       \
    } while (0)

struct Shape {
    int o, v, Rt, R;
    int n[4];
    int nmax;
};

thc_cpd_status check_shape(int o, int v, int Rt, int R, Shape* s) {
    if (o < 1 || v < 1 || Rt < 1 || R < 1)
        return set_err(THC_CPD_ERR_SHAPE, "dimensions must be >= 1 (o=%d v=%d Rt=%d R=%d)", o, v, Rt, R);
    const long lim = 0x7fffffffL;
    if ((long)(o + v) * R >= lim || (long)Rt * R >= lim || (long)R * R >= lim ||
        (long)Rt * Rt >= lim || (long)(R + std::max(o, v)) * R >= lim)
        return set_err(THC_CPD_ERR_SHAPE, "dimensions too large (o=%d v=%d Rt=%d R=%d)", o, v, Rt, R);
    s->o = o;
    s->v = v;
    s->Rt = Rt;
    s->R = R;
    s->n[0] = o;
    s->n[1] = v;
    s->n[2] = o;
    s->n[3] = v;
    s->nmax = std::max(o, v);
    return THC_CPD_OK;
}

thc_cpd_status check_ptrs(const double* Xo, const double* Xv, const double* Z,
                          const double* const* A) {
    if (!Xo || !Xv || !Z) return set_err(THC_CPD_ERR_ARG, "Xo, Xv and Z must be non-null");
    if (A) {
        for (int k = 0; k < 4; ++k)
            if (!A[k]) return set_err(THC_CPD_ERR_ARG, "A[%d] is null", k);
    }
    return THC_CPD_OK;
}

thc_cpd_status check_prec(const thc_cpd_opts* opts) {
    const int p = opts ? opts->precision : THC_CPD_FP64;
    if (p != THC_CPD_FP64 && p != THC_CPD_BF16X3 && p != THC_CPD_TF32X3)
        return set_err(THC_CPD_ERR_ARG, "unknown precision %d", p);
    if (p != THC_CPD_FP64 && !mixed_supported())
        return set_err(THC_CPD_ERR_UNSUPPORTED, "split tensor-core precision needs an sm_103 device");
    const int l = opts ? opts->ldl : THC_CPD_LDL_AUTO;
    if (l != THC_CPD_LDL_AUTO && l != THC_CPD_LDL_BLOCKED && l != THC_CPD_LDL_DATAFLOW &&
        l != THC_CPD_LDL_EMULATED)
        return set_err(THC_CPD_ERR_ARG, "unknown ldl variant %d", l);
    return THC_CPD_OK;
}

// the limit of the dataflow solve's device-side waits for launches from this thread
void set_wait_limit(const thc_cpd_opts* o) {
    const double sec = o ? o->wait_limit_s : 0.0;
    flow_set_wait_ns(sec > 0.0 ? (unsigned long long)std::min(sec * 1e9, 6e10) : 0ull);
}

cudaStream_t stream_of(const thc_cpd_opts* o) {
    return o ? (cudaStream_t)o->stream : (cudaStream_t)0;
}

// Bounded device waits that gave up during this call (flags read and cleared; call after
// the stream has drained).
thc_cpd_status kernel_errors(bool mixed) {
    if (int e = flow_take_error())
        return set_err(THC_CPD_ERR_TIMEOUT, "LDL^T dataflow wait gave up (code %d)", e);
    if (int e = oz_take_error())
        return set_err(THC_CPD_ERR_TIMEOUT, "emulated-product kernel wait gave up (code %d)", e);
    if (mixed) {
        if (int e = mixed_take_error())
            return set_err(THC_CPD_ERR_TIMEOUT, "tensor-core kernel wait gave up (code %d)", e);
    }
    return THC_CPD_OK;
}

// Pinned host copy of the device scalars (one per host thread).
DevScalars* host_scalars() {
    thread_local DevScalars* h = nullptr;
    if (!h) {
        if (cudaMallocHost((void**)&h, sizeof(DevScalars)) != cudaSuccess) h = nullptr;
    }
    return h;
}

// Two pinned slots for the scalars of consecutive sweeps of a pipelined run.
DevScalars* host_scalar_slots() {
    thread_local DevScalars* h = nullptr;
    if (!h) {
        if (cudaMallocHost((void**)&h, 2 * sizeof(DevScalars)) != cudaSuccess) h = nullptr;
    }
    return h;
}

// Everything one call needs on the device, carved from a single stream-ordered block.
struct Ctx {
    Shape s;
    const double* X[4];
    const double* Z;
    cudaStream_t st;
    int prec;
    void* block = nullptr;
    double* W[4] = {};
    double* G[4] = {};
    double* Y = nullptr;
    double* Haug = nullptr;
    double* LinvD = nullptr;
    int* counters = nullptr;
    int* flow_sync = nullptr;
    int* bs_sync = nullptr;
    // Dataflow factorisation (one persistent launch per solve); flow_ctas > 0 caps its grid
    // for the batched driver, where problems share the GPU.
    bool dataflow = true;
    int flow_ctas = 0;
    // two-level factorisation with emulated FP64 tensor-core trailing updates; with it the
    // Grams and the FP64-accuracy products of the split path (its loss, the learned step's
    // trial losses) also run as emulated FP64 products
    bool emulated = false;
    OzWs oz;
    double* part = nullptr;
    size_t part_cap = 0;
    double* red = nullptr;
    double* ones = nullptr;
    DevScalars* sc = nullptr;
    DevScalars* sc_snap = nullptr;  // rollback snapshot in use (one of the two slots below)
    double* Asnap[4] = {};
    double* lamsnap = nullptr;
    DevScalars* sc_slot[2] = {};    // the state before sweeps of either parity
    double* Asnap_slot[2][4] = {};
    double* lamsnap_slot[2] = {};
    cudaEvent_t ev_sc[2] = {nullptr, nullptr};  // a sweep's scalars reached the host slot
    // ||G||^2 set-up
    double* S = nullptr;
    double* T = nullptr;
    double* U = nullptr;
    // checked replay (pseudo-inverse) buffers
    double* Hsave = nullptr;
    double* Msave = nullptr;
    double* pV = nullptr;
    double* pw = nullptr;
    double* pT = nullptr;
    void* safe_block = nullptr;
    MixedWs mx;
    // CUDA graphs of one sweep (index: loss evaluated or not) on an internal stream
    cudaStream_t gst = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int gprec[2] = {-1, -1};
    long glaunch[2] = {0, 0};

    ~Ctx() {
        for (auto& g : gexec)
            if (g) cudaGraphExecDestroy(g);
        for (auto& e : ev_sc)
            if (e) cudaEventDestroy(e);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (gst) cudaStreamDestroy(gst);
        if (safe_block) cudaFreeAsync(safe_block, st);
        if (block) cudaFreeAsync(block, st);
    }
};

enum : unsigned { NEED_ALS = 1, NEED_NORM = 2, NEED_SAFE = 4, NEED_BATCHED = 8 };

// Whether a single problem's LDL^T runs in panels with emulated tensor-core updates: on
// request, and by default from R = 1024 on (measured on GB300, BF16x3 sweeps: emulated vs
// dataflow 334 vs 395 sweeps/s at R = 720, 211 vs 207 at 1080, 104 vs 59 at 1800), within
// the panel plans' range.
constexpr int kEmulatedMinR = 1024;
bool use_emulated_ldl(int ldl, int R, int nmax) {
    const bool fits = R > kOzPanel && R <= 4096 && cdiv((long)R + nmax - kOzPanel, 16) <= 256;
    return fits && (ldl == THC_CPD_LDL_EMULATED || (ldl == THC_CPD_LDL_AUTO && R >= kEmulatedMinR));
}

// grid cap of the dataflow factorisation when the batched driver is asked for it
constexpr int kBatchedFlowCtas = 32;

thc_cpd_status ctx_init(Ctx& c, const Shape& s, const double* Xo, const double* Xv,
                        const double* Z, const thc_cpd_opts* opts, unsigned need) {
    c.s = s;
    c.X[0] = Xo;
    c.X[1] = Xv;
    c.X[2] = Xo;
    c.X[3] = Xv;
    c.Z = Z;
    c.st = stream_of(opts);
    c.prec = opts ? opts->precision : THC_CPD_FP64;
    set_wait_limit(opts);
    const int Rt = s.Rt, R = s.R, nmax = s.nmax;
    size_t pc = 0;
    for (int k = 0; k < 2; ++k) {
        const int n = s.n[k];
        pc = std::max(pc, dgemm_part_need(Rt, R, n));
        pc = std::max(pc, dgemm_part_need(n, R, Rt));
        pc = std::max(pc, dgemm_part_need(R, R, n));
        pc = std::max(pc, dgemm_part_need(Rt, Rt, n));
    }
    pc = std::max(pc, dgemm_part_need(Rt, R, Rt));
    if (need & NEED_NORM) pc = std::max(pc, dgemm_part_need(Rt, Rt, Rt));
    if (need & NEED_SAFE) pc = std::max(pc, dgemm_part_need(nmax, R, R));
    c.part_cap = pc;
    size_t bytes = 0;
    const size_t RtR = (size_t)Rt * R, RR = (size_t)R * R;
    bytes += 4 * Arena::need<double>(RtR);                 // W
    bytes += 4 * Arena::need<double>(RR);                  // G
    bytes += Arena::need<double>(RtR);                     // Y
    bytes += Arena::need<double>((size_t)(R + nmax) * R);  // Haug
    bytes += Arena::need<double>(RR + R);                  // X = L D and D^{-1}
    bytes += Arena::need<int>(cdiv(R, 32));               // arrival counters of the LDL^T
    bytes += Arena::need<int>(flow_sync_ints(R, nmax));   // dataflow LDL^T progress
    bytes += Arena::need<int>(bsolve_sync_ints(nmax));    // sliced backward solve progress
    bytes += Arena::need<double>(pc);
    bytes += Arena::need<double>(loss_red_need() + 2 * kReduceBlocks);
    bytes += Arena::need<double>(R);
    bytes += 2 * Arena::need<DevScalars>(1);
    if (need & NEED_ALS) {  // two rollback snapshots (pipelined runs alternate)
        bytes += Arena::need<DevScalars>(1);
        bytes += 2 * (2 * Arena::need<double>((size_t)s.o * R) + 2 * Arena::need<double>((size_t)s.v * R));
        bytes += 2 * Arena::need<double>(R);
    }
    if (need & NEED_NORM) bytes += 3 * Arena::need<double>((size_t)Rt * Rt);
    const bool mixed = c.prec != THC_CPD_FP64;
    const bool tf32 = c.prec == THC_CPD_TF32X3;
    if (mixed) bytes += mixed_ws_bytes(tf32, s.o, s.v, Rt, R);
    // the factorisation: plans (host task lists, uploaded once per shape) are prepared here,
    // never inside a capture
    const int ldl = opts ? opts->ldl : THC_CPD_LDL_AUTO;
    c.emulated = use_emulated_ldl(ldl, R, nmax) && oz_prepare(R, s.o) && oz_prepare(R, s.v);
    int oz_ra = std::max(R + nmax, Rt), oz_rb = R;
    size_t oz_part = 0;
    if (c.emulated) bsolve_ws_rows(R, nmax, &oz_ra, &oz_rb, &oz_part);
    if (c.emulated) oz_ldl_ws_rows(R, nmax, &oz_ra, &oz_rb);
    if (c.emulated) bytes += oz_ws_bytes(oz_ra, oz_rb, oz_part);
    CK(cudaMallocAsync(&c.block, bytes, c.st));
    Arena ar;
    ar.base = (char*)c.block;
    ar.cap = bytes;
    for (int k = 0; k < 4; ++k) c.W[k] = ar.take<double>(RtR);
    for (int k = 0; k < 4; ++k) c.G[k] = ar.take<double>(RR);
    c.Y = ar.take<double>(RtR);
    c.Haug = ar.take<double>((size_t)(R + nmax) * R);
    c.LinvD = ar.take<double>(RR + R);
    c.counters = ar.take<int>(cdiv(R, 32));
    c.flow_sync = ar.take<int>(flow_sync_ints(R, nmax));
    c.bs_sync = ar.take<int>(bsolve_sync_ints(nmax));
    // zero once: every launch that uses them leaves them zero again
    CK(cudaMemsetAsync(c.flow_sync, 0, sizeof(int) * flow_sync_ints(R, nmax), c.st));
    CK(cudaMemsetAsync(c.bs_sync, 0, sizeof(int) * bsolve_sync_ints(nmax), c.st));
    c.part = ar.take<double>(pc);
    c.red = ar.take<double>(loss_red_need() + 2 * kReduceBlocks);
    c.ones = ar.take<double>(R);
    c.sc = ar.take<DevScalars>(1);
    c.sc_snap = ar.take<DevScalars>(1);
    if (need & NEED_ALS) {
        c.sc_slot[0] = c.sc_snap;
        c.sc_slot[1] = ar.take<DevScalars>(1);
        for (int b = 0; b < 2; ++b) {
            for (int k = 0; k < 4; ++k) c.Asnap_slot[b][k] = ar.take<double>((size_t)s.n[k] * R);
            c.lamsnap_slot[b] = ar.take<double>(R);
        }
        for (int k = 0; k < 4; ++k) c.Asnap[k] = c.Asnap_slot[0][k];
        c.lamsnap = c.lamsnap_slot[0];
    }
    if (need & NEED_NORM) {
        c.S = ar.take<double>((size_t)Rt * Rt);
        c.T = ar.take<double>((size_t)Rt * Rt);
        c.U = ar.take<double>((size_t)Rt * Rt);
    }
    if (mixed) {
        mixed_ws_carve(c.mx, ar, tf32, s.o, s.v, Rt, R);
        CK(mixed_setup(c.mx, c.st, Xo, Xv, Z));
    }
    if (c.emulated) oz_ws_carve(c.oz, ar, oz_ra, oz_rb, oz_part);
    fill(c.st, c.ones, R, 1.0);
    c.dataflow = c.emulated || ldl == THC_CPD_LDL_DATAFLOW ||
                 (ldl == THC_CPD_LDL_AUTO && !(need & NEED_BATCHED));
    c.flow_ctas = (need & NEED_BATCHED) ? kBatchedFlowCtas : 0;
    if (c.dataflow) {
        flow_prepare(R, s.o);
        flow_prepare(R, s.v);
    }
    CK(cudaGetLastError());
    return THC_CPD_OK;
}

thc_cpd_status ctx_safe_buffers(Ctx& c) {
    if (c.Hsave) return THC_CPD_OK;
    const int R = c.s.R, nmax = c.s.nmax;
    const size_t RR = (size_t)R * R;
    const size_t TT = std::max(RR, (size_t)nmax * R);  // pinv scratch T is n x R
    size_t bytes = 2 * Arena::need<double>(RR) + Arena::need<double>(TT) +
                   2 * Arena::need<double>((size_t)nmax * R) + Arena::need<double>(R);
    void* p = nullptr;
    CK(cudaMallocAsync(&p, bytes, c.st));
    Arena ar;
    ar.base = (char*)p;
    ar.cap = bytes;
    c.Hsave = ar.take<double>(RR);
    c.pV = ar.take<double>(RR);
    c.pT = ar.take<double>(TT);
    c.Msave = ar.take<double>((size_t)nmax * R);
    (void)ar.take<double>((size_t)nmax * R);
    c.pw = ar.take<double>(R);
    c.safe_block = p;
    return THC_CPD_OK;
}

// ---- building blocks -----------------------------------------------------------------
void gemm64(Ctx& c, bool trans_a, int M, int N, int K, const double* A, int lda, const double* B,
            const double* B2, int ldb, double* C, int ldc, bool symm);

void compute_normG2(Ctx& c) {
    const int o = c.s.o, v = c.s.v, Rt = c.s.Rt;
    // S = (Xo^T Xo) o (Xv^T Xv); U = S Z S; ||G||^2 = sum Z o U
    dgemm(c.st, true, Rt, Rt, o, c.X[0], Rt, c.X[0], nullptr, Rt, c.T, Rt, nullptr, true, c.part, c.part_cap);
    dgemm(c.st, true, Rt, Rt, v, c.X[1], Rt, c.X[1], nullptr, Rt, c.S, Rt, c.T, true, c.part, c.part_cap);
    gemm64(c, false, Rt, Rt, Rt, c.S, Rt, c.Z, nullptr, Rt, c.T, Rt, false);
    gemm64(c, false, Rt, Rt, Rt, c.T, Rt, c.S, nullptr, Rt, c.U, Rt, false);
    sum_hadamard_normG2(c.st, (long)Rt * Rt, c.Z, c.U, c.red, c.sc);
}

// An FP64-accuracy product: emulated on the tensor cores when the context has the
// emulated path (same result up to rounding), else on the FP64 pipes.
void gemm64(Ctx& c, bool trans_a, int M, int N, int K, const double* A, int lda, const double* B,
            const double* B2, int ldb, double* C, int ldc, bool symm) {
    if (c.emulated && M <= c.oz.rowsA && N <= c.oz.rowsB)
        oz_dgemm(c.st, trans_a, M, N, K, A, lda, B, B2, ldb, C, ldc, nullptr, symm, c.oz);
    else
        dgemm(c.st, trans_a, M, N, K, A, lda, B, B2, ldb, C, ldc, nullptr, symm, c.part, c.part_cap);
}

// W_k = X_k^T A_k; emu: as an emulated product (the split path's FP64 loss), else on the
// FP64 pipes (the FP64 path's MTTKRP)
void project_fp64(Ctx& c, int k, const double* Ak, bool emu = false) {
    if (emu) {
        gemm64(c, true, c.s.Rt, c.s.R, c.s.n[k], c.X[k], c.s.Rt, Ak, nullptr, c.s.R, c.W[k], c.s.R, false);
        return;
    }
    dgemm(c.st, true, c.s.Rt, c.s.R, c.s.n[k], c.X[k], c.s.Rt, Ak, nullptr, c.s.R, c.W[k], c.s.R,
          nullptr, false, c.part, c.part_cap);
}

void gram_fp64(Ctx& c, int k, const double* Ak) {
    if (c.emulated) {
        gemm64(c, true, c.s.R, c.s.R, c.s.n[k], Ak, c.s.R, Ak, nullptr, c.s.R, c.G[k], c.s.R, true);
        return;
    }
    dgemm(c.st, true, c.s.R, c.s.R, c.s.n[k], Ak, c.s.R, Ak, nullptr, c.s.R, c.G[k], c.s.R, nullptr,
          true, c.part, c.part_cap);
}

// Y = Z (W3 o W4) for modes 0,1 and Y = Z^T (W1 o W2) for modes 2,3
void zgemm_fp64(Ctx& c, int half, bool emu = false) {
    const int Rt = c.s.Rt, R = c.s.R;
    if (emu) {
        if (half == 0)
            gemm64(c, false, Rt, R, Rt, c.Z, Rt, c.W[2], c.W[3], R, c.Y, R, false);
        else
            gemm64(c, true, Rt, R, Rt, c.Z, Rt, c.W[0], c.W[1], R, c.Y, R, false);
        return;
    }
    if (half == 0)
        dgemm(c.st, false, Rt, R, Rt, c.Z, Rt, c.W[2], c.W[3], R, c.Y, R, nullptr, false, c.part, c.part_cap);
    else
        dgemm(c.st, true, Rt, R, Rt, c.Z, Rt, c.W[0], c.W[1], R, c.Y, R, nullptr, false, c.part, c.part_cap);
}

int partner_of(int k) { return k == 0 ? 1 : k == 1 ? 0 : k == 2 ? 3 : 2; }

// M_k = X_k (W_partner o Y)
void backproject_fp64(Ctx& c, int k, double* M) {
    dgemm(c.st, false, c.s.n[k], c.s.R, c.s.Rt, c.X[k], c.s.Rt, c.W[partner_of(k)], c.Y, c.s.R, M,
          c.s.R, nullptr, false, c.part, c.part_cap);
}

void others(int k, int* a, int* b, int* d) {
    int t[3], j = 0;
    for (int m = 0; m < 4; ++m)
        if (m != k) t[j++] = m;
    *a = t[0];
    *b = t[1];
    *d = t[2];
}

// W_k and G_k for every mode from the current factors (start of a run / after rollback)
void refresh_state(Ctx& c, const double* const A[4]) {
    for (int k = 0; k < 4; ++k) {
        if (c.prec == THC_CPD_FP64)
            project_fp64(c, k, A[k]);
        else
            mixed_project(c.mx, c.st, k, A[k], false);
        gram_fp64(c, k, A[k]);
    }
}

// One mode update. M_k is formed in the Haug rows; returns with A[k], lam, G_k, W_k new.
thc_cpd_status mode_update(Ctx& c, double* const A[4], double* lam, int k, bool safe,
                           int* used_pinv) {
    NvtxRange nvtx_range("thc_cpd mode update");
    const int R = c.s.R, n = c.s.n[k];
    double* Mrows = c.Haug + (size_t)R * R;
    if (c.prec == THC_CPD_FP64)
        backproject_fp64(c, k, safe ? c.Msave : Mrows);
    else
        CK(mixed_backproject(c.mx, c.st, k, safe ? c.Msave : Mrows));
    int a, b, d;
    others(k, &a, &b, &d);
    hadamard3(c.st, R, c.G[a], c.G[b], c.G[d], safe ? c.Hsave : c.Haug, c.sc);
    if (safe) {
        CK(cudaMemcpyAsync(Mrows, c.Msave, sizeof(double) * n * R, cudaMemcpyDeviceToDevice, c.st));
        CK(cudaMemcpyAsync(c.Haug, c.Hsave, sizeof(double) * R * R, cudaMemcpyDeviceToDevice, c.st));
    }
    chol_solve(c.st, R, n, c.Haug, A[k], c.LinvD, c.LinvD + (size_t)R * R, c.sc, k, c.counters,
               c.dataflow ? c.flow_sync : nullptr, c.flow_ctas, c.bs_sync, c.emulated ? &c.oz : nullptr);
    if (safe) {
        DevScalars* h = host_scalars();
        if (!h) return set_err(THC_CPD_ERR_ALLOC, "pinned host buffer allocation failed");
        CK(cudaMemcpyAsync(h, c.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c.st));
        CK(cudaStreamSynchronize(c.st));
        if (h->fail_mask & (1 << k)) {
            int sweeps = 0;
            CK(pinv_solve(c.st, R, n, c.Hsave, c.Msave, A[k], c.pV, c.pw, c.pT, &sweeps));
            *used_pinv = 1;
            int zero = 0;
            CK(cudaMemcpyAsync(&c.sc->fail_mask, &zero, sizeof(int), cudaMemcpyHostToDevice, c.st));
            CK(cudaStreamSynchronize(c.st));
        }
    }
    normalise_columns(c.st, n, R, A[k], lam, c.LinvD);  // panel buffer is free after the solve
    gram_fp64(c, k, A[k]);
    if (c.prec == THC_CPD_FP64)
        project_fp64(c, k, A[k]);
    else
        CK(mixed_project(c.mx, c.st, k, A[k], true));
    CK(cudaGetLastError());
    return THC_CPD_OK;
}

// One sweep over modes 0..3 (+ the FP64 loss when eval_loss).
thc_cpd_status sweep(Ctx& c, double* const A[4], double* lam, bool safe, bool eval_loss,
                     double tol, int* used_pinv) {
    NvtxRange nvtx_range("thc_cpd sweep");
    for (int k = 0; k < 4; ++k) {
        if (k == 0 || k == 2) {
            if (c.prec == THC_CPD_FP64)
                zgemm_fp64(c, k / 2);
            else
                CK(mixed_zgemm(c.mx, c.st, k / 2));
        }
        CKS(mode_update(c, A, lam, k, safe, used_pinv));
    }
    if (eval_loss) {
        if (c.prec == THC_CPD_FP64) {
            loss_eval(c.st, c.s.Rt, c.s.R, c.Y, c.W[2], c.W[3], lam, c.G, c.red, c.sc, tol);
        } else {
            // the loss is a cancelling difference: FP64 projections and Z product
            for (int k = 0; k < 4; ++k) project_fp64(c, k, A[k], true);
            zgemm_fp64(c, 1, true);
            loss_eval(c.st, c.s.Rt, c.s.R, c.Y, c.W[2], c.W[3], lam, c.G, c.red, c.sc, tol);
        }
    }
    CK(cudaGetLastError());
    return THC_CPD_OK;
}

// One optimistic sweep, replayed from a CUDA graph when possible. The graph is captured
// on an internal non-blocking stream (the legacy default stream cannot be captured) and
// ordered after / before the caller's stream with events.
thc_cpd_status fast_sweep(Ctx& c, double* const A[4], double* lam, bool eval, double tol,
                          bool* use_graph) {
    NvtxRange nvtx_range("thc_cpd sweep (graph)");
    if (*use_graph) {
        const int gi = eval ? 1 : 0;
        if (c.gexec[gi] && c.gprec[gi] != c.prec) {
            cudaGraphExecDestroy(c.gexec[gi]);
            c.gexec[gi] = nullptr;
        }
        if (!c.gst) {
            if (cudaStreamCreateWithFlags(&c.gst, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&c.ev_in, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&c.ev_out, cudaEventDisableTiming) != cudaSuccess) {
                *use_graph = false;
                cudaGetLastError();
            }
        }
        if (*use_graph && !c.gexec[gi]) {
            cudaStream_t caller = c.st;
            c.st = c.gst;
            const long l0 = thc_cpd_launch_count();
            cudaGraph_t graph = nullptr;
            bool ok = cudaStreamBeginCapture(c.gst, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            int used = 0;
            thc_cpd_status st = ok ? sweep(c, A, lam, false, eval, tol, &used) : THC_CPD_ERR_CUDA;
            if (ok) ok = cudaStreamEndCapture(c.gst, &graph) == cudaSuccess && st == THC_CPD_OK;
            if (ok) ok = cudaGraphInstantiate(&c.gexec[gi], graph, 0) == cudaSuccess;
            if (graph) cudaGraphDestroy(graph);
            c.st = caller;
            c.glaunch[gi] = thc_cpd_launch_count() - l0;
            c.gprec[gi] = c.prec;
            if (!ok) {
                if (c.gexec[gi]) cudaGraphExecDestroy(c.gexec[gi]);
                c.gexec[gi] = nullptr;
                *use_graph = false;
                cudaGetLastError();  // clear a capture error; run the sweep directly
            }
        }
        if (*use_graph) {
            CK(cudaEventRecord(c.ev_in, c.st));
            CK(cudaStreamWaitEvent(c.gst, c.ev_in, 0));
            CK(cudaGraphLaunch(c.gexec[gi], c.gst));
            CK(cudaEventRecord(c.ev_out, c.gst));
            CK(cudaStreamWaitEvent(c.st, c.ev_out, 0));
            count_launch((int)c.glaunch[gi]);
            return THC_CPD_OK;
        }
    }
    int used = 0;
    return sweep(c, A, lam, false, eval, tol, &used);
}

thc_cpd_status read_scalars(Ctx& c, DevScalars* out) {
    DevScalars* h = host_scalars();
    if (!h) return set_err(THC_CPD_ERR_ALLOC, "pinned host buffer allocation failed");
    CK(cudaMemcpyAsync(h, c.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c.st));
    CK(cudaStreamSynchronize(c.st));
    *out = *h;
    return THC_CPD_OK;
}

thc_cpd_status obtain_norm(Ctx& c, double normG2, double* out) {
    if (normG2 > 0.0) {
        scalars_init(c.st, c.sc, normG2);
        *out = normG2;
        return THC_CPD_OK;
    }
    scalars_init(c.st, c.sc, 0.0);
    compute_normG2(c);
    DevScalars h;
    CKS(read_scalars(c, &h));
    *out = h.normG2;
    if (!isfinite(h.normG2) || !(h.normG2 > 0.0))
        return set_err(THC_CPD_ERR_NONFINITE, "||G||^2 = %g is not a positive finite number", h.normG2);
    return THC_CPD_OK;
}

// ---- learned extrapolation -------------------------------------------------------------
// After each plain ALS sweep: per-mode change norms of the lam-absorbed factors, the 40
// history features, the network's step factor alpha, the trial point
// T = P + alpha (N - P) (P: previous point, N: the ALS point), its exact FP64 loss, and
// acceptance iff that loss is below the ALS point's. In recording mode the exact losses
// of trial points on a grid of alpha are stored instead and the plain trajectory is kept.
struct LearnArgs {
    const float* mlp = nullptr;     // network parameters (device) or NULL
    const double* alphas = nullptr; // recording: alpha grid (host)
    int nalpha = 0;
    float* feats = nullptr;         // recording: features per sweep (host, 40 each)
    double* tloss = nullptr;        // recording: trial losses per sweep (host, nalpha each)
    int accepted = 0;               // out: accepted extrapolations
};

struct LearnWs {
    double* T[4] = {};
    double* lamk[4] = {};
    double* lamT = nullptr;
    double* Wtr[4] = {};
    double* Gtr[4] = {};
    double* Ytr = nullptr;
    double* red = nullptr;
    double* chg = nullptr;  // 8 doubles: (num, den) per mode
    float* feat = nullptr;
    float* alpha = nullptr;
    DevScalars* sc = nullptr;
    void* block = nullptr;
    cudaStream_t st = nullptr;
    ~LearnWs() {
        if (block) cudaFreeAsync(block, st);
    }
};

thc_cpd_status learn_init(Ctx& c, LearnWs& L) {
    const int Rt = c.s.Rt, R = c.s.R;
    size_t b = 0;
    for (int k = 0; k < 4; ++k) b += Arena::need<double>((size_t)c.s.n[k] * R);
    b += 5 * Arena::need<double>(R) + 5 * Arena::need<double>((size_t)Rt * R) +
         4 * Arena::need<double>((size_t)R * R) + Arena::need<double>(256) + Arena::need<double>(8) +
         Arena::need<float>(64) + Arena::need<DevScalars>(1);
    L.st = c.st;
    CK(cudaMallocAsync(&L.block, b, c.st));
    Arena ar;
    ar.base = (char*)L.block;
    for (int k = 0; k < 4; ++k) L.T[k] = ar.take<double>((size_t)c.s.n[k] * R);
    for (int k = 0; k < 4; ++k) L.lamk[k] = ar.take<double>(R);
    L.lamT = ar.take<double>(R);
    for (int k = 0; k < 4; ++k) L.Wtr[k] = ar.take<double>((size_t)Rt * R);
    L.Ytr = ar.take<double>((size_t)Rt * R);
    for (int k = 0; k < 4; ++k) L.Gtr[k] = ar.take<double>((size_t)R * R);
    L.red = ar.take<double>(256);
    L.chg = ar.take<double>(8);
    L.feat = ar.take<float>(48);
    L.alpha = L.feat + 40;
    L.sc = ar.take<DevScalars>(1);
    return THC_CPD_OK;
}

// 40 features from the histories, most recent first (same formula as the oracle's)
void make_features(const std::vector<double>& loss_hist, const std::vector<std::array<double, 4>>& chg,
                   float* f) {
    for (int i = 0; i < 40; ++i) f[i] = 0.f;
    const int nl = (int)loss_hist.size();
    for (int i = 0; i < 8; ++i) {
        const int s = nl - 1 - i;
        if (s >= 1) {
            const double d = log(loss_hist[s - 1]) - log(loss_hist[s]);
            f[i] = (float)(log10(std::max(d, 1e-12)) / 6.0);
        }
    }
    const int nc = (int)chg.size();
    for (int i = 0; i < 8; ++i) {
        const int s = nc - 1 - i;
        if (s >= 0)
            for (int k = 0; k < 4; ++k) f[8 + 4 * i + k] = (float)(log10(std::max(chg[s][k], 1e-12)) / 6.0);
    }
}

// exact FP64 loss of the trial factors T with weights lamT (W, G, Y into the trial buffers)
thc_cpd_status trial_loss(Ctx& c, LearnWs& L, double* loss) {
    const int Rt = c.s.Rt, R = c.s.R;
    for (int k = 0; k < 4; ++k) {
        gemm64(c, true, Rt, R, c.s.n[k], c.X[k], Rt, L.T[k], nullptr, R, L.Wtr[k], R, false);
        gemm64(c, true, R, R, c.s.n[k], L.T[k], R, L.T[k], nullptr, R, L.Gtr[k], R, true);
    }
    gemm64(c, true, Rt, R, Rt, c.Z, Rt, L.Wtr[0], L.Wtr[1], R, L.Ytr, R, false);
    CK(cudaMemcpyAsync(L.sc, c.sc, sizeof(DevScalars), cudaMemcpyDeviceToDevice, c.st));
    loss_eval(c.st, Rt, R, L.Ytr, L.Wtr[2], L.Wtr[3], L.lamT, L.Gtr, c.red, L.sc, 0.0);
    DevScalars* h = host_scalars();
    if (!h) return set_err(THC_CPD_ERR_ALLOC, "pinned host buffer allocation failed");
    CK(cudaMemcpyAsync(h, L.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c.st));
    CK(cudaStreamSynchronize(c.st));
    *loss = h->loss;
    return THC_CPD_OK;
}

// build T = P + alpha (N - P) and its column normalisation (lamT = product of the norms)
void build_trial(Ctx& c, LearnWs& L, double* const A[4], const double* lam, double alpha) {
    const int R = c.s.R;
    for (int k = 0; k < 4; ++k) {
        trial_point(c.st, c.s.n[k], R, A[k], c.Asnap[k], lam, c.lamsnap, k == 3, alpha, L.T[k]);
        normalise_columns(c.st, c.s.n[k], R, L.T[k], L.lamk[k], L.lamT);
    }
    const double* lk[4] = {L.lamk[0], L.lamk[1], L.lamk[2], L.lamk[3]};
    lam_product(c.st, R, lk, L.lamT);
}

// Rollback snapshot: point the snapshot at slot b, copy the state (factors, lam, scalars)
// there in one launch; and the way back.
void use_snapshot_slot(Ctx& c, int b) {
    for (int k = 0; k < 4; ++k) c.Asnap[k] = c.Asnap_slot[b][k];
    c.lamsnap = c.lamsnap_slot[b];
    c.sc_snap = c.sc_slot[b];
}

thc_cpd_status take_snapshot(Ctx& c, double* const A[4], const double* lam) {
    static_assert(sizeof(DevScalars) % sizeof(double) == 0, "DevScalars in doubles");
    const int R = c.s.R;
    const double* src[6] = {A[0], A[1], A[2], A[3], lam, (const double*)c.sc};
    double* dst[6] = {c.Asnap[0], c.Asnap[1], c.Asnap[2], c.Asnap[3], c.lamsnap, (double*)c.sc_snap};
    const long len[6] = {(long)c.s.n[0] * R, (long)c.s.n[1] * R, (long)c.s.n[2] * R,
                         (long)c.s.n[3] * R, (long)R, (long)(sizeof(DevScalars) / sizeof(double))};
    CK(copy_many(c.st, 6, src, dst, len));
    return THC_CPD_OK;
}

thc_cpd_status restore_snapshot(Ctx& c, double* const A[4], double* lam) {
    const int R = c.s.R;
    for (int k = 0; k < 4; ++k)
        CK(cudaMemcpyAsync(A[k], c.Asnap[k], sizeof(double) * c.s.n[k] * R, cudaMemcpyDeviceToDevice,
                           c.st));
    CK(cudaMemcpyAsync(lam, c.lamsnap, sizeof(double) * R, cudaMemcpyDeviceToDevice, c.st));
    CK(cudaMemcpyAsync(c.sc, c.sc_snap, sizeof(DevScalars), cudaMemcpyDeviceToDevice, c.st));
    return THC_CPD_OK;
}

// The ALS driver shared by thc_cpd_als, thc_cpd_als_sweep and the trajectory recorder.
thc_cpd_status run_als(int o, int v, int Rt, int R, const double* Xo, const double* Xv,
                       const double* Z, double* const A[4], double* lam, int max_sweeps,
                       double tol, double normG2, int* sweeps_done, double* loss_host,
                       double* fit_host, thc_cpd_opts* opts, LearnArgs* la = nullptr) {
    NvtxRange nvtx_range("thc_cpd_als");
    Shape s;
    CKS(check_shape(o, v, Rt, R, &s));
    CKS(check_ptrs(Xo, Xv, Z, A));
    CKS(check_prec(opts));
    if (!lam) return set_err(THC_CPD_ERR_ARG, "lam must be non-null");
    if (max_sweeps < 0) return set_err(THC_CPD_ERR_ARG, "max_sweeps must be >= 0");
    if (opts) opts->flags_out = 0;
    Ctx c;
    CKS(ctx_init(c, s, Xo, Xv, Z, opts, NEED_ALS | (normG2 > 0.0 ? 0u : NEED_NORM)));
    double nG2 = 0.0;
    CKS(obtain_norm(c, normG2, &nG2));
    refresh_state(c, A);
    const bool learning = la && (la->mlp || la->nalpha > 0);
    LearnWs L;
    std::vector<double> loss_hist;
    std::vector<std::array<double, 4>> chg_hist;
    if (learning) {
        CKS(learn_init(c, L));
        // loss of the start point (history entry L_0)
        for (int k = 0; k < 4; ++k) CK(cudaMemcpyAsync(L.T[k], A[k], sizeof(double) * s.n[k] * R,
                                                       cudaMemcpyDeviceToDevice, c.st));
        CK(cudaMemcpyAsync(L.lamT, lam, sizeof(double) * R, cudaMemcpyDeviceToDevice, c.st));
        double l0;
        CKS(trial_loss(c, L, &l0));
        loss_hist.push_back(l0);
    }
    const int loss_every = (opts && opts->loss_every > 0) ? opts->loss_every : 0;
    const double target = (opts && opts->target_fit > 0.0) ? opts->target_fit : 0.0;
    const int polish = (opts && opts->polish_sweeps > 0 && tol <= 0.0) ? opts->polish_sweeps : 0;
    const bool split_run = c.prec != THC_CPD_FP64;
    int flags = 0;
    int done_sweeps = 0;
    DevScalars h;
    h.loss = nan("");
    h.fit = nan("");
    double fit1 = nan(""), fit2 = nan("");  // fits of the last two evaluated sweeps
    bool use_graph = !prof_on() && getenv("THC_CPD_NO_GRAPH") == nullptr;
    const bool tune = opts && opts->autotune && split_run;
    // Fixed-length runs (tol <= 0: no convergence stop; the FP64 hand-over at a known sweep)
    // are pipelined: sweep s+1 is queued before the host reads sweep s's scalars, so the GPU
    // does not idle for the round trip. The state before each sweep goes to the snapshot
    // slot of its parity; if sweep s reports a failed pivot, the speculative sweep s+1 is
    // undone with sweep s's own rollback and sweep s is replayed exactly as below.
    DevScalars* hs2 = host_scalar_slots();
    const bool pipe = use_graph && !learning && !tune && tol <= 0.0 && max_sweeps >= 2 && hs2;
    if (pipe) {
        for (int b = 0; b < 2; ++b)
            if (!c.ev_sc[b]) CK(cudaEventCreateWithFlags(&c.ev_sc[b], cudaEventDisableTiming));
        bool evals[2] = {false, false};
        auto hand_over_at = [&](int sw) {
            return split_run && c.prec != THC_CPD_FP64 && polish > 0 && sw > max_sweeps - polish;
        };
        auto launch = [&](int sw) -> thc_cpd_status {
            if (hand_over_at(sw)) {
                c.prec = THC_CPD_FP64;
                refresh_state(c, A);
                flags |= 4;
            }
            bool eval = true;
            if (c.prec != THC_CPD_FP64 && !(target > 0.0 && loss_every == 0))
                eval = (loss_every > 0 && sw % loss_every == 0) || sw == max_sweeps;
            const int b = sw & 1;
            use_snapshot_slot(c, b);
            CKS(take_snapshot(c, A, lam));
            CKS(fast_sweep(c, A, lam, eval, tol, &use_graph));
            CK(cudaMemcpyAsync(hs2 + b, c.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c.st));
            CK(cudaEventRecord(c.ev_sc[b], c.st));
            evals[b] = eval;
            return THC_CPD_OK;
        };
        CKS(launch(1));
        int next = 2;  // the next sweep to queue
        for (int sw = 1; sw <= max_sweeps; ++sw) {
            const int b = sw & 1;
            // queue sweep sw + 1 unless it starts the FP64 phase (that refreshes the state
            // from the factors, which must be final)
            bool spec = false;
            if (next == sw + 1 && sw + 1 <= max_sweeps && !hand_over_at(sw + 1)) {
                CKS(launch(sw + 1));
                next = sw + 2;
                spec = true;
            }
            CK(cudaEventSynchronize(c.ev_sc[b]));
            h = hs2[b];
            const bool eval = evals[b];
            int used = 0;
            if (h.fail_mask) {
                // undo the speculative sweep, then roll back and replay sweep sw with a host
                // check after every factorisation
                CK(cudaStreamSynchronize(c.st));
                use_snapshot_slot(c, b);
                CKS(restore_snapshot(c, A, lam));
                refresh_state(c, A);
                CKS(ctx_safe_buffers(c));
                CKS(sweep(c, A, lam, true, eval, tol, &used));
                CKS(read_scalars(c, &h));
                flags |= 2;
                next = sw + 1;
                spec = false;
            }
            if (used) flags |= 1;
            done_sweeps = sw;
            if (opts && opts->history) {
                opts->history[2 * (sw - 1)] = eval ? h.loss : nan("");
                opts->history[2 * (sw - 1) + 1] = eval ? h.fit : nan("");
            }
            if (eval && (h.nonfinite || !isfinite(h.loss))) {
                if (spec) {  // leave the factors as sweep sw made them
                    CK(cudaStreamSynchronize(c.st));
                    use_snapshot_slot(c, (sw + 1) & 1);
                    CKS(restore_snapshot(c, A, lam));
                    CK(cudaStreamSynchronize(c.st));
                }
                if (opts) opts->flags_out = flags;
                if (sweeps_done) *sweeps_done = done_sweeps;
                return set_err(THC_CPD_ERR_NONFINITE, "loss became non-finite at sweep %d", sw);
            }
            if (target > 0.0 && eval && h.fit >= target) {
                if (spec) {  // undo the queued sweep sw + 1: the run ends at sweep sw
                    CK(cudaStreamSynchronize(c.st));
                    use_snapshot_slot(c, (sw + 1) & 1);
                    CKS(restore_snapshot(c, A, lam));
                }
                break;
            }
            if (next == sw + 1 && sw + 1 <= max_sweeps) {
                CKS(launch(sw + 1));
                next = sw + 2;
            }
        }
    }
    for (int sw = 1; sw <= max_sweeps && !pipe; ++sw) {
        if (tune) tc_set_tuning(sw == 1);
        // split precision hands over to FP64 sweeps (polish) near convergence or for the
        // last polish_sweeps of a fixed-length run
        if (split_run && c.prec != THC_CPD_FP64 &&
            ((polish > 0 && sw > max_sweeps - polish) ||
             (tol > 0.0 && isfinite(fit1) && isfinite(fit2) && fabs(fit1 - fit2) < 10.0 * tol))) {
            c.prec = THC_CPD_FP64;
            refresh_state(c, A);
            flags |= 4;
        }
        bool eval = true;
        if (c.prec != THC_CPD_FP64 && !learning) {
            if (loss_every > 0)
                eval = (sw % loss_every == 0) || sw == max_sweeps;
            else
                eval = tol > 0.0 || target > 0.0 || sw == max_sweeps;
        }
        CKS(take_snapshot(c, A, lam));  // the state before this sweep, for a rollback
        int used = 0;
        if (tune && sw == 1) {
            CKS(sweep(c, A, lam, false, eval, tol, &used));  // tuned on live operands
            tc_set_tuning(false);
        } else {
            CKS(fast_sweep(c, A, lam, eval, tol, &use_graph));
        }
        CKS(read_scalars(c, &h));
        if (h.fail_mask) {
            // a Cholesky pivot failed somewhere in this sweep: roll back and replay the
            // sweep with a host check after every factorisation
            CKS(restore_snapshot(c, A, lam));
            refresh_state(c, A);
            CKS(ctx_safe_buffers(c));
            CKS(sweep(c, A, lam, true, eval, tol, &used));
            CKS(read_scalars(c, &h));
            flags |= 2;
        }
        if (used) flags |= 1;
        done_sweeps = sw;
        if (learning) {
            // change norms between the previous point (snapshot) and the ALS point
            std::array<double, 4> ch;
            double hc[8];
            for (int k = 0; k < 4; ++k)
                change_norm(c.st, s.n[k], R, A[k], c.Asnap[k], lam, c.lamsnap, k == 3, L.red, L.chg + 2 * k);
            CK(cudaMemcpyAsync(hc, L.chg, sizeof(hc), cudaMemcpyDeviceToHost, c.st));
            CK(cudaStreamSynchronize(c.st));
            for (int k = 0; k < 4; ++k) ch[k] = hc[2 * k + 1] > 0 ? sqrt(hc[2 * k] / hc[2 * k + 1]) : 0.0;
            chg_hist.push_back(ch);
            std::vector<double> lh = loss_hist;
            lh.push_back(h.loss);
            float f[40];
            make_features(lh, chg_hist, f);
            if (la->nalpha > 0) {
                // recording: exact losses of the trial points on the alpha grid
                if (la->feats) memcpy(la->feats + (size_t)40 * (sw - 1), f, sizeof f);
                for (int a = 0; a < la->nalpha; ++a) {
                    double tl = h.loss;
                    if (la->alphas[a] != 1.0) {
                        build_trial(c, L, A, lam, la->alphas[a]);
                        CKS(trial_loss(c, L, &tl));
                    }
                    if (la->tloss) la->tloss[(size_t)la->nalpha * (sw - 1) + a] = tl;
                }
                loss_hist.push_back(h.loss);
            } else {
                CK(cudaMemcpyAsync(L.feat, f, sizeof f, cudaMemcpyHostToDevice, c.st));
                mlp_forward1(c.st, la->mlp, L.feat, L.alpha);
                float ha = 1.f;
                CK(cudaMemcpyAsync(&ha, L.alpha, sizeof(float), cudaMemcpyDeviceToHost, c.st));
                CK(cudaStreamSynchronize(c.st));
                bool accepted = false;
                if (sw >= 2 && ha > 1.02f && isfinite(ha)) {
                    build_trial(c, L, A, lam, (double)ha);
                    double tl;
                    CKS(trial_loss(c, L, &tl));
                    if (tl < h.loss) {
                        // accept: the trial becomes the current point, with its state
                        for (int k = 0; k < 4; ++k) {
                            CK(cudaMemcpyAsync(A[k], L.T[k], sizeof(double) * s.n[k] * R,
                                               cudaMemcpyDeviceToDevice, c.st));
                            CK(cudaMemcpyAsync(c.G[k], L.Gtr[k], sizeof(double) * R * R,
                                               cudaMemcpyDeviceToDevice, c.st));
                            if (c.prec == THC_CPD_FP64)
                                CK(cudaMemcpyAsync(c.W[k], L.Wtr[k], sizeof(double) * Rt * R,
                                                   cudaMemcpyDeviceToDevice, c.st));
                        }
                        CK(cudaMemcpyAsync(lam, L.lamT, sizeof(double) * R, cudaMemcpyDeviceToDevice, c.st));
                        if (c.prec != THC_CPD_FP64)
                            for (int k = 0; k < 4; ++k) CK(mixed_project(c.mx, c.st, k, A[k], false));
                        CK(cudaMemcpyAsync(c.sc, L.sc, sizeof(DevScalars), cudaMemcpyDeviceToDevice, c.st));
                        DevScalars* hs = host_scalars();
                        CK(cudaMemcpyAsync(hs, L.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c.st));
                        CK(cudaStreamSynchronize(c.st));
                        h.loss = hs->loss;
                        h.fit = hs->fit;
                        accepted = true;
                        la->accepted++;
                    }
                }
                loss_hist.push_back(h.loss);
                // convergence decided on the host from the accepted points' fits
                h.done = (tol > 0.0 && isfinite(fit1) && fabs(h.fit - fit1) < tol) ? 1 : 0;
                (void)accepted;
            }
        }
        if (eval) {
            fit2 = fit1;
            fit1 = h.fit;
        }
        if (opts && opts->history) {
            opts->history[2 * (sw - 1)] = eval ? h.loss : nan("");
            opts->history[2 * (sw - 1) + 1] = eval ? h.fit : nan("");
        }
        if (eval && (h.nonfinite || !isfinite(h.loss))) {
            if (opts) opts->flags_out = flags;
            if (sweeps_done) *sweeps_done = done_sweeps;
            return set_err(THC_CPD_ERR_NONFINITE, "loss became non-finite at sweep %d", sw);
        }
        if (target > 0.0 && eval && h.fit >= target) break;
        // a split-precision run that meets tol (|dfit| fell below 10 tol and tol in one
        // sweep) still ends with FP64 sweeps: the hand-over above fires next sweep
        if (h.done && !(split_run && c.prec != THC_CPD_FP64)) break;
    }
    if (opts) opts->flags_out = flags;
    if (sweeps_done) *sweeps_done = done_sweeps;
    if (loss_host) *loss_host = h.loss;
    if (fit_host) *fit_host = h.fit;
    CK(cudaStreamSynchronize(c.st));
    CKS(kernel_errors(c.prec != THC_CPD_FP64));
    return THC_CPD_OK;
}


// ---- batched driver -------------------------------------------------------------------
// Every problem has its own Ctx and stream; one sweep of all running problems is captured
// as one CUDA graph (fork from a capture stream, one branch per problem, join) and
// replayed per sweep. The device scalars of all problems live in one array so that a
// single copy per sweep brings back every problem's loss, fit and failure flags.
thc_cpd_status run_batched(int np, thc_cpd_problem* P, int max_sweeps, double tol,
                           thc_cpd_opts* opts) {
    if (np < 1 || !P) return set_err(THC_CPD_ERR_ARG, "need at least one problem");
    if (max_sweeps < 0) return set_err(THC_CPD_ERR_ARG, "max_sweeps must be >= 0");
    CKS(check_prec(opts));
    std::vector<Shape> shp(np);
    for (int p = 0; p < np; ++p) {
        CKS(check_shape(P[p].o, P[p].v, P[p].Rt, P[p].R, &shp[p]));
        CKS(check_ptrs(P[p].Xo, P[p].Xv, P[p].Z, P[p].A));
        if (!P[p].lam) return set_err(THC_CPD_ERR_ARG, "problem %d: lam must be non-null", p);
        P[p].sweeps_done = 0;
        P[p].flags_out = 0;
        P[p].loss = P[p].fit = nan("");
    }
    if (opts) opts->flags_out = 0;
    const cudaStream_t caller = stream_of(opts);
    const int prec = opts ? opts->precision : THC_CPD_FP64;
    struct Res {
        std::vector<cudaStream_t> streams;
        std::vector<cudaEvent_t> events;
        std::vector<std::unique_ptr<Ctx>> ctx;
        cudaStream_t cap = nullptr;
        cudaGraphExec_t exec[2] = {nullptr, nullptr};
        DevScalars* dsc = nullptr;
        DevScalars* hsc = nullptr;
        cudaStream_t free_on = nullptr;
        ~Res() {
            for (auto& e : exec)
                if (e) cudaGraphExecDestroy(e);
            ctx.clear();  // frees workspaces on their streams
            if (dsc) cudaFreeAsync(dsc, free_on);
            if (hsc) cudaFreeHost(hsc);
            for (auto e : events) cudaEventDestroy(e);
            for (auto s : streams) cudaStreamDestroy(s);
            if (cap) cudaStreamDestroy(cap);
        }
    } r;
    r.free_on = caller;
    CK(cudaStreamCreateWithFlags(&r.cap, cudaStreamNonBlocking));
    r.streams.resize(np);
    for (int p = 0; p < np; ++p) CK(cudaStreamCreateWithFlags(&r.streams[p], cudaStreamNonBlocking));
    r.events.resize(np + 2);
    for (auto& e : r.events) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaEvent_t ev_fork = r.events[np], ev_done = r.events[np + 1];
    // order everything after the caller's prior work
    CK(cudaEventRecord(ev_fork, caller));
    CK(cudaStreamWaitEvent(r.cap, ev_fork, 0));
    for (int p = 0; p < np; ++p) CK(cudaStreamWaitEvent(r.streams[p], ev_fork, 0));
    CK(cudaMallocAsync((void**)&r.dsc, sizeof(DevScalars) * 2 * np, caller));
    CK(cudaMallocHost((void**)&r.hsc, sizeof(DevScalars) * np));
    CK(cudaStreamSynchronize(caller));
    r.ctx.resize(np);
    for (int p = 0; p < np; ++p) {
        r.ctx[p] = std::make_unique<Ctx>();
        thc_cpd_opts o2 = opts ? *opts : thc_cpd_opts{};
        o2.stream = r.streams[p];
        Ctx& c = *r.ctx[p];
        CKS(ctx_init(c, shp[p], P[p].Xo, P[p].Xv, P[p].Z, &o2, NEED_ALS | NEED_NORM | NEED_BATCHED));
        c.sc = r.dsc + p;
        c.sc_snap = r.dsc + np + p;
        double nG2;
        CKS(obtain_norm(c, 0.0, &nG2));
        refresh_state(c, P[p].A);
    }
    for (int p = 0; p < np; ++p) CK(cudaStreamSynchronize(r.streams[p]));
    std::vector<int> active(np);
    for (int p = 0; p < np; ++p) active[p] = p;
    bool graph_ok[2] = {false, false};
    const bool use_graph = !prof_on() && getenv("THC_CPD_NO_GRAPH") == nullptr;
    const bool tune = opts && opts->autotune && prec != THC_CPD_FP64;
    int any_flags = 0;
    for (int sw = 1; sw <= max_sweeps && !active.empty(); ++sw) {
        const bool eval = prec == THC_CPD_FP64 || tol > 0.0 || sw == max_sweeps;
        const int gi = eval ? 1 : 0;
        auto enqueue_sweep = [&](int p) -> thc_cpd_status {
            Ctx& c = *r.ctx[p];
            for (int k = 0; k < 4; ++k)
                CK(cudaMemcpyAsync(c.Asnap[k], P[p].A[k], sizeof(double) * c.s.n[k] * c.s.R,
                                   cudaMemcpyDeviceToDevice, c.st));
            CK(cudaMemcpyAsync(c.lamsnap, P[p].lam, sizeof(double) * c.s.R, cudaMemcpyDeviceToDevice,
                               c.st));
            CK(cudaMemcpyAsync(c.sc_snap, c.sc, sizeof(DevScalars), cudaMemcpyDeviceToDevice, c.st));
            int used = 0;
            return sweep(c, P[p].A, P[p].lam, false, eval, tol, &used);
        };
        if (use_graph && !(tune && sw == 1)) {
            if (!graph_ok[gi]) {
                if (r.exec[gi]) cudaGraphExecDestroy(r.exec[gi]);
                r.exec[gi] = nullptr;
                const long l0 = thc_cpd_launch_count();
                cudaGraph_t g = nullptr;
                CK(cudaStreamBeginCapture(r.cap, cudaStreamCaptureModeThreadLocal));
                CK(cudaEventRecord(ev_fork, r.cap));
                thc_cpd_status st = THC_CPD_OK;
                for (int p : active) {
                    cudaStreamWaitEvent(r.streams[p], ev_fork, 0);
                    if (st == THC_CPD_OK) st = enqueue_sweep(p);
                    cudaEventRecord(r.events[p], r.streams[p]);
                    cudaStreamWaitEvent(r.cap, r.events[p], 0);
                }
                const cudaError_t ce = cudaStreamEndCapture(r.cap, &g);
                if (st != THC_CPD_OK) {
                    if (g) cudaGraphDestroy(g);
                    return st;
                }
                if (ce != cudaSuccess) return set_err(THC_CPD_ERR_CUDA, "batched capture failed: %s", cudaGetErrorString(ce));
                const cudaError_t ie = cudaGraphInstantiate(&r.exec[gi], g, 0);
                cudaGraphDestroy(g);
                if (ie != cudaSuccess) return set_err(THC_CPD_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ie));
                graph_ok[gi] = true;
                r.ctx[0]->glaunch[gi] = thc_cpd_launch_count() - l0;
            }
            CK(cudaGraphLaunch(r.exec[gi], r.cap));
            count_launch((int)r.ctx[0]->glaunch[gi]);
        } else {
            if (tune) tc_set_tuning(sw == 1);
            for (int p : active) {
                CK(cudaEventRecord(ev_fork, r.cap));
                CK(cudaStreamWaitEvent(r.streams[p], ev_fork, 0));
                CKS(enqueue_sweep(p));
                CK(cudaEventRecord(r.events[p], r.streams[p]));
                CK(cudaStreamWaitEvent(r.cap, r.events[p], 0));
            }
            if (tune) tc_set_tuning(false);
        }
        CK(cudaMemcpyAsync(r.hsc, r.dsc, sizeof(DevScalars) * np, cudaMemcpyDeviceToHost, r.cap));
        CK(cudaStreamSynchronize(r.cap));
        std::vector<int> still;
        for (int p : active) {
            DevScalars h = r.hsc[p];
            Ctx& c = *r.ctx[p];
            if (h.fail_mask) {
                // roll this problem back and replay its sweep with checked factorisations
                for (int k = 0; k < 4; ++k)
                    CK(cudaMemcpyAsync(P[p].A[k], c.Asnap[k], sizeof(double) * c.s.n[k] * c.s.R,
                                       cudaMemcpyDeviceToDevice, c.st));
                CK(cudaMemcpyAsync(P[p].lam, c.lamsnap, sizeof(double) * c.s.R,
                                   cudaMemcpyDeviceToDevice, c.st));
                CK(cudaMemcpyAsync(c.sc, c.sc_snap, sizeof(DevScalars), cudaMemcpyDeviceToDevice, c.st));
                refresh_state(c, P[p].A);
                CKS(ctx_safe_buffers(c));
                int used = 0;
                CKS(sweep(c, P[p].A, P[p].lam, true, eval, tol, &used));
                CKS(read_scalars(c, &h));
                P[p].flags_out |= 2 | (used ? 1 : 0);
                r.hsc[p] = h;
            }
            P[p].sweeps_done = sw;
            if (eval) {
                P[p].loss = h.loss;
                P[p].fit = h.fit;
                if (h.nonfinite || !isfinite(h.loss))
                    return set_err(THC_CPD_ERR_NONFINITE, "problem %d: loss became non-finite at sweep %d", p, sw);
            }
            any_flags |= P[p].flags_out;
            if (h.done)
                graph_ok[0] = graph_ok[1] = false;  // re-capture without it
            else
                still.push_back(p);
        }
        active.swap(still);
    }
    // the caller's stream waits for everything
    CK(cudaEventRecord(ev_done, r.cap));
    for (int p = 0; p < np; ++p) {
        CK(cudaEventRecord(r.events[p], r.streams[p]));
        CK(cudaStreamWaitEvent(caller, r.events[p], 0));
    }
    CK(cudaStreamWaitEvent(caller, ev_done, 0));
    CK(cudaStreamSynchronize(caller));
    if (opts) opts->flags_out = any_flags;
    CKS(kernel_errors(prec != THC_CPD_FP64));
    return THC_CPD_OK;
}

}  // namespace

namespace thc {
int set_error(int s, const char* msg) {
    g_err = msg;
    return s;
}

int check_problem_args(int o, int v, int Rt, int R, const double* Xo, const double* Xv,
                       const double* Z, const double* const* A) {
    Shape s;
    CKS(check_shape(o, v, Rt, R, &s));
    if (!A) return set_err(THC_CPD_ERR_ARG, "A must be non-null");
    CKS(check_ptrs(Xo, Xv, Z, A));
    return THC_CPD_OK;
}

int check_mttkrp_args(int o, int v, int Rt, int R, const double* Xo, const double* Xv,
                      const double* Z, const double* const* A, int mode, const double* M) {
    Shape s;
    CKS(check_shape(o, v, Rt, R, &s));
    if (!A) return set_err(THC_CPD_ERR_ARG, "A must be non-null");
    CKS(check_ptrs(Xo, Xv, Z, A));
    if (mode < 0 || mode > 3) return set_err(THC_CPD_ERR_ARG, "mode must be 0..3, got %d", mode);
    if (!M) return set_err(THC_CPD_ERR_ARG, "M must be non-null");
    return THC_CPD_OK;
}
}  // namespace thc

extern "C" {

const char* thc_cpd_last_error(void) { return g_err.c_str(); }

const char* thc_cpd_version(void) { return "thc_cpd 0.1 (sm_103a)"; }

thc_cpd_status thc_cpd_thc_norm2(int o, int v, int Rt, const double* Xo, const double* Xv,
                                 const double* Z, double* normG2_host, const thc_cpd_opts* opts) {
    Shape s;
    CKS(check_shape(o, v, Rt, 1, &s));
    CKS(check_ptrs(Xo, Xv, Z, nullptr));
    if (!normG2_host) return set_err(THC_CPD_ERR_ARG, "normG2_host must be non-null");
    thc_cpd_opts o2 = opts ? *opts : thc_cpd_opts{};
    o2.precision = THC_CPD_FP64;
    Ctx c;
    CKS(ctx_init(c, s, Xo, Xv, Z, &o2, NEED_NORM));
    return obtain_norm(c, 0.0, normG2_host);
}

thc_cpd_status thc_cpd_mttkrp(int o, int v, int Rt, int R, const double* Xo, const double* Xv,
                              const double* Z, const double* const A[4], int mode, double* M,
                              const thc_cpd_opts* opts) {
    NvtxRange nvtx_range("thc_cpd_mttkrp");
    Shape s;
    CKS((thc_cpd_status)check_mttkrp_args(o, v, Rt, R, Xo, Xv, Z, A, mode, M));
    CKS(check_shape(o, v, Rt, R, &s));
    CKS(check_prec(opts));
    Ctx c;
    CKS(ctx_init(c, s, Xo, Xv, Z, opts, 0));
    if (c.prec == THC_CPD_FP64) {
        for (int k = 0; k < 4; ++k)
            if (k != mode) project_fp64(c, k, A[k]);
        zgemm_fp64(c, mode / 2);
        backproject_fp64(c, mode, M);
    } else {
        // projections of the three other modes; their epilogues leave the Hadamard
        // operand of the Z-GEMM (P) in place, the Z-GEMM epilogue the one of modes 0/2
        // the Hadamard operand P of the wanted half must be written last:
        // half 0 needs P34 (from mode 3), half 1 needs P12 (from mode 1)
        static const int order[2][4] = {{0, 1, 2, 3}, {3, 0, 1, 2}};
        for (int i = 0; i < 4; ++i) {
            const int k = order[mode / 2][i];
            if (k != mode) CK(mixed_project(c.mx, c.st, k, A[k], false));
        }
        CK(mixed_zgemm(c.mx, c.st, mode / 2));
        if (mode == 1 || mode == 3) CK(mixed_partner(c.mx, c.st, mode));
        CK(mixed_backproject(c.mx, c.st, mode, M));
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c.st));
    if (int e = mixed_take_error())
        return set_err(THC_CPD_ERR_TIMEOUT, "tensor-core kernel wait gave up (code %d)", e);
    return THC_CPD_OK;
}

thc_cpd_status thc_cpd_split_gemm(int M, int N, int K, const double* A, const double* B, double* C,
                                  const thc_cpd_opts* opts) {
    if (M < 1 || N < 1 || K < 1 || (long)M * K >= 0x7fffffffL || (long)N * K >= 0x7fffffffL ||
        (long)M * N >= 0x7fffffffL)
        return set_err(THC_CPD_ERR_SHAPE, "bad GEMM shape %d x %d x %d", M, N, K);
    if (!A || !B || !C) return set_err(THC_CPD_ERR_ARG, "A, B and C must be non-null");
    CKS(check_prec(opts));
    const int prec = opts ? opts->precision : THC_CPD_FP64;
    if (prec == THC_CPD_FP64) return set_err(THC_CPD_ERR_ARG, "split GEMM needs a split precision");
    const bool tf32 = prec == THC_CPD_TF32X3;
    cudaStream_t st = stream_of(opts);
    const int esz = tf32 ? 4 : 2, pitch = split_pitch(tf32, K);
    const size_t a = Arena::need<uint8_t>((size_t)M * pitch * esz);
    const size_t b = Arena::need<uint8_t>((size_t)N * pitch * esz);
    void* block = nullptr;
    CK(cudaMallocAsync(&block, 2 * a + 2 * b, st));
    Arena ar;
    ar.base = (char*)block;
    SplitMat sa, sb;
    sa.hi = ar.take<uint8_t>((size_t)M * pitch * esz);
    sa.lo = ar.take<uint8_t>((size_t)M * pitch * esz);
    sb.hi = ar.take<uint8_t>((size_t)N * pitch * esz);
    sb.lo = ar.take<uint8_t>((size_t)N * pitch * esz);
    sa.rows = M; sb.rows = N;
    sa.cols = sb.cols = K;
    sa.pitch = sb.pitch = pitch;
    split_rows(st, tf32, A, K, M, K, sa);
    split_rows(st, tf32, B, K, N, K, sb);
    TcEpilogue ep;
    ep.out_f64t = C;  // D'[n][m] = B[n] . A[m] stored transposed: C[m][n]
    ep.ld_f64t = N;
    cudaError_t e = tc_gemm(st, tf32, sb, sa, N, M, K, ep);
    cudaFreeAsync(block, st);
    CK(e);
    CK(cudaStreamSynchronize(st));
    if (int te = mixed_take_error())
        return set_err(THC_CPD_ERR_TIMEOUT, "tensor-core kernel wait gave up (code %d)", te);
    return THC_CPD_OK;
}

thc_cpd_status thc_cpd_loss(int o, int v, int Rt, int R, const double* Xo, const double* Xv,
                            const double* Z, const double* const A[4], const double* lam,
                            double normG2, double* loss_host, double* fit_host,
                            const thc_cpd_opts* opts) {
    NvtxRange nvtx_range("thc_cpd_loss");
    Shape s;
    CKS(check_shape(o, v, Rt, R, &s));
    CKS(check_ptrs(Xo, Xv, Z, A));
    thc_cpd_opts o2 = opts ? *opts : thc_cpd_opts{};
    o2.precision = THC_CPD_FP64;  // the loss is always evaluated in FP64
    Ctx c;
    CKS(ctx_init(c, s, Xo, Xv, Z, &o2, normG2 > 0.0 ? 0u : NEED_NORM));
    double nG2;
    CKS(obtain_norm(c, normG2, &nG2));
    for (int k = 0; k < 4; ++k) {
        project_fp64(c, k, A[k]);
        gram_fp64(c, k, A[k]);
    }
    zgemm_fp64(c, 1);
    loss_eval(c.st, Rt, R, c.Y, c.W[2], c.W[3], lam ? lam : c.ones, c.G, c.red, c.sc, 0.0);
    DevScalars h;
    CKS(read_scalars(c, &h));
    if (loss_host) *loss_host = h.loss;
    if (fit_host) *fit_host = h.fit;
    if (!isfinite(h.loss)) return set_err(THC_CPD_ERR_NONFINITE, "loss is not finite");
    return THC_CPD_OK;
}

thc_cpd_status thc_cpd_als_sweep(int o, int v, int Rt, int R, const double* Xo, const double* Xv,
                                 const double* Z, double* const A[4], double* lam, double normG2,
                                 double* loss_host, double* fit_host, thc_cpd_opts* opts) {
    return run_als(o, v, Rt, R, Xo, Xv, Z, A, lam, 1, 0.0, normG2, nullptr, loss_host, fit_host, opts);
}

thc_cpd_status thc_cpd_als(int o, int v, int Rt, int R, const double* Xo, const double* Xv,
                           const double* Z, double* const A[4], double* lam, int max_sweeps,
                           double tol, int* sweeps_done, double* loss_host, double* fit_host,
                           thc_cpd_opts* opts) {
    LearnArgs la;
    la.mlp = opts ? opts->mlp : nullptr;
    thc_cpd_status st = run_als(o, v, Rt, R, Xo, Xv, Z, A, lam, max_sweeps, tol, 0.0, sweeps_done,
                                loss_host, fit_host, opts, la.mlp ? &la : nullptr);
    if (opts && la.mlp) opts->accepted_out = la.accepted;
    return st;
}

thc_cpd_status thc_cpd_als_trajectory(int o, int v, int Rt, int R, const double* Xo,
                                      const double* Xv, const double* Z, double* const A[4],
                                      double* lam, int sweeps, const double* alphas, int nalpha,
                                      float* feats, double* trial_losses, thc_cpd_opts* opts) {
    if (!alphas || nalpha < 1 || nalpha > 64 || !feats || !trial_losses)
        return set_err(THC_CPD_ERR_ARG, "need 1..64 alphas and host feature / loss buffers");
    LearnArgs la;
    la.alphas = alphas;
    la.nalpha = nalpha;
    la.feats = feats;
    la.tloss = trial_losses;
    int done = 0;
    return run_als(o, v, Rt, R, Xo, Xv, Z, A, lam, sweeps, 0.0, 0.0, &done, nullptr, nullptr, opts, &la);
}

}  // extern "C"

extern "C" thc_cpd_status thc_cpd_emulated_gemm(int M, int N, int K, const double* A, int lda, const double* B,
                                     int ldb, double* C, int ldc, const thc_cpd_opts* opts) {
    if (M < 1 || N < 1 || K < 1 || M > 4096 || N > 4096 || lda < K || ldb < K || ldc < N)
        return set_err(THC_CPD_ERR_SHAPE, "bad emulated GEMM shape %d x %d x %d (lda %d ldb %d ldc %d)",
                       M, N, K, lda, ldb, ldc);
    if (!A || !B || !C) return set_err(THC_CPD_ERR_ARG, "A, B and C must be non-null");
    if (!oz_available())
        return set_err(THC_CPD_ERR_UNSUPPORTED, "the emulated product needs an sm_103 device");
    cudaStream_t st = stream_of(opts);
    // room for every K chunk's digits (one update launch) unless that would pass 65536 rows
    const long nch = cdiv(K, kOzPanel);
    const bool all = nch * (M + N) <= 65536;
    const int rowsA = all ? (int)(nch * M) : M, rowsB = all ? (int)(nch * N) : N;
    const size_t bytes = oz_ws_bytes(rowsA, rowsB);
    struct Ws {
        void* p = nullptr;
        cudaStream_t st;
        ~Ws() {
            if (p) cudaFreeAsync(p, st);
        }
    } ws;
    ws.st = st;
    CK(cudaMallocAsync(&ws.p, bytes, st));
    Arena ar;
    ar.base = (char*)ws.p;
    ar.cap = bytes;
    OzWs oz;
    oz_ws_carve(oz, ar, rowsA, rowsB);
    CK(cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * N, M, st));
    CK(oz_gemm(st, M, N, K, A, lda, B, ldb, C, ldc, 1.0, false, oz));
    CK(cudaStreamSynchronize(st));
    if (int e = oz_take_error())
        return set_err(THC_CPD_ERR_TIMEOUT, "emulated-product kernel wait gave up (code %d)", e);
    return THC_CPD_OK;
}

namespace thc {

int spd_solve(cudaStream_t st, int R, int n, const double* H, const double* M, double* A,
              const short* tasks, int ntasks, int* used_pinv, int ldl) {
    if (used_pinv) *used_pinv = 0;
    if (!flow_prepare(R, n)) return set_err(THC_CPD_ERR_UNSUPPORTED, "no dataflow schedule for R=%d n=%d", R, n);
    const size_t RR = (size_t)R * R, nR = (size_t)n * R;
    const bool emu = use_emulated_ldl(ldl, R, n) && !tasks &&
                     oz_prepare(R, n);
    int oz_ra = R + n, oz_rb = R;
    size_t oz_part = 0;
    if (emu) bsolve_ws_rows(R, n, &oz_ra, &oz_rb, &oz_part);
    if (emu) oz_ldl_ws_rows(R, n, &oz_ra, &oz_rb);
    size_t bytes = (emu ? oz_ws_bytes(oz_ra, oz_rb, oz_part) : 0) + Arena::need<double>(RR + nR) + 3 * Arena::need<double>(RR) + Arena::need<double>(R) +
                   Arena::need<double>(std::max(RR, nR)) + Arena::need<double>(R) +
                   Arena::need<int>(flow_sync_ints(R, n)) + Arena::need<int>(bsolve_sync_ints(n)) +
                   Arena::need<DevScalars>(1) + Arena::need<short>(4 * (size_t)std::max(ntasks, 1));
    struct Ws {
        void* p = nullptr;
        cudaStream_t st;
        ~Ws() {
            if (p) cudaFreeAsync(p, st);
        }
    } ws;
    ws.st = st;
    CK(cudaMallocAsync(&ws.p, bytes, st));
    Arena ar;
    ar.base = (char*)ws.p;
    ar.cap = bytes;
    double* Haug = ar.take<double>(RR + nR);
    double* P = ar.take<double>(RR);
    double* Hsave = ar.take<double>(RR);
    double* V = ar.take<double>(RR);
    double* dinv = ar.take<double>(R);
    double* T = ar.take<double>(std::max(RR, nR));
    double* w = ar.take<double>(R);
    int* fsync = ar.take<int>(flow_sync_ints(R, n));
    int* bsync = ar.take<int>(bsolve_sync_ints(n));
    DevScalars* sc = ar.take<DevScalars>(1);
    void* dtasks = ar.take<short>(4 * (size_t)std::max(ntasks, 1));
    OzWs oz;
    if (emu) oz_ws_carve(oz, ar, oz_ra, oz_rb, oz_part);
    CK(cudaMemsetAsync(fsync, 0, sizeof(int) * flow_sync_ints(R, n), st));
    CK(cudaMemsetAsync(bsync, 0, sizeof(int) * bsolve_sync_ints(n), st));
    scalars_init(st, sc, 0.0);
    copy_with_maxdiag(st, R, H, Haug, sc);
    CK(cudaMemcpyAsync(Hsave, H, sizeof(double) * RR, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(Haug + RR, M, sizeof(double) * nR, cudaMemcpyDeviceToDevice, st));
    {
        ProfScope prof(st, KC_CHOL, (double)R * R * R / 3.0 + (double)n * R * R);
        if (tasks)
            CK(ldl_flow_tasks(st, R, n, Haug, P, dinv, sc, 0, fsync, tasks, ntasks, dtasks));
        else if (emu)
            CK(ldl_oz(st, R, n, Haug, P, dinv, sc, 0, fsync, oz));
        else
            CK(ldl_flow(st, R, n, Haug, P, dinv, sc, 0, fsync));
    }
    backward_solve(st, R, n, Haug, A, bsync, emu ? &oz : nullptr);
    CK(cudaGetLastError());
    DevScalars* h = host_scalars();
    if (!h) return set_err(THC_CPD_ERR_ALLOC, "pinned host buffer allocation failed");
    CK(cudaMemcpyAsync(h, sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (int e = flow_take_error())
        return set_err(THC_CPD_ERR_TIMEOUT, "LDL^T dataflow wait gave up (code %d)", e);
    if (int e = oz_take_error())
        return set_err(THC_CPD_ERR_TIMEOUT, "emulated-product kernel wait gave up (code %d)", e);
    if (h->fail_mask) {
        int sweeps = 0;
        CK(pinv_solve(st, R, n, Hsave, M, A, V, w, T, &sweeps));
        CK(cudaStreamSynchronize(st));
        if (used_pinv) *used_pinv = 1;
    }
    return THC_CPD_OK;
}

}  // namespace thc

thc_cpd_status thc_cpd_ldl_solve(int R, int n, const double* H, const double* M, double* A,
                                 const short* tasks, int ntasks, int* used_pinv,
                                 const thc_cpd_opts* opts) {
    NvtxRange nvtx_range("thc_cpd_ldl_solve");
    if (R < 1 || R > 2048 || n < 1 || n > 4096)
        return set_err(THC_CPD_ERR_SHAPE, "need 1 <= R <= 2048 and 1 <= n <= 4096 (R=%d n=%d)", R, n);
    if (!H || !M || !A) return set_err(THC_CPD_ERR_ARG, "H, M and A must be non-null");
    if (tasks && ntasks < 0) return set_err(THC_CPD_ERR_ARG, "ntasks must be >= 0");
    if (tasks) {
        const int bad = flow_task_check(R, n, tasks, ntasks);
        if (bad >= 0) return set_err(THC_CPD_ERR_ARG, "task %d has an out-of-range type or tile index", bad);
    }
    set_wait_limit(opts);
    return (thc_cpd_status)spd_solve(stream_of(opts), R, n, H, M, A, tasks, ntasks, used_pinv,
                                     opts ? opts->ldl : THC_CPD_LDL_AUTO);
}

thc_cpd_status thc_cpd_als_batched(int nprob, thc_cpd_problem* probs, int max_sweeps,
                                              double tol, thc_cpd_opts* opts) {
    NvtxRange nvtx_range("thc_cpd_als_batched");
    return run_batched(nprob, probs, max_sweeps, tol, opts);
}
