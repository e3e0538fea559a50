// THC-driven CP-ALS of order-d THC-like tensors (Conclusions: the strategy carries over to
// any THC-like network of order d). The d modes form a left group L = {0 .. dL-1} on grid
// index P and a right group R = {dL .. d-1} on Q, each mode with its own grid factor X_k:
//     G[i_0 .. i_{d-1}] = sum_{P,Q} prod_{k in L} X_k[i_k,P] Z[P,Q] prod_{k in R} X_k[i_k,Q]
// (the order-4 block of Eq. THC is d = 4, dL = 2, X = (Xo, Xv, Xo, Xv)). With the
// projections W_m = X_m^T A_m the MTTKRP of mode k is
//     k in L:  M_k = X_k ((o_{m in L, m != k} W_m) o (Z  (o_{m in R} W_m)))
//     k in R:  M_k = X_k ((o_{m in R, m != k} W_m) o (Z^T (o_{m in L} W_m)))
// so a sweep runs d projections, d back-projections and two Z products (one per group:
// the other group's factors do not change while a group is updated), at O((sum n_k) R_thc R
// + R_thc^2 R) instead of O(prod n_k R). The normal equations H_k = o_{m != k} A_m^T A_m,
// their solve, the normalisation and the factor-form loss
//     ||G||^2 = sum Z o (S_L Z S_R),  <G, Gt> = sum_r lam_r sum_Q (Z^T P_L)[Q,r] P_R[Q,r],
//     ||Gt||^2 = lam^T (o_k Gram_k) lam
// are those of the order-4 path. GEMMs on the FP64 pipes, or the FP64-accurate emulated
// tensor-core products with opts->ldl = THC_CPD_LDL_EMULATED.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "f64.cuh"
#include "oz.cuh"
#include "prof.cuh"
#include "thc_cpd.h"

namespace thc {
namespace {

constexpr int ND_MAX = 8;
constexpr int ND_THREADS = 256;

struct PtrList {
    const double* p[ND_MAX];
    int n;
};

// out = prod_j in.p[j] elementwise (n values; no factor: all ones)
__global__ void k_hprod(long n, PtrList in, double* out) {  // out may be one of the inputs
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        double s = 1.0;
        for (int j = 0; j < in.n; ++j) s *= in.p[j][e];
        out[e] = s;
    }
}

thc_cpd_status nerr(thc_cpd_status s, const char* fmt, ...) {
    char msg[320];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    return (thc_cpd_status)set_error(s, msg);
}

struct NdCtx {
    cudaStream_t st;
    int d, dL, Rt, R, nmax, ldl;
    int n[ND_MAX];
    bool emu;
    const double* X[ND_MAX];
    const double* Z;
    double *W[ND_MAX], *G[ND_MAX];
    double *P, *Y, *E, *M, *H, *GH, *ones, *lamtmp, *gpart, *red, *SL, *SR, *U;
    size_t part_cap;
    DevScalars* sc;
    OzWs oz;
    cudaError_t err = cudaSuccess;

    void ck(cudaError_t e) {
        if (err == cudaSuccess && e != cudaSuccess) err = e;
    }
    void gemm(bool ta, int M_, int N_, int K_, const double* A, int lda, const double* B, int ldb, double* C,
              int ldc, bool symm) {
        if (emu)
            ck(oz_dgemm(st, ta, M_, N_, K_, A, lda, B, nullptr, ldb, C, ldc, nullptr, symm, oz));
        else
            dgemm(st, ta, M_, N_, K_, A, lda, B, nullptr, ldb, C, ldc, nullptr, symm, gpart, part_cap);
    }
    // out = Hadamard product of the listed arrays (count values)
    void hprod(long count, std::initializer_list<const double*> l, const std::vector<const double*>& more, double* out) {
        PtrList pl{};
        pl.n = 0;
        for (const double* p : l) pl.p[pl.n++] = p;
        for (const double* p : more) pl.p[pl.n++] = p;
        ProfScope prof(st, KC_AUX, (double)count * std::max(pl.n - 1, 0), 8.0 * count * (pl.n + 1));
        count_launch();
        k_hprod<<<(int)std::min<long>(std::max<long>(cdiv(count, ND_THREADS), 1), 4L * num_sms()), ND_THREADS, 0, st>>>(
            count, pl, out);
    }
    void project(int k, const double* Ak) { gemm(true, Rt, R, n[k], X[k], Rt, Ak, R, W[k], R, false); }
    void gram(int k, const double* Ak) { gemm(true, R, R, n[k], Ak, R, Ak, R, G[k], R, true); }
    // P = Hadamard product of the W of modes [m0, m1)
    void group_product(int m0, int m1) {
        std::vector<const double*> w;
        for (int m = m0; m < m1; ++m) w.push_back(W[m]);
        hprod((long)Rt * R, {}, w, P);
    }
    // Y = Z P_R (left group) or Z^T P_L (right group)
    void zproduct(bool left) {
        if (left) {
            group_product(dL, d);
            gemm(false, Rt, R, Rt, Z, Rt, P, R, Y, R, false);
        } else {
            group_product(0, dL);
            gemm(true, Rt, R, Rt, Z, Rt, P, R, Y, R, false);
        }
    }
    // M = X_k (own-group W except k, o Y)
    void mttkrp_from_y(int k, double* out) {
        const int m0 = k < dL ? 0 : dL, m1 = k < dL ? dL : d;
        std::vector<const double*> w;
        for (int m = m0; m < m1; ++m)
            if (m != k) w.push_back(W[m]);
        hprod((long)Rt * R, {Y}, w, E);
        gemm(false, n[k], R, Rt, X[k], Rt, E, R, out, R, false);
    }
};

thc_cpd_status nd_check(int d, int dL, const int* dims, int Rt, int R, const double* const* X, const double* Z,
                        const void* const* A) {
    if (d < 2 || d > ND_MAX || dL < 1 || dL >= d)
        return nerr(THC_CPD_ERR_SHAPE, "need 2 <= d <= %d and 1 <= dL <= d - 1 (d=%d dL=%d)", ND_MAX, d, dL);
    if (!dims || !X || !Z || !A) return nerr(THC_CPD_ERR_ARG, "dims, X, Z and A must be non-null");
    if (Rt < 1 || R < 1 || R > 2048 || (long)Rt * Rt >= (1L << 31) || (long)Rt * R >= (1L << 31))
        return nerr(THC_CPD_ERR_SHAPE, "need R_thc >= 1, 1 <= R_cp <= 2048 and R_thc^2, R_thc R_cp below 2^31");
    for (int k = 0; k < d; ++k) {
        if (dims[k] < 1 || dims[k] > 4096) return nerr(THC_CPD_ERR_SHAPE, "dims[%d] = %d outside [1, 4096]", k, dims[k]);
        if (!X[k] || !A[k]) return nerr(THC_CPD_ERR_ARG, "X[%d] and A[%d] must be non-null", k, k);
    }
    return THC_CPD_OK;
}

// workspace of one context (set-up buffers only with setup)
thc_cpd_status nd_alloc(NdCtx& c, int d, int dL, const int* dims, int Rt, int R, const double* const* X,
                        const double* Z, const thc_cpd_opts* opts, bool setup, void** block) {
    c.st = opts ? (cudaStream_t)opts->stream : (cudaStream_t)0;
    c.d = d;
    c.dL = dL;
    c.Rt = Rt;
    c.R = R;
    c.nmax = 1;
    for (int k = 0; k < d; ++k) {
        c.n[k] = dims[k];
        c.X[k] = X[k];
        c.nmax = std::max(c.nmax, dims[k]);
    }
    c.Z = Z;
    c.ldl = opts ? opts->ldl : THC_CPD_LDL_AUTO;
    c.emu = c.ldl == THC_CPD_LDL_EMULATED && oz_available();
    const size_t RtR = (size_t)Rt * R, RR = (size_t)R * R, RtRt = (size_t)Rt * Rt;
    c.part_cap = std::max(dgemm_part_need(Rt, R, c.nmax), dgemm_part_need(Rt, R, Rt));
    c.part_cap = std::max(c.part_cap, std::max(dgemm_part_need(c.nmax, R, Rt), dgemm_part_need(R, R, c.nmax)));
    if (setup) c.part_cap = std::max(c.part_cap, std::max(dgemm_part_need(Rt, Rt, c.nmax), dgemm_part_need(Rt, Rt, Rt)));
    const int rowsA = std::max(std::max(c.nmax, Rt), R), rowsB = std::max(R, Rt);
    size_t bytes = (size_t)d * (Arena::need<double>(RtR) + Arena::need<double>(RR)) + 3 * Arena::need<double>(RtR) +
                   Arena::need<double>((size_t)c.nmax * R) + 2 * Arena::need<double>(RR) +
                   Arena::need<double>(std::max(RtR, RR)) + Arena::need<double>(R) + Arena::need<double>(c.part_cap) +
                   Arena::need<double>(loss_red_need()) + Arena::need<DevScalars>(1);
    if (setup) bytes += 3 * Arena::need<double>(RtRt);
    if (c.emu) bytes += oz_ws_bytes(rowsA, rowsB);
    if (cudaMallocAsync(block, bytes, c.st) != cudaSuccess) return nerr(THC_CPD_ERR_ALLOC, "workspace allocation failed");
    Arena ar;
    ar.base = (char*)*block;
    ar.cap = bytes;
    for (int k = 0; k < d; ++k) {
        c.W[k] = ar.take<double>(RtR);
        c.G[k] = ar.take<double>(RR);
    }
    c.P = ar.take<double>(RtR);
    c.Y = ar.take<double>(RtR);
    c.E = ar.take<double>(RtR);
    c.M = ar.take<double>((size_t)c.nmax * R);
    c.H = ar.take<double>(RR);
    c.GH = ar.take<double>(RR);
    c.ones = ar.take<double>(std::max(RtR, RR));
    c.lamtmp = ar.take<double>(R);
    c.gpart = ar.take<double>(c.part_cap);
    c.red = ar.take<double>(loss_red_need());
    c.sc = ar.take<DevScalars>(1);
    c.SL = c.SR = c.U = nullptr;
    if (setup) {
        c.SL = ar.take<double>(RtRt);
        c.SR = ar.take<double>(RtRt);
        c.U = ar.take<double>(RtRt);
    }
    if (c.emu) oz_ws_carve(c.oz, ar, rowsA, rowsB);
    return THC_CPD_OK;
}

struct Free {
    void* p = nullptr;
    cudaStream_t st;
    ~Free() {
        if (p) cudaFreeAsync(p, st);
    }
};

}  // namespace
}  // namespace thc

extern "C" thc_cpd_status thc_cpd_nd_mttkrp(int d, int dL, const int* dims, int Rt, int R, const double* const* X,
                                            const double* Z, const double* const* A, int mode, double* M,
                                            const thc_cpd_opts* opts) {
    using namespace thc;
    const thc_cpd_status chk = nd_check(d, dL, dims, Rt, R, X, Z, (const void* const*)A);
    if (chk != THC_CPD_OK) return chk;
    if (mode < 0 || mode >= d) return nerr(THC_CPD_ERR_ARG, "mode %d outside [0, %d)", mode, d);
    if (!M) return nerr(THC_CPD_ERR_ARG, "M must be non-null");
    if (opts && opts->precision != THC_CPD_FP64)
        return nerr(THC_CPD_ERR_ARG, "the order-d path runs in FP64 (precision must be THC_CPD_FP64)");
    NdCtx c;
    Free fr;
    const thc_cpd_status a = nd_alloc(c, d, dL, dims, Rt, R, X, Z, opts, false, &fr.p);
    fr.st = c.st;
    if (a != THC_CPD_OK) return a;
    for (int m = 0; m < d; ++m)
        if (m != mode) c.project(m, A[m]);
    c.zproduct(mode < dL);
    c.mttkrp_from_y(mode, M);
    c.ck(cudaGetLastError());
    if (c.err == cudaSuccess) c.ck(cudaStreamSynchronize(c.st));
    if (c.err != cudaSuccess) return nerr(THC_CPD_ERR_CUDA, "order-d MTTKRP: %s", cudaGetErrorString(c.err));
    if (c.emu)
        if (int te = oz_take_error()) return nerr(THC_CPD_ERR_TIMEOUT, "emulated-product kernel wait gave up (code %d)", te);
    return THC_CPD_OK;
}

extern "C" thc_cpd_status thc_cpd_nd_als(int d, int dL, const int* dims, int Rt, int R, const double* const* X,
                                         const double* Z, double* const* A, double* lam, int max_sweeps, double tol,
                                         int* sweeps_done, double* fit_host, thc_cpd_opts* opts) {
    using namespace thc;
    const thc_cpd_status chk = nd_check(d, dL, dims, Rt, R, X, Z, (const void* const*)A);
    if (chk != THC_CPD_OK) return chk;
    if (!lam) return nerr(THC_CPD_ERR_ARG, "lam must be non-null");
    if (max_sweeps < 1) return nerr(THC_CPD_ERR_ARG, "max_sweeps must be >= 1");
    if (opts && opts->precision != THC_CPD_FP64)
        return nerr(THC_CPD_ERR_ARG, "the order-d path runs in FP64 (precision must be THC_CPD_FP64)");
    if (opts) {
        opts->flags_out = 0;
        const double lim = opts->wait_limit_s;
        flow_set_wait_ns(lim > 0.0 ? (unsigned long long)(lim * 1e9) : 0ull);
    }
    NdCtx c;
    Free fr;
    const thc_cpd_status a = nd_alloc(c, d, dL, dims, Rt, R, X, Z, opts, true, &fr.p);
    fr.st = c.st;
    if (a != THC_CPD_OK) return a;
    cudaStream_t st = c.st;
    const size_t RtR = (size_t)Rt * R, RR = (size_t)R * R, RtRt = (size_t)Rt * Rt;

    // set-up: ||G||^2 = sum Z o (S_L Z S_R), projections and Grams of the start factors
    scalars_init(st, c.sc, 0.0);
    fill(st, c.ones, (long)std::max(RtR, RR), 1.0);
    {
        std::vector<const double*> gl, gr;
        for (int k = 0; k < d; ++k) {
            c.gemm(true, Rt, Rt, c.n[k], X[k], Rt, X[k], Rt, c.U, Rt, true);  // X_k^T X_k
            // fold it into the group's product right away (U is reused)
            double* S = k < dL ? c.SL : c.SR;
            const bool first = (k == 0) || (k == dL);
            c.hprod((long)RtRt, {c.U}, first ? std::vector<const double*>{} : std::vector<const double*>{S}, S);
        }
        c.gemm(false, Rt, Rt, Rt, c.SL, Rt, Z, Rt, c.U, Rt, false);
        c.gemm(false, Rt, Rt, Rt, c.U, Rt, c.SR, Rt, c.SL, Rt, false);  // S_L Z S_R (S_L no longer needed)
        sum_hadamard_normG2(st, (long)RtRt, Z, c.SL, c.red, c.sc);
    }
    for (int k = 0; k < d; ++k) {
        c.project(k, A[k]);
        c.gram(k, A[k]);
    }
    c.ck(cudaGetLastError());
    if (c.err != cudaSuccess) return nerr(THC_CPD_ERR_CUDA, "order-d set-up: %s", cudaGetErrorString(c.err));

    DevScalars hs{};
    int s = 0, pinv_any = 0;
    for (s = 1; s <= max_sweeps; ++s) {
        for (int k = 0; k < d; ++k) {
            if (k == 0) c.zproduct(true);
            if (k == dL) c.zproduct(false);
            c.mttkrp_from_y(k, c.M);
            std::vector<const double*> g;
            for (int m = 0; m < d; ++m)
                if (m != k) g.push_back(c.G[m]);
            c.hprod((long)RR, {}, g, c.H);
            c.ck(cudaGetLastError());
            if (c.err != cudaSuccess) return nerr(THC_CPD_ERR_CUDA, "order-d sweep: %s", cudaGetErrorString(c.err));
            int pinv = 0;
            const int rs = spd_solve(st, R, c.n[k], c.H, c.M, A[k], nullptr, 0, &pinv, c.ldl);
            if (rs != THC_CPD_OK) return (thc_cpd_status)rs;
            pinv_any |= pinv;
            normalise_columns(st, c.n[k], R, A[k], lam, c.lamtmp);
            c.gram(k, A[k]);
            c.project(k, A[k]);
        }
        // inner = sum_r lam_r sum_Q Y[Q,r] P_R[Q,r] with Y = Z^T P_L of this sweep; the CPD norm
        // from the Hadamard product of all Grams (the three remaining Gram slots all ones)
        c.group_product(dL, d);
        std::vector<const double*> g;
        for (int m = 0; m < d; ++m) g.push_back(c.G[m]);
        c.hprod((long)RR, {}, g, c.GH);
        const double* Gs[4] = {c.GH, c.ones, c.ones, c.ones};
        loss_eval(st, Rt, R, c.Y, c.P, c.ones, lam, Gs, c.red, c.sc, tol > 0.0 ? tol : -1.0);
        c.ck(cudaMemcpyAsync(&hs, c.sc, sizeof hs, cudaMemcpyDeviceToHost, st));
        c.ck(cudaStreamSynchronize(st));
        if (c.err != cudaSuccess) return nerr(THC_CPD_ERR_CUDA, "order-d sweep: %s", cudaGetErrorString(c.err));
        if (opts && opts->history) {
            opts->history[2 * (s - 1)] = hs.loss;
            opts->history[2 * (s - 1) + 1] = hs.fit;
        }
        if (hs.nonfinite || !isfinite(hs.fit)) return nerr(THC_CPD_ERR_NONFINITE, "order-d ALS loss is not finite");
        if (tol > 0.0 && hs.done) break;
    }
    if (s > max_sweeps) s = max_sweeps;
    if (c.emu)
        if (int te = oz_take_error()) return nerr(THC_CPD_ERR_TIMEOUT, "emulated-product kernel wait gave up (code %d)", te);
    if (opts && pinv_any) opts->flags_out |= 1;
    if (sweeps_done) *sweeps_done = s;
    if (fit_host) *fit_host = hs.fit;
    return THC_CPD_OK;
}
