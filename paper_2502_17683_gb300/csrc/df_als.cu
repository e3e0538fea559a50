// DF-driven CP-ALS (Sec. 2.1, Eq. df_loss): the prior-work variant that the THC-driven
// method replaces. CP-ALS of the (o,v,o,v) block of density-fitted integrals
//     G_DF[i,a,j,b] = sum_X B[X,i,a] B[X,j,b]      (B: naux x o x v)
// with every MTTKRP formed from the order-3 DF tensor at O(naux o v R) per mode:
//     V12[X,r] = sum_{i,a} B[X,i,a] A1[i,r] A2[a,r],   V34[X,r] = sum_{j,b} B[X,j,b] A3[j,r] A4[b,r]
//     M1 = sum_X (B[X] A2) V34[X,:]     M2 = sum_X (B[X]^T A1) V34[X,:]
//     M3 = sum_X (B[X] A4) V12[X,:]     M4 = sum_X (B[X]^T A3) V12[X,:]   (row-wise products)
// One sweep runs four GEMMs of 2 naux o v R flop (the O(N^3 R) bulk) and, around them,
// reductions over X that read each GEMM result once:
//   mode 1: T = B A2            (naux o x R)  M1[i,r] = sum_X T[(X,i),r] V34[X,r]
//   mode 2: T = B^T-per-X A1    (naux v x R)  M2[a,r] = sum_X T[(X,a),r] V34[X,r];
//           after the update    V12[X,r] = sum_a T[(X,a),r] A2[a,r]
//   mode 3: T = B A4                          M3 from V12
//   mode 4: T = B^T-per-X A3                  M4 from V12; after the update V34 from T and A4
// The second kind of GEMM reads a copy of B permuted to (o, naux, v), so that both kinds are
// single GEMMs over all X. The normal equations, their solve (LDL^T, pseudo-inverse on a
// failed pivot), the column normalisation and the factor-form loss are those of the
// THC-driven path; only the MTTKRP and ||G_DF||^2 = ||D D^T||_F^2 (D = B as naux x o v)
// differ. GEMMs on the FP64 pipes, or the FP64-accurate emulated products of the tensor
// cores with opts->ldl = THC_CPD_LDL_EMULATED (the solve then uses the emulated two-level
// LDL^T too).
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

constexpr int DF_THREADS = 256;

int df_grid(long n) { return (int)std::min<long>(std::max<long>(cdiv(n, DF_THREADS), 1), 4L * num_sms()); }

// Bp[(i * naux + X) * v + a] = B[(X * o + i) * v + a]
__global__ void k_df_permute(int naux, int o, int v, const double* __restrict__ B, double* __restrict__ Bp) {
    const long total = (long)naux * o * v;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int a = (int)(e % v);
        const long t = e / v;
        const int X = (int)(t % naux), i = (int)(t / naux);
        Bp[e] = B[((size_t)X * o + i) * v + a];
    }
}

// M[n, r] = sum_X T[(X * nn + n) * R + r] V[X * R + r]   (X ascending; one thread per (n, r))
__global__ void k_df_contract(int naux, int nn, int R, const double* __restrict__ T,
                              const double* __restrict__ V, double* __restrict__ M) {
    const long total = (long)nn * R;
    const size_t xs = (size_t)nn * R;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int r = (int)(e % R);
        const double* t = T + e;
        double s = 0.0;
        for (int X = 0; X < naux; ++X) s = fma(t[X * xs], V[(size_t)X * R + r], s);
        M[e] = s;
    }
}

// V[X, r] = sum_n T[(X * nn + n) * R + r] A[n * R + r]   (n ascending; one thread per (X, r))
__global__ void k_df_pair(int naux, int nn, int R, const double* __restrict__ T, const double* __restrict__ A,
                          double* __restrict__ V) {
    const long total = (long)naux * R;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int X = (int)(e / R), r = (int)(e % R);
        const double* t = T + (size_t)X * nn * R + r;
        double s = 0.0;
        for (int n = 0; n < nn; ++n) s = fma(t[(size_t)n * R], A[(size_t)n * R + r], s);
        V[e] = s;
    }
}

thc_cpd_status derr(thc_cpd_status s, const char* fmt, ...) {
    char msg[320];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    return (thc_cpd_status)set_error(s, msg);
}

struct DfCtx {
    cudaStream_t st;
    int o, v, naux, R, ldl;
    bool emu;
    const double* B;
    double *Bp, *T, *V12, *V34, *ones, *H, *M, *lamtmp, *gpart, *red;
    double* G[4];
    size_t part_cap;
    DevScalars* sc;
    OzWs oz;
    cudaError_t err = cudaSuccess;

    void ck(cudaError_t e) {
        if (err == cudaSuccess && e != cudaSuccess) err = e;
    }
    void gemm(bool ta, int M_, int N_, int K_, const double* A, int lda, const double* Bm, int ldb, double* C,
              int ldc, bool symm) {
        if (emu)
            ck(oz_dgemm(st, ta, M_, N_, K_, A, lda, Bm, nullptr, ldb, C, ldc, nullptr, symm, oz));
        else
            dgemm(st, ta, M_, N_, K_, A, lda, Bm, nullptr, ldb, C, ldc, nullptr, symm, gpart, part_cap);
    }
    // T[(X,i),r] = sum_a B[X,i,a] Aq[a,r]  (B's virtual index contracted)
    void t_virtual(const double* Aq) { gemm(false, naux * o, R, v, B, v, Aq, R, T, R, false); }
    // T[(X,a),r] = sum_i B[X,i,a] Ap[i,r]  (B's occupied index contracted, through Bp)
    void t_occupied(const double* Ap) { gemm(true, naux * v, R, o, Bp, naux * v, Ap, R, T, R, false); }
    void contract(int nn, const double* V, double* out) {
        ProfScope prof(st, KC_AUX, 2.0 * naux * (double)nn * R, 8.0 * naux * (double)nn * R);
        count_launch();
        k_df_contract<<<df_grid((long)nn * R), DF_THREADS, 0, st>>>(naux, nn, R, T, V, out);
    }
    void pair(int nn, const double* A, double* V) {
        ProfScope prof(st, KC_AUX, 2.0 * naux * (double)nn * R, 8.0 * naux * (double)nn * R);
        count_launch();
        k_df_pair<<<df_grid((long)naux * R), DF_THREADS, 0, st>>>(naux, nn, R, T, A, V);
    }
    void gram(int k, const double* Ak) {
        const int n = (k & 1) ? v : o;
        gemm(true, R, R, n, Ak, R, Ak, R, G[k], R, true);
    }
};

}  // namespace
}  // namespace thc

extern "C" thc_cpd_status thc_cpd_df_als(int o, int v, int naux, int R, const double* B, double* const A[4],
                                         double* lam, int max_sweeps, double tol, int* sweeps_done,
                                         double* fit_host, thc_cpd_opts* opts) {
    using namespace thc;
    if (o < 1 || v < 1 || naux < 1 || R < 1 || R > 2048 || o > 4096 || v > 4096)
        return derr(THC_CPD_ERR_SHAPE, "need o, v in [1, 4096], naux >= 1 and 1 <= R_cp <= 2048 (o=%d v=%d naux=%d R=%d)",
                    o, v, naux, R);
    const long nmax = std::max(o, v);
    if ((long)o * v >= (1L << 31) || naux * nmax >= (1L << 31) || (long)naux * naux >= (1L << 31))
        return derr(THC_CPD_ERR_SHAPE, "DF shape too large for 32-bit GEMM sizes");
    if (!B || !A || !A[0] || !A[1] || !A[2] || !A[3] || !lam)
        return derr(THC_CPD_ERR_ARG, "B, the four factors and lam must be non-null");
    if (max_sweeps < 1) return derr(THC_CPD_ERR_ARG, "max_sweeps must be >= 1");
    if (opts && opts->precision != THC_CPD_FP64)
        return derr(THC_CPD_ERR_ARG, "DF-driven ALS runs in FP64 (precision must be THC_CPD_FP64)");
    if (opts) opts->flags_out = 0;
    DfCtx c;
    c.st = opts ? (cudaStream_t)opts->stream : (cudaStream_t)0;
    c.o = o;
    c.v = v;
    c.naux = naux;
    c.R = R;
    c.ldl = opts ? opts->ldl : THC_CPD_LDL_AUTO;
    c.emu = c.ldl == THC_CPD_LDL_EMULATED && oz_available();
    c.B = B;
    if (opts) {
        const double lim = opts->wait_limit_s;
        flow_set_wait_ns(lim > 0.0 ? (unsigned long long)(lim * 1e9) : 0ull);
    }
    const size_t RR = (size_t)R * R, ov = (size_t)o * v, nR = (size_t)naux * R;
    c.part_cap = std::max(dgemm_part_need((int)(naux * nmax), R, (int)nmax), dgemm_part_need(R, R, (int)nmax));
    c.part_cap = std::max(c.part_cap, dgemm_part_need(naux, naux, (int)ov));
    const int rowsA = (int)std::max<long>(naux * nmax, R), rowsB = std::max(R, naux);
    size_t bytes = Arena::need<double>(ov * naux) * 2 + Arena::need<double>((size_t)naux * nmax * R) +
                   3 * Arena::need<double>(nR) + 5 * Arena::need<double>(RR) + Arena::need<double>(nmax * R) +
                   Arena::need<double>(R) + Arena::need<double>(c.part_cap) + Arena::need<double>(loss_red_need()) +
                   Arena::need<double>((size_t)naux * naux) + Arena::need<DevScalars>(1);
    if (c.emu) bytes += oz_ws_bytes(rowsA, rowsB);
    void* block = nullptr;
    if (cudaMallocAsync(&block, bytes, c.st) != cudaSuccess) return derr(THC_CPD_ERR_ALLOC, "workspace allocation failed");
    struct Free {
        void* p;
        cudaStream_t st;
        ~Free() { cudaFreeAsync(p, st); }
    } fr{block, c.st};
    Arena ar;
    ar.base = (char*)block;
    ar.cap = bytes;
    c.Bp = ar.take<double>(ov * naux);
    double* Dt = ar.take<double>(ov * naux);
    c.T = ar.take<double>((size_t)naux * nmax * R);
    c.V12 = ar.take<double>(nR);
    c.V34 = ar.take<double>(nR);
    c.ones = ar.take<double>(nR);
    for (int k = 0; k < 4; ++k) c.G[k] = ar.take<double>(RR);
    c.H = ar.take<double>(RR);
    c.M = ar.take<double>(nmax * R);
    c.lamtmp = ar.take<double>(R);
    c.gpart = ar.take<double>(c.part_cap);
    c.red = ar.take<double>(loss_red_need());
    double* Q = ar.take<double>((size_t)naux * naux);
    c.sc = ar.take<DevScalars>(1);
    if (c.emu) oz_ws_carve(c.oz, ar, rowsA, rowsB);
    cudaStream_t st = c.st;

    // set-up: permuted B, ||G_DF||^2 = ||D D^T||^2, Grams, V34 of the start factors
    count_launch();
    k_df_permute<<<df_grid((long)ov * naux), DF_THREADS, 0, st>>>(naux, o, v, B, c.Bp);
    fill(st, c.ones, (long)nR, 1.0);
    scalars_init(st, c.sc, 0.0);
    transpose64(st, naux, (int)ov, B, Dt);
    c.gemm(false, naux, naux, (int)ov, B, (int)ov, Dt, naux, Q, naux, true);
    sum_hadamard_normG2(st, (long)naux * naux, Q, Q, c.red, c.sc);
    for (int k = 0; k < 4; ++k) c.gram(k, A[k]);
    c.t_virtual(A[3]);
    c.pair(o, A[2], c.V34);
    c.ck(cudaGetLastError());
    if (c.err != cudaSuccess) return derr(THC_CPD_ERR_CUDA, "DF set-up: %s", cudaGetErrorString(c.err));

    DevScalars hs{};
    int s = 0;
    int pinv_any = 0;
    for (s = 1; s <= max_sweeps; ++s) {
        for (int k = 0; k < 4; ++k) {
            const int n = (k & 1) ? v : o;
            // MTTKRP of mode k
            switch (k) {
                case 0: c.t_virtual(A[1]); c.contract(o, c.V34, c.M); break;
                case 1: c.t_occupied(A[0]); c.contract(v, c.V34, c.M); break;
                case 2: c.t_virtual(A[3]); c.contract(o, c.V12, c.M); break;
                default: c.t_occupied(A[2]); c.contract(v, c.V12, c.M); break;
            }
            int a = 0, b = 0, d = 0, idx = 0;
            for (int m = 0; m < 4; ++m)
                if (m != k) (idx == 0 ? a : idx == 1 ? b : d) = m, ++idx;
            hadamard3(st, R, c.G[a], c.G[b], c.G[d], c.H, c.sc);
            c.ck(cudaGetLastError());
            if (c.err != cudaSuccess) return derr(THC_CPD_ERR_CUDA, "DF sweep: %s", cudaGetErrorString(c.err));
            int pinv = 0;
            const int rs = spd_solve(st, R, n, c.H, c.M, A[k], nullptr, 0, &pinv, c.ldl);
            if (rs != THC_CPD_OK) return (thc_cpd_status)rs;
            pinv_any |= pinv;
            normalise_columns(st, n, R, A[k], lam, c.lamtmp);
            c.gram(k, A[k]);
            if (k == 1) c.pair(v, A[1], c.V12);  // T still holds B^T-per-X A1
            if (k == 3) c.pair(v, A[3], c.V34);  // T holds B^T-per-X A3
        }
        const double* Gc[4] = {c.G[0], c.G[1], c.G[2], c.G[3]};
        loss_eval(st, naux, R, c.V12, c.V34, c.ones, lam, Gc, c.red, c.sc, tol > 0.0 ? tol : -1.0);
        c.ck(cudaMemcpyAsync(&hs, c.sc, sizeof hs, cudaMemcpyDeviceToHost, st));
        c.ck(cudaStreamSynchronize(st));
        if (c.err != cudaSuccess) return derr(THC_CPD_ERR_CUDA, "DF sweep: %s", cudaGetErrorString(c.err));
        if (opts && opts->history) {
            opts->history[2 * (s - 1)] = hs.loss;
            opts->history[2 * (s - 1) + 1] = hs.fit;
        }
        if (hs.nonfinite || !isfinite(hs.fit)) return derr(THC_CPD_ERR_NONFINITE, "DF-driven ALS loss is not finite");
        if (tol > 0.0 && hs.done) break;
    }
    if (s > max_sweeps) s = max_sweeps;
    if (c.emu) {
        if (int te = oz_take_error()) return derr(THC_CPD_ERR_TIMEOUT, "emulated-product kernel wait gave up (code %d)", te);
    }
    if (opts && pinv_any) opts->flags_out |= 1;
    if (sweeps_done) *sweeps_done = s;
    if (fit_host) *fit_host = hs.fit;
    return THC_CPD_OK;
}
