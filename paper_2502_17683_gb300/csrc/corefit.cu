// THC core least-squares fit f(Z) (Sec. 3, Computational Details): the core Z of a THC
// block on given grid factors Xo (o x Rt), Xv (v x Rt) that best reproduces the (o,v,o,v)
// block of density-fitted integrals G_DF[i,a,j,b] = sum_X B[X,i,a] B[X,j,b]:
//     f(Z) = 1/2 || G_DF - sum_PQ Xo[i,P] Xv[a,P] Z[P,Q] Xo[j,Q] Xv[b,Q] ||^2.
// Its normal equations are S Z S = E^T E with
//     S = (Xo^T Xo) o (Xv^T Xv)  (Rt x Rt),   E[X,P] = sum_{i,a} B[X,i,a] Xo[i,P] Xv[a,P],
// so Z = S^-1 E^T E S^-1 = F^T F with F = E S^-1: one factorisation of S and one solve with
// naux right-hand sides, and the result is symmetric by construction.
// Steps (all on the GPU):
//   T[(X,i),P] = sum_a B[X,i,a] Xv[a,P]        GEMM (X chunk * o) x v x Rt, the O(N^4) bulk
//   E[X,P]     = sum_i Xo[i,P] T[(X,i),P]      k_pair_reduce (reads T once)
//   S          = (Xo^T Xo) o (Xv^T Xv)         two symmetric GEMMs + k_hadamard2
//   F          = E S^-1                        LDL^T solve (spd_solve; pseudo-inverse fallback)
//   Z          = F^T F                         symmetric GEMM
// and, on request, the loss ||G_DF - G_THC(Z)||^2 = ||D D^T||^2 - 2 <E^T E, Z> + <Z, S Z S>
// (D[X,(i,a)] = B[X,i,a]) with three fixed-order dot products.
// The GEMMs run on the FP64 pipes, or as the FP64-accurate emulated products of the BF16
// tensor cores (oz_dgemm) when opts->ldl is THC_CPD_LDL_EMULATED.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>

#include "f64.cuh"
#include "oz.cuh"
#include "prof.cuh"
#include "thc_cpd.h"

namespace thc {
namespace {

constexpr int CF_THREADS = 256;
constexpr int CF_BLOCKS = 304;
constexpr size_t kChunkDoubles = size_t(1) << 25;  // T chunk: at most 256 MiB

// E[X,P] = sum_i Xo[i,P] T[(X * o + i) * Rt + P]   (one thread per (X, P); coalesced in P)
__global__ void k_pair_reduce(int nx, int o, int Rt, const double* __restrict__ T,
                              const double* __restrict__ Xo, double* __restrict__ E) {
    const long total = (long)nx * Rt;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int X = (int)(e / Rt), P = (int)(e % Rt);
        const double* t = T + (size_t)X * o * Rt + P;
        double s = 0.0;
        for (int i = 0; i < o; ++i) s = fma(Xo[(size_t)i * Rt + P], t[(size_t)i * Rt], s);
        E[e] = s;
    }
}

// C = A o B elementwise (n values)
__global__ void k_hadamard2(long n, const double* __restrict__ A, const double* __restrict__ B,
                            double* __restrict__ C) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        C[e] = A[e] * B[e];
}

__device__ double cf_block_sum(double v, double* sh) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    if (w == 0) {
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    }
    __syncthreads();
    return v;
}

// part[b] = block b's share of sum a o b over n values (grid-stride, fixed order)
__global__ void __launch_bounds__(CF_THREADS)
k_dot_partials(long n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ part) {
    __shared__ double sh[32];
    double s = 0.0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        s = fma(a[e], b[e], s);
    s = cf_block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out[j] = sum of part[j * nb .. (j + 1) * nb) for j < 3 (one block, fixed order)
__global__ void __launch_bounds__(CF_THREADS) k_dot_final3(const double* __restrict__ part, int nb, double* out) {
    __shared__ double sh[32];
    for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[(size_t)j * nb + i];
        s = cf_block_sum(s, sh);
        if (threadIdx.x == 0) out[j] = s;
    }
}

int grid_for(long n) { return (int)std::min<long>(std::max<long>(cdiv(n, CF_THREADS), 1), 4L * num_sms()); }

thc_cpd_status cerr(thc_cpd_status s, const char* fmt, ...) {
    char msg[320];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    return (thc_cpd_status)set_error(s, msg);
}

}  // namespace
}  // namespace thc

extern "C" thc_cpd_status thc_cpd_core_fit(int o, int v, int Rt, int naux, const double* Xo, const double* Xv,
                                           const double* B, double* Z, double* loss, int* used_pinv,
                                           const thc_cpd_opts* opts) {
    using namespace thc;
    if (o < 1 || v < 1 || naux < 1 || Rt < 1 || Rt > 2048)
        return cerr(THC_CPD_ERR_SHAPE, "need o, v, naux >= 1 and 1 <= R_thc <= 2048 (o=%d v=%d R_thc=%d naux=%d)",
                    o, v, Rt, naux);
    if ((long)o * v >= (1L << 31) || (long)naux * o >= (1L << 31) || (long)naux * Rt >= (1L << 31) ||
        (long)naux * naux >= (1L << 31))
        return cerr(THC_CPD_ERR_SHAPE, "core-fit shape too large for 32-bit GEMM sizes");
    if (!Xo || !Xv || !B || !Z) return cerr(THC_CPD_ERR_ARG, "Xo, Xv, B and Z must be non-null");
    if (used_pinv) *used_pinv = 0;
    cudaStream_t st = opts ? (cudaStream_t)opts->stream : (cudaStream_t)0;
    const int ldl = opts ? opts->ldl : THC_CPD_LDL_AUTO;
    const bool emu = ldl == THC_CPD_LDL_EMULATED && oz_available();
    if (opts) {
        const double lim = opts->wait_limit_s;
        flow_set_wait_ns(lim > 0.0 ? (unsigned long long)(lim * 1e9) : 0ull);
    }
    const size_t RR = (size_t)Rt * Rt, oRt = (size_t)o * Rt, ov = (size_t)o * v;
    // X chunk of the T stage: T holds xc * o * Rt doubles
    const int xc = (int)std::max<size_t>(1, std::min<size_t>((size_t)naux, kChunkDoubles / oRt));
    const int rows_t = xc * o;
    size_t part_cap = std::max(dgemm_part_need(rows_t, Rt, v), dgemm_part_need(Rt, Rt, std::max(o, v)));
    part_cap = std::max(part_cap, dgemm_part_need(Rt, Rt, naux));
    if (loss) part_cap = std::max(part_cap, std::max(dgemm_part_need(naux, naux, (int)ov), dgemm_part_need(Rt, Rt, Rt)));
    size_t bytes = Arena::need<double>((size_t)rows_t * Rt) + 2 * Arena::need<double>((size_t)naux * Rt) +
                   3 * Arena::need<double>(RR) + Arena::need<double>(part_cap) + Arena::need<double>(3 * CF_BLOCKS + 3);
    if (loss) bytes += Arena::need<double>(ov * naux) + Arena::need<double>((size_t)naux * naux) + 2 * Arena::need<double>(RR);
    int rowsA = std::max(rows_t, Rt), rowsB = Rt;
    if (loss) {
        rowsA = std::max(rowsA, naux);
        rowsB = std::max(rowsB, naux);
    }
    if (emu) bytes += oz_ws_bytes(rowsA, rowsB);
    void* block = nullptr;
    if (cudaMallocAsync(&block, bytes, st) != cudaSuccess) return cerr(THC_CPD_ERR_ALLOC, "workspace allocation failed");
    struct Free {
        void* p;
        cudaStream_t st;
        ~Free() { cudaFreeAsync(p, st); }
    } fr{block, st};
    Arena ar;
    ar.base = (char*)block;
    ar.cap = bytes;
    double* T = ar.take<double>((size_t)rows_t * Rt);
    double* E = ar.take<double>((size_t)naux * Rt);
    double* F = ar.take<double>((size_t)naux * Rt);
    double* S = ar.take<double>(RR);
    double* Go = ar.take<double>(RR);
    double* Gv = ar.take<double>(RR);
    double* gpart = ar.take<double>(part_cap);
    double* red = ar.take<double>(3 * CF_BLOCKS + 3);
    double *Dt = nullptr, *Q = nullptr, *W1 = nullptr, *W2 = nullptr;
    if (loss) {
        Dt = ar.take<double>(ov * naux);
        Q = ar.take<double>((size_t)naux * naux);
        W1 = ar.take<double>(RR);
        W2 = ar.take<double>(RR);
    }
    OzWs oz;
    if (emu) oz_ws_carve(oz, ar, rowsA, rowsB);
    auto gemm = [&](bool ta, int M, int N, int K, const double* A, int lda, const double* Bp, int ldb, double* C,
                    int ldc, bool symm) {
        if (emu)
            return oz_dgemm(st, ta, M, N, K, A, lda, Bp, nullptr, ldb, C, ldc, nullptr, symm, oz);
        dgemm(st, ta, M, N, K, A, lda, Bp, nullptr, ldb, C, ldc, nullptr, symm, gpart, part_cap);
        return cudaGetLastError();
    };
    cudaError_t ce = cudaSuccess;
    auto ck = [&](cudaError_t e) {
        if (ce == cudaSuccess && e != cudaSuccess) ce = e;
    };
    // E in X chunks: T = B_chunk Xv, then the occupied reduction
    for (int x0 = 0; x0 < naux && ce == cudaSuccess; x0 += xc) {
        const int nx = std::min(xc, naux - x0);
        ck(gemm(false, nx * o, Rt, v, B + (size_t)x0 * ov, v, Xv, Rt, T, Rt, false));
        k_pair_reduce<<<grid_for((long)nx * Rt), CF_THREADS, 0, st>>>(nx, o, Rt, T, Xo, E + (size_t)x0 * Rt);
        count_launch();
    }
    // S = (Xo^T Xo) o (Xv^T Xv)
    ck(gemm(true, Rt, Rt, o, Xo, Rt, Xo, Rt, Go, Rt, true));
    ck(gemm(true, Rt, Rt, v, Xv, Rt, Xv, Rt, Gv, Rt, true));
    k_hadamard2<<<grid_for((long)RR), CF_THREADS, 0, st>>>((long)RR, Go, Gv, S);
    count_launch();
    ck(cudaGetLastError());
    if (ce != cudaSuccess) return cerr(THC_CPD_ERR_CUDA, "core fit: %s", cudaGetErrorString(ce));
    // F = E S^-1 in row chunks of at most 4096 right-hand sides
    for (int r0 = 0; r0 < naux; r0 += 4096) {
        const int nr = std::min(4096, naux - r0);
        int pinv = 0;
        const int s = spd_solve(st, Rt, nr, S, E + (size_t)r0 * Rt, F + (size_t)r0 * Rt, nullptr, 0, &pinv, ldl);
        if (s != THC_CPD_OK) return (thc_cpd_status)s;
        if (pinv && used_pinv) *used_pinv = 1;
    }
    // Z = F^T F
    ck(gemm(true, Rt, Rt, naux, F, Rt, F, Rt, Z, Rt, true));
    double h[3] = {0.0, 0.0, 0.0};
    if (loss && ce == cudaSuccess) {
        // ||D D^T||^2, <E^T E, Z>, <Z, S Z S>
        transpose64(st, naux, (int)ov, B, Dt);
        ck(gemm(false, naux, naux, (int)ov, B, (int)ov, Dt, naux, Q, naux, true));
        ck(gemm(true, Rt, Rt, naux, E, Rt, E, Rt, W2, Rt, true));  // E^T E
        k_dot_partials<<<CF_BLOCKS, CF_THREADS, 0, st>>>((long)naux * naux, Q, Q, red);
        k_dot_partials<<<CF_BLOCKS, CF_THREADS, 0, st>>>((long)RR, W2, Z, red + CF_BLOCKS);
        ck(gemm(false, Rt, Rt, Rt, S, Rt, Z, Rt, W1, Rt, false));   // S Z
        ck(gemm(false, Rt, Rt, Rt, W1, Rt, S, Rt, W2, Rt, false));  // S Z S
        k_dot_partials<<<CF_BLOCKS, CF_THREADS, 0, st>>>((long)RR, Z, W2, red + 2 * CF_BLOCKS);
        k_dot_final3<<<1, CF_THREADS, 0, st>>>(red, CF_BLOCKS, red + 3 * CF_BLOCKS);
        count_launch(4);
        ck(cudaMemcpyAsync(h, red + 3 * CF_BLOCKS, sizeof h, cudaMemcpyDeviceToHost, st));
    }
    ck(cudaGetLastError());
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return cerr(THC_CPD_ERR_CUDA, "core fit: %s", cudaGetErrorString(ce));
    if (emu) {
        if (int te = oz_take_error()) return cerr(THC_CPD_ERR_TIMEOUT, "emulated-product kernel wait gave up (code %d)", te);
    }
    if (loss) {
        *loss = h[0] - 2.0 * h[1] + h[2];
        if (!isfinite(*loss)) return cerr(THC_CPD_ERR_NONFINITE, "core-fit loss is not finite");
    }
    return THC_CPD_OK;
}
