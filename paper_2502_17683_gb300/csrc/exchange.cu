// The CPD+THC LT-MP2 exchange energy (Sec. 2.2): the consumer of the CPD factors that ALS
// produces. Per Laplace quadrature point alpha (Eq. lt_D, factors Lam (occupied) and Gam
// (virtual) of Eq. mp1_t):
//   single CPD (Eq. cpd_single_k):  U1 = (Lam o Xo)^T A1, U3 = (Lam o Xo)^T A3,
//       U2 = (Gam o Xv)^T A2, U4 = (Gam o Xv)^T A4, Y = Z (U3 o U2),
//       E_single = - sum_{P,r} lam_r U1[P,r] U4[P,r] Y[P,r]             O(R_thc^2 R)
//   double CPD:  M1 = A1^T diag(Lam) A1, M3 = A3^T diag(Lam) A3, N = A2^T diag(Gam) A4,
//       E_double = - lam^T (M1 o N o M3 o N^T) lam                       O(N R^2)
//   robust (Eq. rob_K):  E_robust = 2 E_single - E_double (no first-order CPD error).
// The products run as FP64 GEMMs, on the FP64 pipes or, on request, as the FP64-accurate
// emulated products of the BF16 tensor cores (oz_dgemm); the reductions are fixed-order.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "f64.cuh"
#include "oz.cuh"
#include "prof.cuh"
#include "thc_cpd.h"

namespace thc {
namespace {

constexpr int XR_THREADS = 256;
constexpr int XR_BLOCKS = 304;

__device__ double xr_block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    if (w == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    return v;
}

// out[r * n + c] = s[r] * X[r * n + c]   (rows scaled by the quadrature factors)
__global__ void k_scale_rows(int rows, int n, const double* __restrict__ s, const double* __restrict__ X,
                             double* __restrict__ out) {
    const long total = (long)rows * n;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x)
        out[e] = s[e / n] * X[e];
}

// partial sums of lam_r U1 U4 Y over the Rt x R grid (one per block, fixed order)
__global__ void __launch_bounds__(XR_THREADS)
k_single_partials(long n, int R, const double* __restrict__ U1, const double* __restrict__ U4,
                  const double* __restrict__ Y, const double* __restrict__ lam, double* __restrict__ part) {
    __shared__ double sh[32];
    double s = 0.0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
        s = fma(lam[e % R] * U1[e], U4[e] * Y[e], s);
    s = xr_block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// partial sums of lam_r lam_s M1[r,s] N[r,s] M3[r,s] N[s,r] over 32 x 32 tiles (N^T through
// shared memory so that both reads are coalesced)
__global__ void __launch_bounds__(XR_THREADS)
k_double_partials(int R, const double* __restrict__ M1, const double* __restrict__ N,
                  const double* __restrict__ M3, const double* __restrict__ lam, double* __restrict__ part) {
    __shared__ double nt[32][33];
    __shared__ double sh[32];
    const int tiles = (R + 31) / 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    double s = 0.0;
    for (int t = blockIdx.x; t < tiles * tiles; t += gridDim.x) {
        const int r0 = (t / tiles) * 32, c0 = (t % tiles) * 32;
        __syncthreads();
        for (int k = ty; k < 32; k += 8) {  // nt[k][tx] = N[c0 + k][r0 + tx]
            const int rr = c0 + k, cc = r0 + tx;
            nt[k][tx] = (rr < R && cc < R) ? N[(size_t)rr * R + cc] : 0.0;
        }
        __syncthreads();
        for (int k = ty; k < 32; k += 8) {
            const int r = r0 + k, c = c0 + tx;
            if (r < R && c < R) {
                const size_t e = (size_t)r * R + c;
                s = fma(lam[r] * lam[c], M1[e] * N[e] * M3[e] * nt[tx][k], s);
            }
        }
    }
    s = xr_block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out[slot] = -sum of the partials (one block, fixed order)
__global__ void __launch_bounds__(XR_THREADS)
k_neg_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
    s = xr_block_sum(s, sh);
    if (threadIdx.x == 0) *out = -s;
}

thc_cpd_status xerr(thc_cpd_status s, const char* m) { return (thc_cpd_status)set_error(s, m); }

}  // namespace
}  // namespace thc

extern "C" thc_cpd_status thc_cpd_exchange(int o, int v, int Rt, int R, int nalpha, const double* Xo,
                                           const double* Xv, const double* Z, const double* const A[4],
                                           const double* lam, const double* Lam, const double* Gam,
                                           double* e_single, double* e_double, double* e_robust,
                                           const thc_cpd_opts* opts) {
    using namespace thc;
    const int chk = check_problem_args(o, v, Rt, R, Xo, Xv, Z, A);
    if (chk != THC_CPD_OK) return (thc_cpd_status)chk;
    if (nalpha < 1 || nalpha > 1024) return xerr(THC_CPD_ERR_SHAPE, "need 1 <= nalpha <= 1024");
    if (!lam || !Lam || !Gam) return xerr(THC_CPD_ERR_ARG, "lam, Lam and Gam must be non-null");
    const bool emu = opts && opts->ldl == THC_CPD_LDL_EMULATED && oz_available() && Rt <= 8192 && R <= 8192;
    cudaStream_t st = opts ? (cudaStream_t)opts->stream : (cudaStream_t)0;
    const size_t RtR = (size_t)Rt * R, RR = (size_t)R * R;
    const int nmax = std::max(o, v);
    const size_t part_cap = std::max(dgemm_part_need(Rt, R, Rt),
                                     std::max(dgemm_part_need(Rt, R, nmax), dgemm_part_need(R, R, nmax)));
    size_t bytes = Arena::need<double>((size_t)o * Rt) + Arena::need<double>((size_t)v * Rt) +
                   5 * Arena::need<double>(RtR) + 3 * Arena::need<double>((size_t)nmax * R) +
                   3 * Arena::need<double>(RR) + Arena::need<double>(XR_BLOCKS) +
                   Arena::need<double>(2 * (size_t)nalpha) + Arena::need<double>(part_cap);
    if (emu) bytes += oz_ws_bytes(std::max(Rt, R), R);
    void* block = nullptr;
    if (cudaMallocAsync(&block, bytes, st) != cudaSuccess) return xerr(THC_CPD_ERR_ALLOC, "workspace allocation failed");
    Arena ar;
    ar.base = (char*)block;
    ar.cap = bytes;
    double* XoL = ar.take<double>((size_t)o * Rt);
    double* XvG = ar.take<double>((size_t)v * Rt);
    double* U[4];
    for (int k = 0; k < 4; ++k) U[k] = ar.take<double>(RtR);
    double* Y = ar.take<double>(RtR);
    double* A1L = ar.take<double>((size_t)nmax * R);
    double* A3L = ar.take<double>((size_t)nmax * R);
    double* A4G = ar.take<double>((size_t)nmax * R);
    double* M1 = ar.take<double>(RR);
    double* M3 = ar.take<double>(RR);
    double* N = ar.take<double>(RR);
    double* part = ar.take<double>(XR_BLOCKS);
    double* res = ar.take<double>(2 * (size_t)nalpha);
    double* gpart = ar.take<double>(part_cap);
    OzWs oz;
    if (emu) oz_ws_carve(oz, ar, std::max(Rt, R), R);
    auto gemm = [&](bool ta, int M, int Nn, int K, const double* Ap, int lda, const double* Bp,
                    const double* B2, int ldb, double* C, int ldc) {
        if (emu)
            oz_dgemm(st, ta, M, Nn, K, Ap, lda, Bp, B2, ldb, C, ldc, nullptr, false, oz);
        else
            dgemm(st, ta, M, Nn, K, Ap, lda, Bp, B2, ldb, C, ldc, nullptr, false, gpart, part_cap);
    };
    auto scale = [&](int rows, int n, const double* s, const double* X, double* out) {
        const long total = (long)rows * n;
        k_scale_rows<<<(int)std::min<long>(cdiv(total, 256), 4L * num_sms()), 256, 0, st>>>(rows, n, s, X, out);
        count_launch();
    };
    {
        ProfScope prof(st, emu ? KC_OZ : KC_DGEMM,
                       (double)nalpha * (4.0 * (o + v) * RtR + 2.0 * Rt * RtR + (4.0 * o + 2.0 * v) * RR));
        for (int al = 0; al < nalpha; ++al) {
            const double* lA = Lam + (size_t)al * o;
            const double* gA = Gam + (size_t)al * v;
            // single CPD
            scale(o, Rt, lA, Xo, XoL);
            scale(v, Rt, gA, Xv, XvG);
            gemm(true, Rt, R, o, XoL, Rt, A[0], nullptr, R, U[0], R);
            gemm(true, Rt, R, o, XoL, Rt, A[2], nullptr, R, U[2], R);
            gemm(true, Rt, R, v, XvG, Rt, A[1], nullptr, R, U[1], R);
            gemm(true, Rt, R, v, XvG, Rt, A[3], nullptr, R, U[3], R);
            gemm(false, Rt, R, Rt, Z, Rt, U[2], U[1], R, Y, R);  // Z (U3 o U2)
            k_single_partials<<<XR_BLOCKS, XR_THREADS, 0, st>>>((long)RtR, R, U[0], U[3], Y, lam, part);
            k_neg_final<<<1, XR_THREADS, 0, st>>>(part, XR_BLOCKS, res + 2 * al);
            // double CPD
            scale(o, R, lA, A[0], A1L);
            scale(o, R, lA, A[2], A3L);
            scale(v, R, gA, A[3], A4G);
            gemm(true, R, R, o, A[0], R, A1L, nullptr, R, M1, R);
            gemm(true, R, R, o, A[2], R, A3L, nullptr, R, M3, R);
            gemm(true, R, R, v, A[1], R, A4G, nullptr, R, N, R);
            k_double_partials<<<XR_BLOCKS, XR_THREADS, 0, st>>>(R, M1, N, M3, lam, part);
            k_neg_final<<<1, XR_THREADS, 0, st>>>(part, XR_BLOCKS, res + 2 * al + 1);
            count_launch(4);
        }
    }
    std::vector<double> h(2 * (size_t)nalpha);
    cudaError_t e = cudaMemcpyAsync(h.data(), res, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(block, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "exchange energy failed: %s", cudaGetErrorString(e));
        return xerr(THC_CPD_ERR_CUDA, msg);
    }
    if (emu) {
        if (int te = oz_take_error()) {
            char msg[128];
            snprintf(msg, sizeof msg, "emulated-product kernel wait gave up (code %d)", te);
            return xerr(THC_CPD_ERR_TIMEOUT, msg);
        }
    }
    double e1 = 0.0, e2 = 0.0;
    for (int al = 0; al < nalpha; ++al) {
        e1 += h[2 * al];
        e2 += h[2 * al + 1];
    }
    if (!isfinite(e1) || !isfinite(e2)) return xerr(THC_CPD_ERR_NONFINITE, "exchange energy is not finite");
    if (e_single) *e_single = e1;
    if (e_double) *e_double = e2;
    if (e_robust) *e_robust = 2.0 * e1 - e2;
    return THC_CPD_OK;
}
