// FP64 kernels of THC-driven CP-ALS for GB300 (sm_103a).
//
// GB300 executes FP64 at roughly two DFMA per clock per SM (about 1 TFLOP/s for the
// chip), so these kernels are bound by the FP64 pipe, not by HBM: data stays L2
// resident (the 129 MB L2 holds every per-problem buffer of the paper-shaped
// workloads), tiles are small so that every SM gets work, and split-K with a
// fixed-order reduction keeps results deterministic.
#include <float.h>
#include <math.h>

#include <algorithm>

#include "f64.cuh"
#include "oz.cuh"
#include "ldl_common.cuh"
#include "prof.cuh"

namespace thc {

// ------------------------------------------------------------------------------------
// generic FP64 GEMM: C = op(A) (B o B2) [o E]
// ------------------------------------------------------------------------------------
template <int BM, int BN, int BK, int TM, int TN, bool TA, bool HADB, bool SYMM>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_dgemm(int M, int N, int K, const double* __restrict__ A, int lda,
        const double* __restrict__ B, const double* __restrict__ B2, int ldb,
        double* __restrict__ C, int ldc, const double* __restrict__ E,
        int kchunk, double* __restrict__ part) {
    constexpr int TX = BN / TN;
    constexpr int TY = BM / TM;
    constexpr int NT = TX * TY;
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;
    if (SYMM && by < bx) return;  // strictly upper tile of a symmetric result
    const int m0 = by * BM, n0 = bx * BN;
    const int kbeg = bz * kchunk;
    const int kend = min(K, kbeg + kchunk);
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    double acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        for (int idx = tid; idx < BM * BK; idx += NT) {
            int r, c;
            if (TA) { r = idx % BM; c = idx / BM; } else { r = idx / BK; c = idx % BK; }
            const int m = m0 + r, k = k0 + c;
            double val = 0.0;
            if (m < M && k < kend) val = TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
            As[c][r] = val;
        }
        for (int idx = tid; idx < BN * BK; idx += NT) {
            const int r = idx % BN, c = idx / BN;
            const int n = n0 + r, k = k0 + c;
            double val = 0.0;
            if (n < N && k < kend) {
                const size_t o = (size_t)k * ldb + n;
                val = B[o];
                if (HADB) val *= B2[o];
            }
            Bs[c][r] = val;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * TY];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + j * TX];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int m = m0 + ty + i * TY;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int n = n0 + tx + j * TX;
            if (n >= N) continue;
            if (part) {
                part[((size_t)bz * M + m) * N + n] = acc[i][j];
            } else {
                double val = acc[i][j];
                if (E) val *= E[(size_t)m * ldc + n];
                C[(size_t)m * ldc + n] = val;
                if (SYMM) C[(size_t)n * ldc + m] = val;
            }
        }
    }
}

__global__ void k_splitk_reduce(int M, int N, int splits, const double* __restrict__ part,
                                double* __restrict__ C, int ldc, const double* __restrict__ E,
                                int symm_tile) {
    const long total = (long)M * N;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total;
         idx += (long)gridDim.x * blockDim.x) {
        const int m = (int)(idx / N), n = (int)(idx % N);
        if (symm_tile > 0 && (m / symm_tile) < (n / symm_tile)) continue;
        double s = 0.0;
        for (int z = 0; z < splits; ++z) s += part[(size_t)z * total + idx];
        if (E) s *= E[(size_t)m * ldc + n];
        C[(size_t)m * ldc + n] = s;
        if (symm_tile > 0) C[(size_t)n * ldc + m] = s;
    }
}

// Symmetric C = A^T B (A, B: K x N row-major with leading dimension ld; the product is
// symmetric, e.g. a Gram matrix A^T A) on 32 x 32 tiles of the lower triangle, mirrored.
// Small tiles so that every SM gets a tile (a 720 x 720 Gram has 276 of them) and K is not
// split (no partials); the last K chunk runs only its valid columns. 256 threads, 2 x 2
// outputs each, fixed summation order.
constexpr int SYT = 32;
__global__ void __launch_bounds__(256)
k_dsyrk32(int N, int K, const double* __restrict__ A, const double* __restrict__ B, int ld,
          double* __restrict__ C, int ldc) {
    constexpr int BK = 16;
    __shared__ double As[BK][SYT + 1];
    __shared__ double Bs[BK][SYT + 1];
    // lower-triangle tile (ti, tj), tj <= ti, from the linear index
    const int t = blockIdx.x;
    int ti = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    if ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    if (ti * (ti + 1) / 2 > t) --ti;
    const int tj = t - ti * (ti + 1) / 2;
    const int m0 = ti * SYT, n0 = tj * SYT;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double c00 = 0.0, c01 = 0.0, c10 = 0.0, c11 = 0.0;
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int e = tid; e < BK * SYT; e += 256) {
            const int kk = e / SYT, r = e % SYT, k = k0 + kk;
            As[kk][r] = (k < K && m0 + r < N) ? A[(size_t)k * ld + m0 + r] : 0.0;
            Bs[kk][r] = (k < K && n0 + r < N) ? B[(size_t)k * ld + n0 + r] : 0.0;
        }
        __syncthreads();
        const int kn = min(BK, K - k0);
        if (kn == BK) {
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                const double a0 = As[kk][ty], a1 = As[kk][ty + 16];
                const double b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
                c00 = fma(a0, b0, c00);
                c01 = fma(a0, b1, c01);
                c10 = fma(a1, b0, c10);
                c11 = fma(a1, b1, c11);
            }
        } else {
            for (int kk = 0; kk < kn; ++kk) {
                const double a0 = As[kk][ty], a1 = As[kk][ty + 16];
                const double b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
                c00 = fma(a0, b0, c00);
                c01 = fma(a0, b1, c01);
                c10 = fma(a1, b0, c10);
                c11 = fma(a1, b1, c11);
            }
        }
        __syncthreads();
    }
    const double cv[2][2] = {{c00, c01}, {c10, c11}};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= N) continue;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n >= N) continue;
            C[(size_t)m * ldc + n] = cv[i][j];
            C[(size_t)n * ldc + m] = cv[i][j];
        }
    }
}

namespace {
struct GemmPlan {
    int BM, BN, splits, kchunk, tiles;
};

GemmPlan plan_gemm(int M, int N, int K, bool symm) {
    GemmPlan p;
    p.BN = 64;
    if (K <= 0) {
        p.BM = (!symm && M <= 32) ? 32 : 64;
        p.splits = 1;
        p.kchunk = 0;
        p.tiles = 1;
        return p;
    }
    p.BM = (!symm && M <= 32) ? 32 : 64;
    const int tm = cdiv(M, p.BM), tn = cdiv(N, p.BN);
    p.tiles = symm ? (tm * (tm + 1)) / 2 : tm * tn;
    // split K so that the busiest SM finishes first: the FP64 pipe of an SM is shared by
    // its CTAs, so the cost is (CTAs per SM, rounded up) x (K per CTA) plus a small charge
    // per split for the partials' write and fixed-order reduction
    int best_s = 1, best_kc = ((K + 15) / 16) * 16;
    double best = 1e300;
    for (int s = 1; s <= 32; ++s) {
        const int kc = ((cdiv(K, s) + 15) / 16) * 16;
        const int ss = cdiv(K, kc);
        if (ss != s) continue;
        const double waves = (double)cdiv((long)p.tiles * ss, num_sms());
        const double cost = waves * kc + (ss > 1 ? 0.5 * ss : 0.0);
        if (cost < best) {
            best = cost;
            best_s = ss;
            best_kc = kc;
        }
    }
    p.kchunk = best_kc;
    p.splits = best_s;
    return p;
}

template <int BM, bool TA, bool HADB, bool SYMM>
void launch_gemm(cudaStream_t st, const GemmPlan& p, int M, int N, int K, const double* A,
                 int lda, const double* B, const double* B2, int ldb, double* C, int ldc,
                 const double* E, double* part) {
    constexpr int BN = 64, BK = 16, TN = 4, TM = BM / 16;
    dim3 grid(cdiv(N, BN), cdiv(M, BM), p.splits);
    k_dgemm<BM, BN, BK, TM, TN, TA, HADB, SYMM><<<grid, (BM / TM) * (BN / TN), 0, st>>>(
        M, N, K, A, lda, B, B2, ldb, C, ldc, E, p.kchunk, p.splits > 1 ? part : nullptr);
}

template <int BM>
void dispatch_gemm(cudaStream_t st, const GemmPlan& p, bool ta, bool hadb, bool symm, int M,
                   int N, int K, const double* A, int lda, const double* B, const double* B2,
                   int ldb, double* C, int ldc, const double* E, double* part) {
#define THC_G(TA_, HB_, SY_)                                                              \
    if (ta == TA_ && hadb == HB_ && symm == SY_) {                                        \
        launch_gemm<BM, TA_, HB_, SY_>(st, p, M, N, K, A, lda, B, B2, ldb, C, ldc, E, part); \
        return;                                                                           \
    }
    THC_G(false, false, false)
    THC_G(false, true, false)
    THC_G(true, false, false)
    THC_G(true, true, false)
    THC_G(true, false, true)
    THC_G(false, false, true)
#undef THC_G
}
}  // namespace

size_t dgemm_part_need(int M, int N, int K) {
    GemmPlan p = plan_gemm(M, N, K, false);
    GemmPlan q = plan_gemm(M, N, K, true);
    size_t a = p.splits > 1 ? (size_t)p.splits * M * N : 0;
    size_t b = q.splits > 1 ? (size_t)q.splits * M * N : 0;
    return std::max(a, b);
}

void dgemm(cudaStream_t st, bool trans_a, int M, int N, int K, const double* A, int lda,
           const double* B, const double* B2, int ldb, double* C, int ldc, const double* E,
           bool symm, double* part, size_t part_cap) {
    if (M <= 0 || N <= 0) return;
    GemmPlan p = plan_gemm(M, N, K, symm);
    if (p.splits > 1 && (size_t)p.splits * M * N > part_cap) {
        p.splits = 1;
        p.kchunk = K;
    }
    if (K <= 0) {  // empty contraction: C = 0
        p.splits = 1;
        p.kchunk = 0;
    }
    const bool hadb = B2 != nullptr;
    ProfScope prof(st, KC_DGEMM, (symm ? 1.0 : 2.0) * M * (double)N * K);
    if (symm && trans_a && !hadb && !E && M == N && lda == ldb && K > 0) {
        const int nt = cdiv(N, SYT);
        count_launch();
        k_dsyrk32<<<nt * (nt + 1) / 2, 256, 0, st>>>(N, K, A, B, lda, C, ldc);
        return;
    }
    count_launch(p.splits > 1 ? 2 : 1);
    if (p.BM == 32)
        dispatch_gemm<32>(st, p, trans_a, hadb, symm, M, N, K, A, lda, B, B2, ldb, C, ldc, E, part);
    else
        dispatch_gemm<64>(st, p, trans_a, hadb, symm, M, N, K, A, lda, B, B2, ldb, C, ldc, E, part);
    if (p.splits > 1) {
        const long total = (long)M * N;
        int blocks = (int)std::min<long>(cdiv(total, 256), 4L * num_sms());
        k_splitk_reduce<<<blocks, 256, 0, st>>>(M, N, p.splits, part, C, ldc, E, symm ? p.BM : 0);
    }
}

// ------------------------------------------------------------------------------------
// Hadamard product of three Gram matrices (the ALS normal matrix) + max diagonal
// ------------------------------------------------------------------------------------
__device__ double block_reduce_sum(double v, double* sh) {
    // fixed-order reduction: warp shuffles then one warp over the partials
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    return v;  // valid in thread 0
}

__device__ double block_reduce_max(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    __syncthreads();
    return v;
}

__global__ void k_hadamard3(int R, const double* __restrict__ Ga, const double* __restrict__ Gb,
                            const double* __restrict__ Gc, double* __restrict__ H,
                            DevScalars* sc) {
    const long n = (long)R * R;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
         i += (long)gridDim.x * blockDim.x)
        H[i] = Ga[i] * Gb[i] * Gc[i];
    if (blockIdx.x == 0) {
        __shared__ double sh[32];
        double mx = 0.0;
        for (int i = threadIdx.x; i < R; i += blockDim.x) {
            const size_t d = (size_t)i * R + i;
            mx = fmax(mx, Ga[d] * Gb[d] * Gc[d]);
        }
        mx = block_reduce_max(mx, sh);
        if (threadIdx.x == 0) sc->maxdiag = mx;
    }
}

void hadamard3(cudaStream_t st, int R, const double* Ga, const double* Gb, const double* Gc,
               double* H, DevScalars* sc) {
    const long n = (long)R * R;
    int blocks = (int)std::min<long>(cdiv(n, 256), 4L * num_sms());
    ProfScope prof(st, KC_AUX, 2.0 * n, 32.0 * n);
    count_launch();
    k_hadamard3<<<blocks, 256, 0, st>>>(R, Ga, Gb, Gc, H, sc);
}

__global__ void k_copy_maxdiag(int R, const double* __restrict__ H, double* __restrict__ out,
                               DevScalars* sc) {
    const long n = (long)R * R;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
         i += (long)gridDim.x * blockDim.x)
        out[i] = H[i];
    if (blockIdx.x == 0) {
        __shared__ double sh[32];
        double mx = 0.0;
        for (int i = threadIdx.x; i < R; i += blockDim.x) mx = fmax(mx, H[(size_t)i * R + i]);
        mx = block_reduce_max(mx, sh);
        if (threadIdx.x == 0) sc->maxdiag = mx;
    }
}

void copy_with_maxdiag(cudaStream_t st, int R, const double* H, double* H_out, DevScalars* sc) {
    const long n = (long)R * R;
    int blocks = (int)std::min<long>(cdiv(n, 256), 4L * num_sms());
    count_launch();
    k_copy_maxdiag<<<blocks, 256, 0, st>>>(R, H, H_out, sc);
}

// ------------------------------------------------------------------------------------
// Solve of the ALS normal equations A H = M: blocked right-looking LDL^T factorisation
// of H (the square-root-free form of the Cholesky factorisation, same pivots) with the
// M rows carried along as extra rows, so that the forward solve is fused into the
// factorisation (this file: the blocked variant, one launch per 32-column step; the
// dataflow variant and the backward solve with the unit lower factor are in ldl_flow.cu).
//
// GB300 issues one FP64 warp-instruction per SM sub-partition every 64 clocks, whatever
// the number of active lanes, and FP64 divide / sqrt cost 400-700 clocks. So the
// sequential part (one pivot per column) uses a single Newton-Raphson reciprocal per
// pivot and no sqrt or divide; row substitutions run one row per warp with the
// column values passed by shuffles.
//
//   H = L D L^T (L unit lower).  For the appended rows B = M: after elimination they
//   hold Y = M L^{-T} D^{-1}; then A = Y L^{-1} by the backward solve (unit L).
//   Storage after the factorisation: strictly-lower L and diag(D) in H, D^{-1} in dinv,
//   Y in the appended rows; P (R x 32) holds the unscaled panel X = L D of the current
//   block column for the trailing update.
// ------------------------------------------------------------------------------------
constexpr int NB = 32;          // block size of the factorisation
constexpr int UT = 16;          // trailing-update tile (one output per thread)

struct BlockSmem {
    double Ds[NB][NB + 1];
    double Ls[NB][NB + 1];
    double dinv[NB];
    unsigned short pairs[NB * (NB + 1) / 2];
    int bad;
};

// LDL^T of the jb x jb diagonal block at (j0, j0) of H, in place: strictly lower L, D on the
// diagonal, D^-1 in dinv[j0..]; a pivot <= tau sets bit `mode` of sc->fail_mask. Called by
// every thread of the CTA (barriers inside); threads 0..127 compute: thread 0 carries the
// pivot chain one column ahead (pivot update and its reciprocal), warps 1-3 apply the
// current column to the rest of the block over a packed pair list, one barrier per column.
// Loads go through L2 (__ldcg): other CTAs of the same kernel may have written the block.
__device__ void factor_block(double* __restrict__ H, int R, int j0, int jb,
                             double* __restrict__ dinv, DevScalars* sc, int mode, BlockSmem& S) {
    const int tid = threadIdx.x;
    const double tau = (double)R * DBL_EPSILON * sc->maxdiag;
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        const int r = e / NB, c = e % NB;
        S.Ds[r][c] = (r < jb && c <= r) ? __ldcg(H + (size_t)(j0 + r) * R + j0 + c) : 0.0;
        S.Ls[r][c] = (r == c) ? 1.0 : 0.0;
    }
    for (int e = tid; e < NB * (NB + 1) / 2; e += blockDim.x) S.pairs[e] = pair_code<NB>(e);
    __syncthreads();
    if (tid == 0) {
        S.bad = 0;
        double d = S.Ds[0][0];
        if (!pivot_ok(d, tau)) {
            S.bad = 1;
            d = 1.0;  // keep going; the caller replays this mode with the pseudo-inverse
            S.Ds[0][0] = d;
        }
        S.dinv[0] = recip_nr(d);
    }
    for (int c = 0; c < jb; ++c) {
        __syncthreads();  // dinv[c] and column c of D are final
        const double inv = S.dinv[c];
        if (tid == 0) {
            if (c + 1 < jb) {
                const double x = S.Ds[c + 1][c];
                const double l = x * inv;
                double d1 = fma(-l, x, S.Ds[c + 1][c + 1]);
                S.Ls[c + 1][c] = l;
                if (!pivot_ok(d1, tau)) {
                    S.bad = 1;
                    d1 = 1.0;
                }
                S.Ds[c + 1][c + 1] = d1;
                S.dinv[c + 1] = recip_nr(d1);
            }
        } else if (tid >= 32 && tid < 128) {
            // D[r][s] -= (D[r][c] / d_c) D[s][c] for c < s <= r < jb except (c+1, c+1)
            const int hi = NB - 1 - c;
            const int npair = hi * (hi + 1) / 2;
            for (int e = tid - 32; e < npair; e += 96) {
                const int rs = S.pairs[e];
                const int r = rs >> 8, ss = rs & 0xFF;
                if (r >= jb || (r == c + 1 && ss == c + 1)) continue;
                const double l = S.Ds[r][c] * inv;
                if (ss == c + 1) S.Ls[r][c] = l;
                S.Ds[r][ss] = fma(-l, S.Ds[ss][c], S.Ds[r][ss]);
            }
        }
    }
    __syncthreads();
    if (tid == 0 && S.bad) atomicOr(&sc->fail_mask, 1 << mode);
    for (int e = tid; e < jb * jb; e += blockDim.x) {
        const int r = e / jb, c = e % jb;
        if (c < r) H[(size_t)(j0 + r) * R + j0 + c] = S.Ls[r][c];
        else if (c == r) H[(size_t)(j0 + r) * R + j0 + c] = S.Ds[r][r];
    }
    if (tid < jb) dinv[j0 + tid] = S.dinv[tid];
}

// First diagonal block; also clears the per-step arrival counters of the update kernels.
__global__ void __launch_bounds__(128)
k_ldl_diag(double* __restrict__ H, double* __restrict__ dinv, int R, int jb, DevScalars* sc,
           int mode, int* counters, int nsteps) {
    __shared__ BlockSmem S;
    for (int i = threadIdx.x; i < nsteps; i += blockDim.x) counters[i] = 0;
    factor_block(H, R, 0, jb, dinv, sc, mode, S);
}

// Panel rows below block j (rows of H and the appended rows), one per warp: unit-triangular
// substitution X L_jj^T = B with the column values passed by shuffles, then L = X D^-1;
// X goes to P for the trailing update (rows of H only).
__global__ void __launch_bounds__(128)
k_ldl_subst(double* __restrict__ H, double* __restrict__ P, const double* __restrict__ dinv,
            int R, int nrows, int j0, int jb) {
    __shared__ double Lj[NB][NB + 1];
    __shared__ double di[NB];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int i = j0 + jb + blockIdx.x * 4 + w;
    double b = (i < nrows && lane < jb) ? H[(size_t)i * R + j0 + lane] : 0.0;
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        const int r = e / NB, c = e % NB;
        Lj[r][c] = (r < jb && c < r) ? H[(size_t)(j0 + r) * R + j0 + c] : 0.0;
    }
    if (tid < NB) di[tid] = tid < jb ? dinv[j0 + tid] : 0.0;
    __syncthreads();
    if (i >= nrows) return;
    for (int c = 0; c + 1 < jb; ++c) {
        const double xc = __shfl_sync(0xffffffffu, b, c);
        if (lane > c) b = fma(-xc, Lj[lane][c], b);
    }
    if (lane < jb) {
        H[(size_t)i * R + j0 + lane] = b * di[lane];
        if (i < R) P[(size_t)i * NB + lane] = b;
    }
}

// Trailing update H[i][c] -= sum_s L[i][j0+s] X[c][s] for i >= j1 (rows of H and of the
// appended M block), j1 <= c < R, lower triangle only for rows of H. One output per thread
// on 16 x 16 tiles, so that the late (small) steps still spread over the SMs. The tiles
// that cover the next diagonal block count their arrivals (fence + atomic); the last one to
// arrive factorises that block while the rest of the update is still running, so the
// factorisation leaves the critical path of the step. No CTA ever waits for another.
__global__ void __launch_bounds__(256)
k_ldl_update(double* __restrict__ H, const double* __restrict__ P, double* __restrict__ dinv,
             int R, int nrows, int j0, int jb, int nHtiles, DevScalars* sc, int mode,
             int* counter) {
    const int j1 = j0 + jb;
    int r0, rend;
    if ((int)blockIdx.y < nHtiles) {
        r0 = j1 + blockIdx.y * UT;
        rend = min(R, r0 + UT);
    } else {
        r0 = R + (blockIdx.y - nHtiles) * UT;
        rend = min(nrows, r0 + UT);
    }
    const int c0 = j1 + blockIdx.x * UT;
    if (c0 >= R || r0 >= rend) return;
    const bool hrows = r0 < R;
    if (hrows && c0 > rend - 1) return;  // tile strictly above the diagonal
    __shared__ double As[UT][NB + 1];
    __shared__ double Bs[UT][NB + 1];
    const int tid = threadIdx.x;
    for (int e = tid; e < UT * NB; e += 256) {
        const int r = e / NB, s = e % NB;
        As[r][s] = (r0 + r < rend && s < jb) ? H[(size_t)(r0 + r) * R + j0 + s] : 0.0;
        Bs[r][s] = (c0 + r < R && s < jb) ? P[(size_t)(c0 + r) * NB + s] : 0.0;
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
    const int row = r0 + ty, col = c0 + tx;
    if (row < rend && col < R && !(hrows && col > row)) {
        double a0 = 0.0, a1 = 0.0;
#pragma unroll
        for (int s = 0; s < NB; s += 2) {
            a0 = fma(As[ty][s], Bs[tx][s], a0);
            a1 = fma(As[ty][s + 1], Bs[tx][s + 1], a1);
        }
        H[(size_t)row * R + col] -= (a0 + a1);
    }
    // next diagonal block: rows and columns [j1, j1 + jbn)
    const int jbn = min(NB, R - j1);
    const int kt = (jbn + UT - 1) / UT;  // tiles per side of the block
    if (!(hrows && (int)blockIdx.y < kt && (int)blockIdx.x < kt)) return;
    __shared__ int last;
    __threadfence();  // this tile's writes before the arrival count
    __syncthreads();
    if (tid == 0) last = (atomicAdd(counter, 1) == kt * (kt + 1) / 2 - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ BlockSmem S;
    factor_block(H, R, j1, jbn, dinv, sc, mode, S);
}

// Column where a block of m columns of the backward solve of an emulated factorisation
// splits (0: it does not). With n >= 128 right-hand sides the solve is bound by the FP64
// pipe, so the coupling between the two halves (half of the block's flops) goes to the
// tensor cores; with fewer it is bound by each row's substitution chain, which a split only
// lengthens. Blocks of fewer than 768 columns are not split (their coupling products are
// too small to fill the GPU). Measured on GB300, BF16x3 sweeps/s at (o, v, R_cp) = (50,
// 250, 1800): 110.0 unsplit, 116.3 halves, 118.5 quarters, 118.4 eighths (116.7 with the
// o modes split as well, n = 50: 114.9); at (30, 150, 1080): 232.9 halves, 230.5 quarters.
constexpr int kBsSplitMinN = 128;
constexpr int kBsSplitMinCols = 6 * kOzPanel;
int bsolve_split_point(int m, int n) {
    if (n < kBsSplitMinN || m < kBsSplitMinCols) return 0;
    return (m / 2 / kOzPanel) * kOzPanel;
}

void chol_solve(cudaStream_t st, int R, int n, double* Haug, double* A, double* P, double* dinv,
                DevScalars* sc, int mode, int* counters, int* flow_sync, int flow_ctas,
                int* bs_sync, const OzWs* oz) {
    NvtxRange nvtx_range("thc_cpd LDL^T and solve");
    const int nrows = R + n;
    const int nJ = cdiv(R, NB);
    if (oz && flow_sync) {
        ldl_oz(st, R, n, Haug, P, dinv, sc, mode, flow_sync, *oz, flow_ctas);
    } else if (flow_sync && flow_prepare(R, n)) {
        ProfScope prof(st, KC_CHOL, (double)R * R * R / 3.0 + (double)n * R * R);
        ldl_flow(st, R, n, Haug, P, dinv, sc, mode, flow_sync, flow_ctas);
    } else {
        ProfScope prof(st, KC_CHOL, (double)R * R * R / 3.0 + (double)n * R * R);
        k_ldl_diag<<<1, 128, 0, st>>>(Haug, dinv, R, std::min(NB, R), sc, mode, counters, nJ);
        count_launch();
        for (int j0 = 0, step = 0; j0 < R; j0 += NB, ++step) {
            const int jb = std::min(NB, R - j0);
            const int j1 = j0 + jb;
            const int below = nrows - j1;
            if (below > 0) {
                k_ldl_subst<<<cdiv(below, 4), 128, 0, st>>>(Haug, P, dinv, R, nrows, j0, jb);
                count_launch();
            }
            if (j1 < R) {
                const int nH = cdiv(R - j1, UT);
                dim3 grid(cdiv(R - j1, UT), nH + cdiv(n, UT));
                k_ldl_update<<<grid, 256, 0, st>>>(Haug, P, dinv, R, nrows, j0, jb, nH, sc, mode,
                                                   counters + step);
                count_launch();
            }
        }
    }
    backward_solve(st, R, n, Haug, A, bs_sync, oz);
}

namespace {
// Columns [c0, c0 + m) of A L = Y (L, Y, A with row pitch R), the columns after them already
// applied to Y: the block as one solve, or split at h into its trailing and leading parts
// with the coupling Y[:, c0 .. c0 + h) -= A[:, c0 + h .. c0 + m) L[c0 + h .. c0 + m, c0 .. c0 + h)
// as an emulated product between them.
void bsolve_block(cudaStream_t st, int R, int c0, int m, int n, double* Haug, double* A, int* bs_sync,
                  const OzWs* oz) {
    double* Y = Haug + (size_t)R * R;
    const int h = oz ? bsolve_split_point(m, n) : 0;
    if (h == 0) {
        ProfScope prof(st, KC_BSOLVE, (double)n * m * m);
        bsolve_slices(st, m, n, Y + c0, A + c0, Haug + (size_t)c0 * R + c0, bs_sync, R);
        return;
    }
    bsolve_block(st, R, c0 + h, m - h, n, Haug, A, bs_sync, oz);
    oz_gemm_sub(st, n, h, m - h, A + c0 + h, R, Haug + (size_t)(c0 + h) * R + c0, R, Y + c0, R, *oz);
    bsolve_block(st, R, c0, h, n, Haug, A, bs_sync, oz);
}
}  // namespace

namespace {
void coupling_rows(int m, int n, long* ra, long* rb, long* part) {
    const int h = bsolve_split_point(m, n);
    if (h == 0) return;
    const long nch = cdiv(m - h, kOzPanel);
    *ra = std::max(*ra, nch * n);
    *rb = std::max(*rb, nch * h);
    // the K groups oz_gemm_sub forms for an n x h product (128 x 32 tiles)
    const long tiles = (long)cdiv(n, 128) * cdiv(h, 32);
    const long groups = std::min<long>(nch, std::max<long>(1, num_sms() / tiles));
    *part = std::max(*part, (groups - 1) * n * (long)h);
    coupling_rows(m - h, n, ra, rb, part);
    coupling_rows(h, n, ra, rb, part);
}
}  // namespace

void bsolve_ws_rows(int R, int nmax, int* rowsA, int* rowsB, size_t* part_doubles) {
    long ra = 0, rb = 0, part = 0;
    coupling_rows(R, nmax, &ra, &rb, &part);
    *rowsA = std::max<long>(*rowsA, ra);
    *rowsB = std::max<long>(*rowsB, rb);
    *part_doubles = std::max<size_t>(*part_doubles, (size_t)part);
}

void backward_solve(cudaStream_t st, int R, int n, double* Haug, double* A, int* bs_sync, const OzWs* oz) {
    NvtxRange nvtx_range("thc_cpd backward solve");
    if (n <= 0) return;
    // A = [A1 A2], L = [L11 0; L21 L22]: A2 L22 = Y2, then A1 L11 = Y1 - A2 L21 with the
    // coupling term (half of the block's flops) as an emulated tensor-core product, each
    // half split again while it is large enough
    bsolve_block(st, R, 0, R, n, Haug, A, bs_sync, oz);
}

// ------------------------------------------------------------------------------------
// column normalisation, loss, norms
// ------------------------------------------------------------------------------------
// lam_r = ||A[:, r]||_2 (32 columns x 8 row slices per block, fixed-order reduction) and
// the reciprocal, then A[:, r] *= 1 / lam_r by the same block (it owns its 32 columns over
// all rows): one sqrt and one divide per column instead of a divide per element (a divide
// costs ~430 clocks on GB300's FP64 pipe), one launch per normalisation.
__global__ void __launch_bounds__(256)
k_colnorm(int n, int R, double* __restrict__ A, double* __restrict__ lam) {
    __shared__ double sh[8][33];
    __shared__ double inv[32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int r = blockIdx.x * 32 + tx;
    double s = 0.0;
    if (r < R)
        for (int i = ty; i < n; i += 8) {
            const double x = A[(size_t)i * R + r];
            s = fma(x, x, s);
        }
    sh[ty][tx] = s;
    __syncthreads();
    if (ty == 0) {
        double f = 1.0;
        if (r < R) {
            double t = 0.0;
            for (int k = 0; k < 8; ++k) t += sh[k][tx];
            const double l = sqrt(t);
            lam[r] = l;
            f = l > 0.0 ? 1.0 / l : 1.0;  // zero columns are left as they are
        }
        inv[tx] = f;
    }
    __syncthreads();
    if (r < R) {
        const double f = inv[tx];
        for (int i = ty; i < n; i += 8) A[(size_t)i * R + r] *= f;
    }
}

void normalise_columns(cudaStream_t st, int n, int R, double* A, double* lam, double* scratch) {
    (void)scratch;
    ProfScope prof(st, KC_AUX, 3.0 * n * R, 24.0 * n * R);
    count_launch(1);
    k_colnorm<<<cdiv(R, 32), 256, 0, st>>>(n, R, A, lam);
}

struct CopyMany {
    const double* src[8];
    double* dst[8];
    long len[8];
    int np;
};

__global__ void __launch_bounds__(256) k_copy_many(CopyMany a) {
    const long stride = (long)gridDim.x * blockDim.x;
    for (int p = 0; p < a.np; ++p)
        for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < a.len[p]; i += stride)
            a.dst[p][i] = a.src[p][i];
}

cudaError_t copy_many(cudaStream_t st, int np, const double* const* src, double* const* dst,
                      const long* len) {
    if (np < 1 || np > 8) return cudaErrorInvalidValue;
    CopyMany a{};
    long total = 0;
    for (int p = 0; p < np; ++p) {
        a.src[p] = src[p];
        a.dst[p] = dst[p];
        a.len[p] = len[p];
        total += len[p];
    }
    a.np = np;
    count_launch();
    k_copy_many<<<(int)std::max<long>(1, std::min<long>(cdiv(total, 256), 2L * num_sms())), 256, 0, st>>>(a);
    return cudaGetLastError();
}

constexpr int RED_BLOCKS = kReduceBlocks;
constexpr int RED_THREADS = 256;

size_t loss_red_need() { return 2 * RED_BLOCKS; }

__global__ void __launch_bounds__(RED_THREADS)
k_loss_partials(int Rt, int R, const double* __restrict__ Y, const double* __restrict__ W3,
                const double* __restrict__ W4, const double* __restrict__ lam,
                const double* __restrict__ G1, const double* __restrict__ G2,
                const double* __restrict__ G3, const double* __restrict__ G4,
                double* __restrict__ red) {
    __shared__ double sh[32];
    const long stride = (long)gridDim.x * blockDim.x;
    const long g = blockIdx.x * (long)blockDim.x + threadIdx.x;
    double s1 = 0.0, s2 = 0.0;
    const long n1 = (long)Rt * R;
    for (long i = g; i < n1; i += stride) {
        const int r = (int)(i % R);
        s1 = fma(lam[r] * Y[i], W3[i] * W4[i], s1);
    }
    const long n2 = (long)R * R;
    for (long i = g; i < n2; i += stride) {
        const int r = (int)(i / R), c = (int)(i % R);
        s2 = fma(lam[r] * lam[c], G1[i] * G2[i] * G3[i] * G4[i], s2);
    }
    s1 = block_reduce_sum(s1, sh);
    s2 = block_reduce_sum(s2, sh);
    if (threadIdx.x == 0) {
        red[2 * blockIdx.x] = s1;
        red[2 * blockIdx.x + 1] = s2;
    }
}

__global__ void __launch_bounds__(RED_THREADS)
k_loss_final(const double* __restrict__ red, int nb, DevScalars* sc, double tol) {
    __shared__ double sh[32];
    double s1 = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        s1 += red[2 * i];
        s2 += red[2 * i + 1];
    }
    s1 = block_reduce_sum(s1, sh);
    s2 = block_reduce_sum(s2, sh);
    if (threadIdx.x == 0) {
        const double nG2 = sc->normG2;
        const double loss = nG2 - 2.0 * s1 + s2;
        const double fit = 1.0 - sqrt(fmax(loss, 0.0)) / sqrt(nG2);
        sc->inner = s1;
        sc->cpdn2 = s2;
        sc->loss = loss;
        if (!isfinite(loss)) sc->nonfinite = 1;
        const double prev = sc->prev_fit;
        if (tol > 0.0 && isfinite(prev) && fabs(fit - prev) < tol) sc->done = 1;
        sc->prev_fit = fit;
        sc->fit = fit;
    }
}

void loss_eval(cudaStream_t st, int Rt, int R, const double* Y, const double* W3,
               const double* W4, const double* lam, const double* const G[4], double* red,
               DevScalars* sc, double tol) {
    ProfScope prof(st, KC_AUX, 4.0 * Rt * R + 6.0 * R * R, 24.0 * Rt * R + 32.0 * R * R);
    count_launch(2);
    k_loss_partials<<<RED_BLOCKS, RED_THREADS, 0, st>>>(Rt, R, Y, W3, W4, lam, G[0], G[1],
                                                         G[2], G[3], red);
    k_loss_final<<<1, RED_THREADS, 0, st>>>(red, RED_BLOCKS, sc, tol);
}

__global__ void __launch_bounds__(RED_THREADS)
k_sumprod_partials(long n, const double* __restrict__ a, const double* __restrict__ b,
                   double* __restrict__ red) {
    __shared__ double sh[32];
    const long stride = (long)gridDim.x * blockDim.x;
    double s = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += stride)
        s = fma(a[i], b[i], s);
    s = block_reduce_sum(s, sh);
    if (threadIdx.x == 0) red[blockIdx.x] = s;
}

__global__ void __launch_bounds__(RED_THREADS)
k_norm_final(const double* __restrict__ red, int nb, DevScalars* sc) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += red[i];
    s = block_reduce_sum(s, sh);
    if (threadIdx.x == 0) sc->normG2 = s;
}

void sum_hadamard_normG2(cudaStream_t st, long n, const double* Z, const double* U,
                         double* red, DevScalars* sc) {
    ProfScope prof(st, KC_AUX, 2.0 * n, 16.0 * n);
    count_launch(2);
    k_sumprod_partials<<<RED_BLOCKS, RED_THREADS, 0, st>>>(n, Z, U, red);
    k_norm_final<<<1, RED_THREADS, 0, st>>>(red, RED_BLOCKS, sc);
}

// out (cols x rows) = in (rows x cols)^T through 32 x 32 shared-memory tiles
__global__ void k_transpose(int rows, int cols, const double* __restrict__ in, double* __restrict__ out) {
    __shared__ double t[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int k = ty; k < 32; k += 8) {
        const int r = r0 + k, c = c0 + tx;
        if (r < rows && c < cols) t[k][tx] = in[(size_t)r * cols + c];
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int c = c0 + k, r = r0 + tx;
        if (r < rows && c < cols) out[(size_t)c * rows + r] = t[tx][k];
    }
}

void transpose64(cudaStream_t st, int rows, int cols, const double* in, double* out) {
    if (rows <= 0 || cols <= 0) return;
    count_launch();
    k_transpose<<<dim3(cdiv(cols, 32), cdiv(rows, 32)), 256, 0, st>>>(rows, cols, in, out);
}

__global__ void k_scalars_init(DevScalars* sc, double normG2) {
    sc->normG2 = normG2;
    sc->loss = nan("");
    sc->fit = nan("");
    sc->inner = 0.0;
    sc->cpdn2 = 0.0;
    sc->prev_fit = nan("");
    sc->maxdiag = 0.0;
    sc->fail_mask = 0;
    sc->done = 0;
    sc->nonfinite = 0;
}

void scalars_init(cudaStream_t st, DevScalars* sc, double normG2) {
    count_launch();
    k_scalars_init<<<1, 1, 0, st>>>(sc, normG2);
}

__global__ void k_fill(double* p, long n, double v) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
         i += (long)gridDim.x * blockDim.x)
        p[i] = v;
}

void fill(cudaStream_t st, double* p, long n, double v) {
    if (n <= 0) return;
    count_launch();
    k_fill<<<(int)std::min<long>(cdiv(n, 256), 1024), 256, 0, st>>>(p, n, v);
}

}  // namespace thc

namespace thc {

// ---- learned extrapolation helpers (FP64) --------------------------------------------
// Factors with lam absorbed into the last mode: X = A (k < 3) or A diag(lam) (k = 3).
__global__ void __launch_bounds__(RED_THREADS)
k_change_partials(long n, int R, const double* __restrict__ An, const double* __restrict__ Ao,
                  const double* __restrict__ ln, const double* __restrict__ lo, int absorb,
                  double* __restrict__ red) {
    __shared__ double sh[32];
    double num = 0.0, den = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i % R);
        const double a = absorb ? An[i] * ln[r] : An[i];
        const double b = absorb ? Ao[i] * lo[r] : Ao[i];
        num = fma(a - b, a - b, num);
        den = fma(a, a, den);
    }
    num = block_reduce_sum(num, sh);
    den = block_reduce_sum(den, sh);
    if (threadIdx.x == 0) {
        red[2 * blockIdx.x] = num;
        red[2 * blockIdx.x + 1] = den;
    }
}

__global__ void __launch_bounds__(RED_THREADS)
k_change_final(const double* __restrict__ red, int nb, double* __restrict__ out) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a += red[2 * i];
        b += red[2 * i + 1];
    }
    a = block_reduce_sum(a, sh);
    b = block_reduce_sum(b, sh);
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
    }
}

void change_norm(cudaStream_t st, int n, int R, const double* An, const double* Ao,
                 const double* ln, const double* lo, bool absorb, double* red, double* out2) {
    const int nb = 64;
    k_change_partials<<<nb, RED_THREADS, 0, st>>>((long)n * R, R, An, Ao, ln, lo, absorb ? 1 : 0, red);
    k_change_final<<<1, RED_THREADS, 0, st>>>(red, nb, out2);
    count_launch(2);
}

// T = P + alpha (N - P) on lam-absorbed factors
__global__ void k_trial(long n, int R, const double* __restrict__ An, const double* __restrict__ Ao,
                        const double* __restrict__ ln, const double* __restrict__ lo, int absorb,
                        double alpha, double* __restrict__ T) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i % R);
        const double a = absorb ? An[i] * ln[r] : An[i];
        const double b = absorb ? Ao[i] * lo[r] : Ao[i];
        T[i] = fma(alpha, a - b, b);
    }
}

void trial_point(cudaStream_t st, int n, int R, const double* An, const double* Ao,
                 const double* ln, const double* lo, bool absorb, double alpha, double* T) {
    const long N = (long)n * R;
    k_trial<<<(int)std::min<long>(cdiv(N, 256), 4L * num_sms()), 256, 0, st>>>(N, R, An, Ao, ln, lo,
                                                                           absorb ? 1 : 0, alpha, T);
    count_launch();
}

__global__ void k_lam_product(int R, const double* a, const double* b, const double* c,
                              const double* d, double* out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R) out[r] = a[r] * b[r] * c[r] * d[r];
}

void lam_product(cudaStream_t st, int R, const double* const l[4], double* out) {
    k_lam_product<<<cdiv(R, 128), 128, 0, st>>>(R, l[0], l[1], l[2], l[3], out);
    count_launch();
}

}  // namespace thc
