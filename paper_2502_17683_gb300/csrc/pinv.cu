// Pseudo-inverse fallback of the ALS normal equations on the GPU (FP64):
// cyclic Jacobi eigendecomposition of the symmetric normal matrix with the
// round-robin (tournament) pair ordering, so that each round applies R/2 disjoint
// rotations in parallel; then A = M V diag(w+) V^T with eigenvalues at or below
// R * eps * max|w| dropped. Only used when the Cholesky meets a non-positive pivot,
// so it favours simplicity over speed.
#include <float.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "f64.cuh"
#include "prof.cuh"

namespace thc {

__device__ __forceinline__ void rr_pair(int Rp, int round, int i, int* p, int* q) {
    // players 0..Rp-1 (Rp even); player 0 fixed, the others rotate by `round`
    auto pos = [&](int k) { return k == 0 ? 0 : 1 + ((k - 1 + round) % (Rp - 1)); };
    int a = pos(i), b = pos(Rp - 1 - i);
    *p = min(a, b);
    *q = max(a, b);
}

__global__ void k_jacobi_angles(const double* __restrict__ H, int R, int Rp, int round,
                                double* __restrict__ cs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Rp / 2) return;
    int p, q;
    rr_pair(Rp, round, i, &p, &q);
    double c = 1.0, s = 0.0;
    if (q < R) {
        const double app = H[(size_t)p * R + p], aqq = H[(size_t)q * R + q];
        const double apq = H[(size_t)p * R + q];
        if (apq != 0.0 && isfinite(apq)) {
            const double theta = (aqq - app) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
        }
    }
    cs[2 * i] = c;
    cs[2 * i + 1] = s;
}

// rows p, q of H <- P^T H (all columns)
__global__ void k_jacobi_rows(double* __restrict__ H, int R, int Rp, int round,
                              const double* __restrict__ cs) {
    const int i = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= R) return;
    int p, q;
    rr_pair(Rp, round, i, &p, &q);
    if (q >= R) return;
    const double c = cs[2 * i], s = cs[2 * i + 1];
    const double hp = H[(size_t)p * R + j], hq = H[(size_t)q * R + j];
    H[(size_t)p * R + j] = c * hp - s * hq;
    H[(size_t)q * R + j] = s * hp + c * hq;
}

// columns p, q of H and V <- H P, V P (all rows)
__global__ void k_jacobi_cols(double* __restrict__ H, double* __restrict__ V, int R, int Rp,
                              int round, const double* __restrict__ cs) {
    const int i = blockIdx.y;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    int p, q;
    rr_pair(Rp, round, i, &p, &q);
    if (q >= R) return;
    const double c = cs[2 * i], s = cs[2 * i + 1];
    double hp = H[(size_t)r * R + p], hq = H[(size_t)r * R + q];
    H[(size_t)r * R + p] = c * hp - s * hq;
    H[(size_t)r * R + q] = s * hp + c * hq;
    hp = V[(size_t)r * R + p];
    hq = V[(size_t)r * R + q];
    V[(size_t)r * R + p] = c * hp - s * hq;
    V[(size_t)r * R + q] = s * hp + c * hq;
}

__global__ void k_identity(double* V, int R) {
    const long n = (long)R * R;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
         i += (long)gridDim.x * blockDim.x)
        V[i] = (i / R == i % R) ? 1.0 : 0.0;
}

// off = sum_{i != j} H_ij^2, tot = sum H_ij^2 (single block, fixed order)
__global__ void k_offnorm(const double* __restrict__ H, int R, double* out) {
    __shared__ double s1[256], s2[256];
    double a = 0.0, b = 0.0;
    const long n = (long)R * R;
    for (long i = threadIdx.x; i < n; i += blockDim.x) {
        const double x = H[i];
        b = fma(x, x, b);
        if (i / R != i % R) a = fma(x, x, a);
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = s1[0];
        out[1] = s2[0];
    }
}

// w_k = H_kk; inv_k = 1/w_k if w_k > R eps max|w| else 0 (single block)
__global__ void k_eig_inv(const double* __restrict__ H, int R, double* __restrict__ w) {
    __shared__ double sh[256];
    double m = 0.0;
    for (int i = threadIdx.x; i < R; i += blockDim.x) m = fmax(m, fabs(H[(size_t)i * R + i]));
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    const double cut = (double)R * DBL_EPSILON * sh[0];
    for (int i = threadIdx.x; i < R; i += blockDim.x) {
        const double d = H[(size_t)i * R + i];
        w[i] = (d > cut) ? 1.0 / d : 0.0;
    }
}

// A[i][j] = sum_k T[i][k] w[k] V[j][k]
__global__ void k_pinv_apply(const double* __restrict__ T, const double* __restrict__ w,
                             const double* __restrict__ V, double* __restrict__ A, int n, int R) {
    const int i = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= R || i >= n) return;
    double s = 0.0;
    for (int k = 0; k < R; ++k) s = fma(T[(size_t)i * R + k] * w[k], V[(size_t)j * R + k], s);
    A[(size_t)i * R + j] = s;
}

cudaError_t pinv_solve(cudaStream_t st, int R, int n, double* H, const double* M, double* A,
                       double* V, double* w, double* T, int* host_sweeps) {
    const int Rp = R + (R & 1);
    std::vector<double> hbuf(2);
    k_identity<<<256, 256, 0, st>>>(V, R);
    count_launch();
    int sweeps = 0;
    // rotation parameters (Rp doubles) followed by the two norms of the convergence test
    double* csbuf = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&csbuf, sizeof(double) * (Rp + 2), st);
    if (e != cudaSuccess) return e;
    double* d_off = csbuf + Rp;
    for (sweeps = 0; sweeps < 40 && Rp > 1; ++sweeps) {
        for (int round = 0; round < Rp - 1; ++round) {
            k_jacobi_angles<<<cdiv(Rp / 2, 128), 128, 0, st>>>(H, R, Rp, round, csbuf);
            dim3 g(cdiv(R, 128), Rp / 2);
            k_jacobi_rows<<<g, 128, 0, st>>>(H, R, Rp, round, csbuf);
            k_jacobi_cols<<<g, 128, 0, st>>>(H, V, R, Rp, round, csbuf);
            count_launch(3);
        }
        k_offnorm<<<1, 256, 0, st>>>(H, R, d_off);
        count_launch();
        e = cudaMemcpyAsync(hbuf.data(), d_off, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) break;
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) break;
        if (!(hbuf[0] > 1e-30 * hbuf[1])) {
            ++sweeps;
            break;
        }
    }
    if (host_sweeps) *host_sweeps = sweeps;
    if (e == cudaSuccess) {
        k_eig_inv<<<1, 256, 0, st>>>(H, R, w);
        dgemm(st, false, n, R, R, M, R, V, nullptr, R, T, R, nullptr, false, nullptr, 0);
        dim3 g(cdiv(R, 128), n);
        k_pinv_apply<<<g, 128, 0, st>>>(T, w, V, A, n, R);
        count_launch(2);
        e = cudaGetLastError();
    }
    cudaFreeAsync(csbuf, st);
    return e;
}

}  // namespace thc
