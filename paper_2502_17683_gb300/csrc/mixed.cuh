// Split-precision (BF16x3 / TF32x3) MTTKRP on tcgen05 tensor cores.
//
// Dataflow of one sweep (all intermediates stored r-major, i.e. transposed, so that
// every GEMM operand is K-major):
//   Z-GEMM half 0: Y12 = Z (W3 o W4)   -> Y (FP32) and E = split(W2 o Y12)
//   mode 0: M1 = Xo E (FP64 out) ... solve ... projection W1 -> Wt[0] and E = split(W1 o Y12)
//   mode 1: M2 = Xv E ... projection W2 -> Wt[1] and P = split(W1 o W2)
//   Z-GEMM half 1: Y34 = Z^T (W1 o W2) -> Y and E = split(W4 o Y34)
//   mode 2: M3 = Xo E ... projection W3 -> Wt[2] and E = split(W3 o Y34)
//   mode 3: M4 = Xv E ... projection W4 -> Wt[3] and P = split(W3 o W4)
// so each Hadamard product of the method is fused into the epilogue of the GEMM that
// produces its last factor.
#pragma once
#include "common.cuh"
#include "tc_gemm.cuh"

namespace thc {

struct MixedWs {
    bool tf32 = false;
    int o = 0, v = 0, Rt = 0, R = 0;
    SplitMat Zs, ZTs;    // Z (P x Q) and Z^T, B operands of the Z-GEMMs
    SplitMat XT[2];      // Xo^T, Xv^T (Rt x n): B operands of the projections
    SplitMat Xs[2];      // Xo, Xv (n x Rt): B operands of the back-projections
    SplitMat At[4];      // A_k^T (R x n_k): A operands of the projections
    SplitMat Pt, Et;     // Hadamard operands (R x Rt): A of Z-GEMM / back-projection
    float* Wt[4] = {};   // W_k^T (R x Rt, FP32)
    float* Yf = nullptr; // Y12 or Y34 (R x Rt, FP32)
    double* part = nullptr;  // split-K partials of the back-projection
    size_t part_cap = 0;
};

bool mixed_supported();
size_t mixed_ws_bytes(bool tf32, int o, int v, int Rt, int R);
void mixed_ws_carve(MixedWs& mx, Arena& ar, bool tf32, int o, int v, int Rt, int R);
// split Z, Z^T, Xo, Xv, Xo^T, Xv^T once per call
cudaError_t mixed_setup(MixedWs& mx, cudaStream_t st, const double* Xo, const double* Xv,
                        const double* Z);
// W_k = X_k^T A_k on tensor cores with the fused Hadamard epilogue; `in_sweep` enables
// the E products that need the current Y.
cudaError_t mixed_project(MixedWs& mx, cudaStream_t st, int k, const double* Ak, bool in_sweep);
cudaError_t mixed_zgemm(MixedWs& mx, cudaStream_t st, int half);
// E = split(W_partner o Y) for modes 1 and 3 outside a sweep
cudaError_t mixed_partner(MixedWs& mx, cudaStream_t st, int mode);
// M_k = X_k E (n_k x R, FP64)
cudaError_t mixed_backproject(MixedWs& mx, cudaStream_t st, int k, double* M);
int mixed_take_error();

}  // namespace thc
