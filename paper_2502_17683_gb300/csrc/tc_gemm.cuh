// Split-operand GEMM on the 5th-generation tensor cores (tcgen05) of sm_103a.
//
// D[m][n] = sum_k A[m][k] B[n][k], A and B K-major, each held as two words per value
// (hi + lo) so that D = Ah Bh + Ah Bl + Al Bh recovers about 16 (BF16x3) or 22 (TF32x3)
// significant bits per product; accumulation in FP32 in tensor memory (TMEM).
// Operands arrive through TMA (128-byte swizzle) into a multi-stage shared-memory ring;
// one thread issues the MMAs; four warps drain TMEM and run a fused epilogue.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace thc {

// Split operand matrix: rows x cols (K-major), row pitch `pitch` elements (multiple of
// the 128-byte K block), element 2 bytes (BF16) or 4 bytes (TF32 in FP32 words).
struct SplitMat {
    void* hi = nullptr;
    void* lo = nullptr;
    int rows = 0, cols = 0, pitch = 0;
};

// Epilogue of one GEMM; all outputs indexed [m][n] unless stated.
struct TcEpilogue {
    float* out_f32 = nullptr;  // D (ld_f32)
    int ld_f32 = 0;
    const float* mul = nullptr;  // if set: split(D o mul) -> out_split (same layout)
    int ld_mul = 0;
    SplitMat* out_split = nullptr;
    double* out_f64t = nullptr;  // D^T as FP64: out_f64t[n * ld_f64t + m]
    int ld_f64t = 0;
    int prof_class = 4;          // kernel class of the launch in the profile (KC_TC)
};

bool tc_available();
// D = A B^T for A (M x K) and B (N x K) split operands; tf32 selects the TF32x3 kind.
// With only the transposed FP64 output requested, K may be split over CTAs: the partial
// sums go to `part` (capacity part_cap doubles) and are reduced in a fixed order.
cudaError_t tc_gemm(cudaStream_t st, bool tf32, const SplitMat& A, const SplitMat& B, int M,
                    int N, int K, const TcEpilogue& ep, double* part = nullptr,
                    size_t part_cap = 0);
// Autotuning of the tile N: while on, the first call of every (M, N, K, precision,
// epilogue) outside stream capture times the candidates and caches the fastest.
void tc_set_tuning(bool on);
int tc_tuned_entries();
// Device error word of the tensor-core kernels (bounded waits that gave up); read and
// clear.
int tc_take_error();

// Conversions into split operands (elements per 128-byte K block: 64 BF16 or 32 TF32).
int split_kblock(bool tf32);
int split_pitch(bool tf32, int cols);
// dst[r][c] = split(src[r * ld + c]) for r < rows, c < cols
void split_rows(cudaStream_t st, bool tf32, const double* src, int ld, int rows, int cols,
                SplitMat& dst);
// dst[c][r] = split(src[r * ld + c]) (transposed)
void split_transpose(cudaStream_t st, bool tf32, const double* src, int ld, int rows, int cols,
                     SplitMat& dst);
// dst[r][c] = split(a[r][c] * b[r][c]) for FP32 operands with leading dimension ld
void split_hadamard(cudaStream_t st, bool tf32, const float* a, const float* b, int ld, int rows,
                    int cols, SplitMat& dst);

}  // namespace thc
