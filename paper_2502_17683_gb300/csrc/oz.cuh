// FP64-accurate products on the BF16 tensor cores (tcgen05) by exact integer slicing, and
// the two-level LDL^T of the normal equations built on them (oz_gemm.cu).
//
// Slicing (the error-free splitting of Ozaki, Ogita, Oishi & Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012): every row of an FP64
// operand is scaled by a power of two 2^e (|x| < 2^e over the row) and written as
//     x = 2^e sum_{a=0}^{S-1} d_a 2^{-7-8a},  d_a integers with |d_a| <= 128,
// dropping what lies below 2^{e-55} (the row maximum's 55th bit). Each d_a is exact in
// BF16, each product d_a d'_b is exact in FP32, and a K-sum of at most 128 of them
// (<= 2^21) stays an exact FP32 integer, so the tensor cores return every slice product
// exactly. Products whose slice indices satisfy a + b = g share the scale 2^{-14-8g} and
// are accumulated in one TMEM accumulator (at most 7 * 2^21 < 2^24: still exact); the
// diagonals g = 0..S-1 are kept (the dropped ones lie below 2^-56 of the row maxima). The
// epilogue recombines the integer accumulators exactly in 64-bit integers, rounds once to
// FP64 and applies the result to the FP64 output with one fused multiply-add. The error is
// thus about 2^-53 of |result| plus 2^-55 of (row max)(column max) K: that of an FP64
// GEMM, with 28 BF16 MMAs per 16 of K instead of FP64 FMAs (GB300: 2 FP64 FMA per clock
// per SM against ~3500 BF16 MAC).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace thc {

constexpr int kOzSlices = 7;    // S: integer digits per value
constexpr int kOzPanel = 128;   // K of one emulated product (panel width of the LDL^T)

// Device workspace of the two-level LDL^T (slices of the two operands of one trailing
// update and their row exponents).
struct OzWs {
    uint16_t* sA = nullptr;  // [S][rowsA][kOzPanel] BF16 digits of the left operand
    uint16_t* sB = nullptr;  // [S][rowsB][kOzPanel] right operand
    int* eA = nullptr;
    int* eB = nullptr;
    int rowsA = 0, rowsB = 0;
    double* part = nullptr;  // split-K partial sums of a product (optional)
    size_t part_cap = 0;     // doubles at part
};

// Workspace for left operands of up to rowsA rows and right operands of up to rowsB rows
// (the LDL^T of an R x R matrix with n appended rows: rowsA = R + n, rowsB = R; a product
// of several K chunks in one launch takes chunks x rows), and part_doubles doubles of
// split-K partial sums.
size_t oz_ws_bytes(int rowsA, int rowsB, size_t part_doubles = 0);
void oz_ws_carve(OzWs& w, Arena& ar, int rowsA, int rowsB, size_t part_doubles = 0);

// Raises *rowsA / *rowsB to the rows the two-level LDL^T of an R x R matrix with up to
// nmax appended rows needs for its trailing updates when its panels are wider than
// kOzPanel (all of a panel's chunks split at once).
void oz_ldl_ws_rows(int R, int nmax, int* rowsA, int* rowsB);

// The tensor-core kernels can run on the current device (sm_103, enough shared memory).
bool oz_available();

// True when the two-level factorisation is available for (R, n) on the current device
// (tensor cores, plans of every panel); prepares those plans (call outside capture).
bool oz_prepare(int R, int n);

// Two-level LDL^T of Haug ((R + n) x R, ld R; H in the first R rows, lower triangle read,
// M in the rest), same result layout as ldl_flow: panels of 2 kOzPanel columns (kOzPanel below R = 1536) factorised by
// the dataflow kernel (ldl_flow_panel), each followed by the emulated FP64 trailing update
//   Haug[i][j] -= sum_{k in panel} L[i][k] D[k] L[j][k]   (j <= i for H rows; all j < R for M rows)
// of the rows and columns after the panel; the last few hundred columns (oz_gemm.cu,
// kTailCols) as one dataflow factorisation of the trailing block. P: R x R (X = L D of the diagonal blocks), dinv:
// R, sync: flow_sync_ints(R, n) ints (zero; left zero).
// max_ctas > 0: the panels run on at most that many CTAs (problems side by side).
cudaError_t ldl_oz(cudaStream_t st, int R, int n, double* Haug, double* P, double* dinv,
                   DevScalars* sc, int mode, int* sync, const OzWs& ws, int max_ctas = 0);

// C (M x N, ldc) += sign * A B^T for FP64 row-major A (M x K, lda) and B (N x K, ldb),
// emulated in K chunks of kOzPanel through the split and tensor-core kernels; lower: rows
// i < N are updated only for j <= i. ws must hold M (rowsA) and N (rowsB) rows.
cudaError_t oz_gemm(cudaStream_t st, int M, int N, int K, const double* A, int lda, const double* B,
                    int ldb, double* C, int ldc, double sign, bool lower, const OzWs& ws);

// The FP64 GEMM of f64.cuh (dgemm) emulated on the tensor cores, same semantics:
//   C[M x N] = op(A)[M x K] (B o B2)[K x N], or E o that product when E is given;
//   op(A)[m][k] = trans_a ? A[k * lda + m] : A[m * lda + k]; B, B2 row-major (ldb);
//   symm: C symmetric (M == N); the lower triangle is computed and mirrored.
// ws must hold M (rowsA) and N (rowsB) rows.
cudaError_t oz_dgemm(cudaStream_t st, bool trans_a, int M, int N, int K, const double* A, int lda,
                     const double* B, const double* B2, int ldb, double* C, int ldc, const double* E,
                     bool symm, const OzWs& ws);

// C (M x N, ldc) -= A B for row-major FP64 A (M x K, lda) and B (K x N, ldb), emulated in K
// chunks of kOzPanel (the coupling term of a split backward solve). ws must hold M (rowsA)
// and N (rowsB) rows.
cudaError_t oz_gemm_sub(cudaStream_t st, int M, int N, int K, const double* A, int lda, const double* B,
                        int ldb, double* C, int ldc, const OzWs& ws);

// Device error word of the emulated-product kernel (bounded waits that gave up); read and
// clear.
int oz_take_error();

}  // namespace thc
