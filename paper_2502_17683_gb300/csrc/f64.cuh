// FP64 kernels of the THC-CPD path: launchers (definitions in f64_kernels.cu).
#pragma once
#include "common.cuh"

namespace thc {

// C[M x N] = op(A)[M x K] * (B o B2)[K x N], optionally C = E o (that product).
//   op(A)[m,k] = trans_a ? A[k*lda + m] : A[m*lda + k];  B, B2 row-major with ldb.
//   symm: C is symmetric (A^T A-like); only lower tiles are computed and mirrored.
// Split-K partials go to `part` (capacity part_cap doubles); deterministic reduction.
void dgemm(cudaStream_t st, bool trans_a, int M, int N, int K, const double* A, int lda,
           const double* B, const double* B2, int ldb, double* C, int ldc,
           const double* E, bool symm, double* part, size_t part_cap);

// Split-K partial capacity (doubles) that dgemm may use for an M x N output.
size_t dgemm_part_need(int M, int N, int K);

// H = Ga o Gb o Gc (R x R) written to H (ld R); sc->maxdiag = max_i H_ii.
void hadamard3(cudaStream_t st, int R, const double* Ga, const double* Gb, const double* Gc,
               double* H, DevScalars* sc);

// In-place solve of A H = M for A (n x R), H SPD (R x R), by LDL^T with the M rows
// carried along (fused forward solve) and a unit backward solve.
//   Haug: (R + n) x R, rows 0..R-1 hold H (lower triangle read), rows R.. hold M.
//   P: R x 32 panel workspace (R x R for the dataflow path), dinv: R doubles.
//   A pivot <= R * eps * sc->maxdiag sets bit `mode` of sc->fail_mask (the result is then
//   garbage and the caller replays the mode with the pseudo-inverse).
//   counters: cdiv(R, 32) ints (arrival counters of the update kernels, cleared inside).
//   flow_sync: flow_sync_ints(R, n) ints, zero before the first use (each launch leaves
//   them zero), or null: with it (and a plan for (R, n)) the factorisation runs as one
//   persistent dataflow launch (P is then R x R), else as one launch per block step.
//   flow_ctas: 0 = the dataflow kernel takes one CTA per SM; > 0 = at most that many CTAs
//   with only the shared memory they use (problems running side by side).
//   bs_sync: bsolve_sync_ints(n) ints, the progress counters of the backward solve (by
//   column slices, ldl_flow.cu); zero before the first use, left zero by each launch.
//   oz: with it (and flow_sync) the factorisation runs in 256- (below R = 1536: 128-) column panels with emulated
//   FP64 tensor-core trailing updates (ldl_oz, oz.cuh).
struct OzWs;
void chol_solve(cudaStream_t st, int R, int n, double* Haug, double* A, double* P, double* dinv,
                DevScalars* sc, int mode, int* counters, int* flow_sync, int flow_ctas,
                int* bs_sync, const OzWs* oz = nullptr);
// The backward solve A L = Y of a factorised Haug (Y in its rows R..R+n): with an emulated
// factorisation's workspace (oz) and n >= 128, a block of >= 768 columns is split at a
// column h0: the trailing block first, the coupling Y1 -= A2 L21 as an emulated product,
// then the leading block, each of them split again by the same rule.
void backward_solve(cudaStream_t st, int R, int n, double* Haug, double* A, int* bs_sync,
                    const OzWs* oz = nullptr);
// Raises *rowsA / *rowsB (emulated-product workspace rows, oz_ws_carve) to what the split
// backward solve of an R x R factor with up to nmax right-hand sides needs to form each
// coupling product in one launch (all its K chunks' digits at once), and *part_doubles to
// its split-K partial sums; with less the products run chunk by chunk / unsplit.
void bsolve_ws_rows(int R, int nmax, int* rowsA, int* rowsB, size_t* part_doubles);

// A = M H^-1 for H symmetric positive definite (R x R, lower triangle read) and M (n x R),
// all device pointers, 1 <= R <= 2048, 1 <= n <= 4096: the solve of thc_cpd_ldl_solve (LDL^T
// with the forward solve fused, dataflow or emulated two-level by `ldl` (thc_cpd_ldl values),
// backward solve, pseudo-inverse when a pivot fails: *used_pinv = 1). tasks: null or a
// caller-built dataflow task list (ntasks entries). Allocates its workspace on st and
// synchronises st. Returns a thc_cpd_status; the message is set on failure.
int spd_solve(cudaStream_t st, int R, int n, const double* H, const double* M, double* A,
              const short* tasks, int ntasks, int* used_pinv, int ldl);

// Dataflow LDL^T (ldl_flow.cu): ints of progress state for R and n <= nmax; plan set-up
// for (R, n) (false: too large or the task order failed its check; use the blocked path);
// the launch; the error flag of bounded waits that gave up (read and cleared).
size_t flow_sync_ints(int R, int nmax);
bool flow_prepare(int R, int n);
cudaError_t ldl_flow(cudaStream_t st, int R, int n, double* Haug, double* P, double* dinv,
                     DevScalars* sc, int mode, int* sync, int max_ctas = 0);
int flow_take_error();
// The same launch with a caller-provided task list (host, 4 shorts per task as
// thc_cpd_ldl_schedule writes them; dev_tasks: 8 * ntasks bytes of device memory). The list
// is used as given: an incomplete or misordered one ends in bounded waits that give up.
cudaError_t ldl_flow_tasks(cudaStream_t st, int R, int n, double* Haug, double* P, double* dinv,
                           DevScalars* sc, int mode, int* sync, const short* host_tasks,
                           int ntasks, void* dev_tasks);
// One panel of the two-level factorisation: columns [j0, j0 + bw) of the (R + n) x R matrix
// Haug (ld R), all rows from j0 down, as one dataflow launch whose "appended rows" are every
// row below the panel's diagonal block (their L, or Y for the M rows, in the panel columns).
// The trailing update is the caller's. A plan for (bw, R + n - j0 - bw) must exist
// (flow_prepare); the pivot threshold uses the whole order R.
cudaError_t ldl_flow_panel(cudaStream_t st, int R, int n, int j0, int bw, double* Haug, double* P,
                           double* dinv, DevScalars* sc, int mode, int* sync, int max_ctas = 0);
// Index of the first task whose type or tile indices are out of range, or -1.
int flow_task_check(int R, int n, const short* tasks, int ntasks);
// Limit of every wait of the dataflow LDL^T and the backward solve launched afterwards from
// this host thread (0: the default, 1 s).
void flow_set_wait_ns(unsigned long long ns);

// H_out = H (R x R) and sc->maxdiag = max_i H_ii.
void copy_with_maxdiag(cudaStream_t st, int R, const double* H, double* H_out, DevScalars* sc);

// Backward solve A L = Y (unit lower L in the strictly-lower part of H, R x R; Y and A n x R)
// by column slices claimed from a ticket (ldl_flow.cu); sync: bsolve_sync_ints(n) ints.
// ld: row pitch of Y, A and H (0: R), so that a diagonal block of a larger factor can be
// solved on its own.
size_t bsolve_sync_ints(int nmax);
cudaError_t bsolve_slices(cudaStream_t st, int R, int n, const double* Yf, double* A,
                          const double* H, int* sync, int ld = 0);

// lam_r = ||A[:,r]||_2; A[:,r] /= lam_r (lam_r = 0 leaves the column); scratch >= R doubles.
void normalise_columns(cudaStream_t st, int n, int R, double* A, double* lam, double* scratch);

// dst[p][0 .. len[p]) = src[p][...] for p < np (np <= 8) in one launch (the state snapshot
// taken before every sweep for a rollback).
cudaError_t copy_many(cudaStream_t st, int np, const double* const* src, double* const* dst,
                      const long* len);

// Loss in factor form after a sweep: inner = sum lam_r Y[Q,r] W3[Q,r] W4[Q,r],
// cpdn2 = lam^T (G1 o G2 o G3 o G4) lam; loss, fit, convergence into sc.
void loss_eval(cudaStream_t st, int Rt, int R, const double* Y, const double* W3,
               const double* W4, const double* lam, const double* const G[4],
               double* red, DevScalars* sc, double tol);
size_t loss_red_need();

// sc->normG2 = sum Z o U (U = S Z S computed by the caller).
void sum_hadamard_normG2(cudaStream_t st, long n, const double* Z, const double* U,
                         double* red, DevScalars* sc);

// Initialise the scalars struct (normG2 kept if keep_norm).
void scalars_init(cudaStream_t st, DevScalars* sc, double normG2);

// Jacobi eigen-decomposition based pseudo-inverse solve: A = M pinv(H).
//   H (R x R, full symmetric, destroyed), M (n x R), V workspace R x R, w R,
//   T workspace n x R. Returns cudaError of the last launch.
cudaError_t pinv_solve(cudaStream_t st, int R, int n, double* H, const double* M,
                       double* A, double* V, double* w, double* T, int* host_sweeps);

// Learned extrapolation helpers on lam-absorbed factors (lam multiplies the last mode):
// out2 = (||N - P||_F^2, ||N||_F^2); T = P + alpha (N - P); out = a o b o c o d.
void change_norm(cudaStream_t st, int n, int R, const double* An, const double* Ao,
                 const double* ln, const double* lo, bool absorb, double* red, double* out2);
void trial_point(cudaStream_t st, int n, int R, const double* An, const double* Ao,
                 const double* ln, const double* lo, bool absorb, double alpha, double* T);
void lam_product(cudaStream_t st, int R, const double* const l[4], double* out);
// the network's alpha for one 40-feature vector (device pointers)
void mlp_forward1(cudaStream_t st, const float* P, const float* x, float* alpha);

// out (cols x rows) = in (rows x cols)^T (32 x 32 tiles through shared memory)
void transpose64(cudaStream_t st, int rows, int cols, const double* in, double* out);

// fill lam with ones
void fill(cudaStream_t st, double* p, long n, double v);

}  // namespace thc
