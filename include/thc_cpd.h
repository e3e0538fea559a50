/*
 * thc_cpd.h - C ABI of the GB300 (sm_103a) library for THC-driven matrix-free CP-ALS.
 *
 * The library fits an order-4 CP decomposition (Eq. cp4)
 *     Gt[i,a,j,b] = sum_r lam_r A1[i,r] A2[a,r] A3[j,r] A4[b,r]
 * to the (o,v,o,v) block of a THC-factorised two-electron integral tensor (Eq. THC)
 *     G[i,a,j,b]  = sum_PQ Xo[i,P] Xv[a,P] Z[P,Q] Xo[j,Q] Xv[b,Q]
 * by alternating least squares on the loss ||G - Gt||_F^2 (Eq. loss and Eq. lossF,
 * Sec. 2.1). G is never formed: every MTTKRP runs through the THC factors.
 *
 * Conventions shared by every entry point
 *   - All matrices are row-major FP64 arrays in DEVICE memory owned by the caller:
 *       Xo  o  x Rt        Xv  v x Rt        Z  Rt x Rt (need not be symmetric)
 *       A[0] = A1  o x R   A[1] = A2  v x R  A[2] = A3  o x R   A[3] = A4  v x R
 *       lam  R             M  n_mode x R
 *     A is passed as a HOST array of 4 device pointers.
 *   - Modes are numbered 0..3 for the tensor indices (i, a, j, b); n = (o, v, o, v).
 *   - loss = ||G - Gt||_F^2 (no 1/2), fit = 1 - ||G - Gt|| / ||G||.
 *   - Work is enqueued on opts->stream (NULL = legacy default stream). Scalar results
 *     (loss, fit, norms) are returned in HOST memory, so those calls synchronise the
 *     stream before returning.
 *   - Device workspace is allocated per call with the stream-ordered allocator
 *     (cudaMallocAsync) and released before return. The library never frees caller
 *     memory.
 *   - Errors: a status code is returned and thc_cpd_last_error() gives a message
 *     (per host thread). Arguments are validated before any work is enqueued; on an
 *     argument error no device memory is touched. A CUDA error leaves outputs
 *     unspecified.
 *   - Shapes: 1 <= o, v, Rt, R and (o + v) * R, Rt * R, R * R below 2^31.
 */
#ifndef THC_CPD_H
#define THC_CPD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    THC_CPD_OK = 0,
    THC_CPD_ERR_ARG = 1,        /* null pointer, bad mode, bad option */
    THC_CPD_ERR_SHAPE = 2,      /* non-positive or too large dimension */
    THC_CPD_ERR_CUDA = 3,       /* a CUDA runtime or driver call failed */
    THC_CPD_ERR_NONFINITE = 4,  /* a result came out NaN / Inf */
    THC_CPD_ERR_TIMEOUT = 5,    /* a bounded device-side wait gave up */
    THC_CPD_ERR_ALLOC = 6,      /* device workspace allocation failed */
    THC_CPD_ERR_UNSUPPORTED = 7 /* option not available on this device */
} thc_cpd_status;

typedef enum {
    THC_CPD_FP64 = 0,      /* every step in FP64 */
    THC_CPD_BF16X3 = 1,    /* MTTKRP GEMMs on tcgen05 tensor cores with each operand split
                              into two BF16 words (hi*hi + hi*lo + lo*hi), FP32
                              accumulation in TMEM; Gram, solve and loss stay FP64 */
    THC_CPD_TF32X3 = 2     /* as BF16X3 with two TF32 words per operand */
} thc_cpd_precision;

typedef struct thc_cpd_opts {
    int precision;       /* thc_cpd_precision */
    int loss_every;      /* mixed precision only: evaluate the FP64 loss every n sweeps
                            (0: every sweep when tol > 0, else only after the last) */
    void* stream;        /* cudaStream_t */
    double* history;     /* optional HOST buffer of 2*max_sweeps doubles: (loss, fit)
                            per sweep, NaN for sweeps whose loss was not evaluated */
    int flags_out;       /* out: bit 0 = pseudo-inverse fallback used at least once,
                                 bit 1 = a sweep was rolled back and replayed,
                                 bit 2 = the run switched to FP64 sweeps (polish) */
    int polish_sweeps;   /* split precision, tol <= 0 only: the last polish_sweeps of the
                            max_sweeps run in FP64. With tol > 0 the run switches to FP64
                            by itself once |fit_s - fit_{s-1}| < 10 tol and stops at tol,
                            so that it ends on a fixed point of FP64 ALS */
    int autotune;        /* split precision: nonzero times the candidate tensor-core tile
                            shapes of every GEMM shape the first time it is met (on the
                            live operands, before any graph capture) and keeps the fastest
                            for the rest of the process */
    int accepted_out;    /* out (thc_cpd_als with mlp): accepted extrapolated steps */
    const float* mlp;    /* thc_cpd_als: device parameters of the step-proposer network
                            (THC_CPD_MLP_NPARAM floats) or NULL for plain ALS; see below */
    int ldl;             /* thc_cpd_ldl: how the LDL^T of the normal equations runs.
                            AUTO (0): the dataflow kernel for a single problem with R <= 2048,
                            the blocked launches for larger R and for thc_cpd_als_batched
                            (problems side by side fill the GPU better with short launches).
                            Both give the same factorisation up to rounding order; each is
                            bit-reproducible on its own. */
    double wait_limit_s; /* limit of every device-side wait of the dataflow LDL^T and the
                            backward solve, in seconds (0: 1 s). A wait that runs out makes
                            the launch give up and the call return THC_CPD_ERR_TIMEOUT. */
    double target_fit;   /* thc_cpd_als: > 0 stops after the first evaluated sweep whose
                            FP64 fit is >= target_fit (split precision evaluates the loss
                            every loss_every sweeps, or every sweep when loss_every is 0);
                            0: off. Used to compare runs at equal fit. */
} thc_cpd_opts;

/* Values of thc_cpd_opts.ldl. */
typedef enum {
    THC_CPD_LDL_AUTO = 0,
    THC_CPD_LDL_BLOCKED = 1,   /* one launch per 32-column block step */
    THC_CPD_LDL_DATAFLOW = 2,  /* one persistent launch (R <= 2048; blocked beyond) */
    THC_CPD_LDL_EMULATED = 3   /* two-level: 256-column panels (128 below R = 1536) by the dataflow kernel, each
                                  trailing update as an FP64-accurate product on the BF16
                                  tensor cores (exact integer slices, see
                                  thc_cpd_emulated_gemm), the last few hundred columns in
                                  one dataflow launch; the factorisation stays FP64 in
                                  every value it stores (R <= 4096; dataflow otherwise) */
} thc_cpd_ldl;

/* One independent problem of a batched run (thc_cpd_als_batched). Inputs as for
 * thc_cpd_als (device pointers); sweeps_done, flags_out, loss and fit are outputs. */
typedef struct thc_cpd_problem {
    int o, v, Rt, R;
    const double* Xo;
    const double* Xv;
    const double* Z;
    double* A[4];
    double* lam;
    int sweeps_done;
    int flags_out;
    double loss;
    double fit;
} thc_cpd_problem;

/* ||G||_F^2 = sum_PQ Z[P,Q] (S Z S)[P,Q], S = (Xo^T Xo) o (Xv^T Xv): the THC norm in
 * O(Rt^3), the contraction pattern of the J term of Eq. thc_Ej. Result in *normG2_host. */
thc_cpd_status thc_cpd_thc_norm2(int o, int v, int Rt,
                                 const double* Xo, const double* Xv, const double* Z,
                                 double* normG2_host, const thc_cpd_opts* opts);

/* Matrix-free MTTKRP of mode `mode` (0..3), the gradient building block of Eq. lossF:
 *   M1 = Xo (W2 o (Z   (W3 o W4)))     M2 = Xv (W1 o (Z   (W3 o W4)))
 *   M3 = Xo (W4 o (Z^T (W1 o W2)))     M4 = Xv (W3 o (Z^T (W1 o W2)))
 * with W_k = X_k^T A_k. lam is not applied. M (device, n_mode x R) is overwritten.
 * opts->precision selects FP64 or a split tensor-core path. */
thc_cpd_status thc_cpd_mttkrp(int o, int v, int Rt, int R,
                              const double* Xo, const double* Xv, const double* Z,
                              const double* const A[4], int mode, double* M,
                              const thc_cpd_opts* opts);

/* Loss in factor form (Eq. lossF): ||G||^2 - 2 <G, Gt> + lam^T (G1 o G2 o G3 o G4) lam,
 * evaluated in FP64 for every precision. lam may be NULL (all ones). normG2 <= 0 makes
 * the call compute ||G||^2 itself. Outputs in host memory (either may be NULL). */
thc_cpd_status thc_cpd_loss(int o, int v, int Rt, int R,
                            const double* Xo, const double* Xv, const double* Z,
                            const double* const A[4], const double* lam, double normG2,
                            double* loss_host, double* fit_host, const thc_cpd_opts* opts);

/* One ALS sweep: for modes 0..3 in order, M_k by the matrix-free MTTKRP, H_k the
 * Hadamard product of the other three Gram matrices, A_k <- M_k H_k^{-1} by Cholesky
 * (pseudo-inverse from a symmetric eigendecomposition if a pivot is <= R*eps*max H_ii),
 * then lam_r = ||A_k[:,r]||, A_k[:,r] /= lam_r. A and lam (device) are updated in place;
 * the incoming lam is absorbed by the first update. Loss and fit of the result are
 * returned (FP64). normG2 <= 0 makes the call compute ||G||^2. */
thc_cpd_status thc_cpd_als_sweep(int o, int v, int Rt, int R,
                                 const double* Xo, const double* Xv, const double* Z,
                                 double* const A[4], double* lam, double normG2,
                                 double* loss_host, double* fit_host, thc_cpd_opts* opts);

/* CP-ALS: up to max_sweeps sweeps, stopping after sweep s when |fit_s - fit_{s-1}| < tol
 * (tol <= 0: run all sweeps). A holds the start point on entry and the normalised
 * factors on exit; lam receives the weights. sweeps_done, loss_host and fit_host (host,
 * may be NULL) receive the sweep count and the final FP64 loss and fit. */
thc_cpd_status thc_cpd_als(int o, int v, int Rt, int R,
                           const double* Xo, const double* Xv, const double* Z,
                           double* const A[4], double* lam, int max_sweeps, double tol,
                           int* sweeps_done, double* loss_host, double* fit_host,
                           thc_cpd_opts* opts);

/* C (M x N, FP64, row-major, device) = A (M x K) B (N x K)^T with A and B row-major FP64
 * device matrices split into two words per value (opts->precision THC_CPD_BF16X3 or
 * THC_CPD_TF32X3) and multiplied on the tcgen05 tensor cores with FP32 accumulation:
 * hi*hi + hi*lo + lo*hi. The contraction kernel of the split-precision MTTKRP
 * (Sec. 2.1 gradients of Eq. lossF), exposed for testing and reuse. Synchronises. */
thc_cpd_status thc_cpd_split_gemm(int M, int N, int K, const double* A, const double* B,
                                  double* C, const thc_cpd_opts* opts);

/* CP-ALS of many independent problems of uneven (o, v, R_thc, R_cp) at once: each problem
 * follows thc_cpd_als (same sweeps, same results bit for bit), but one sweep of every
 * still-running problem is captured into a single CUDA graph whose branches run
 * concurrently, and the graph is replayed once per sweep; problems that meet
 * |fit_s - fit_{s-1}| < tol leave the graph. opts->precision applies to all problems
 * (split precisions run without the FP64 polish phase); opts->history is not used. */
thc_cpd_status thc_cpd_als_batched(int nprob, thc_cpd_problem* probs, int max_sweeps, double tol,
                                   thc_cpd_opts* opts);

/* ---- learned extrapolation of the ALS step (the paper's ALS has no line search; this
 * is an acceleration on top of it) -------------------------------------------------------
 * A 40-64-64-1 tanh network maps the ALS history to a step factor alpha = 1 + 3 sigmoid(z)
 * in [1, 4]. Inputs, most recent sweep first, zero-padded: 8 values
 * log10(max(log L_{s-1} - log L_s, 1e-12)) / 6 of the loss decrements, then per sweep the
 * four log10(max(||B_k^s - B_k^{s-1}|| / ||B_k^s||, 1e-12)) / 6 of the lam-absorbed
 * factors (lam multiplies the last mode). With opts->mlp set, thc_cpd_als tries after each
 * sweep the point P + alpha (P_ALS - P) and keeps it only if its exact FP64 loss is below
 * the plain ALS point's, so the run is never worse than plain ALS step by step.
 * Parameters (FP32 masters; the kernels use BF16-rounded weights with FP32 accumulation):
 * W1 (64 x 40 row-major), b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3 (1). */
#define THC_CPD_MLP_NPARAM 6849

/* Glorot-uniform weights and zero biases from a counter-based generator (SplitMix64). */
thc_cpd_status thc_cpd_mlp_init(float* params, unsigned long long seed, const thc_cpd_opts* opts);
/* alpha[i] for the n feature rows X (n x 40, device). Synchronises. */
thc_cpd_status thc_cpd_mlp_forward(const float* params, const float* X, int n, float* alpha,
                                   const thc_cpd_opts* opts);
/* Gradient (device, THC_CPD_MLP_NPARAM) of the MSE (1/n) sum (alpha_i - y_i)^2 and the loss
 * (host). Synchronises. */
thc_cpd_status thc_cpd_mlp_grad(const float* params, const float* X, const float* y, int n,
                                float* grad, float* loss_host, const thc_cpd_opts* opts);
/* One Adam update (Kingma & Ba 2015, b1 = 0.9, b2 = 0.999, eps = 1e-8, bias-corrected with
 * step count t >= 1) of params with gradient grad and the moments m, v (all device, FP32,
 * THC_CPD_MLP_NPARAM each; params, m, v updated in place): the optimiser step that
 * thc_cpd_mlp_train applies after every batch. Synchronises. */
thc_cpd_status thc_cpd_mlp_adam(float* params, const float* grad, float* m, float* v, int t,
                                float lr, const thc_cpd_opts* opts);
/* Adam training (lr, batches of `batch`, reshuffled every epoch from `seed`) of the MSE on
 * (X, y); params updated in place; final loss over all rows in *final_loss_host. */
thc_cpd_status thc_cpd_mlp_train(float* params, const float* X, const float* y, int n, int epochs,
                                 int batch, float lr, unsigned long long seed,
                                 float* final_loss_host, const thc_cpd_opts* opts);
/* Training data from a plain ALS trajectory: after each of `sweeps` sweeps, the 40
 * features (feats, host, sweeps x 40) and the exact FP64 losses of the trial points for
 * each alpha in alphas (trial_losses, host, sweeps x nalpha; alpha = 1 is the ALS point).
 * The trajectory itself is plain ALS (A and lam end at its last point). */
thc_cpd_status thc_cpd_als_trajectory(int o, int v, int Rt, int R, const double* Xo,
                                      const double* Xv, const double* Z, double* const A[4],
                                      double* lam, int sweeps, const double* alphas, int nalpha,
                                      float* feats, double* trial_losses, thc_cpd_opts* opts);

/* ---- launch accounting and kernel timing (tracing support; the paper has no
 * counterpart: it reports wall-times only) ---------------------------------------- */

/* Kernels this library has launched since it was loaded (all threads). */
long thc_cpd_launch_count(void);

/* Per kernel class: summed CUDA-event time of the launch groups, their algorithmic
 * FLOPs and bytes, and the number of groups. Classes: 0 FP64 GEMM, 1 Cholesky
 * (factorisation with the fused forward solve; on the emulated path its FP64 panels),
 * 2 backward solve, 3 element-wise and reduction kernels, 4 split tensor-core GEMM
 * (projections and back-projections), 5 FP64-accurate emulated products on the tensor
 * cores (digit split and product; FLOPs counted as the FP64 work they replace), 6 the
 * split tensor-core Z contraction of the MTTKRP (Eq. THC's core). */
typedef struct thc_cpd_kstat {
    double ms;
    double flops;
    double bytes;
    long groups;
} thc_cpd_kstat;

/* enable != 0 starts recording CUDA events around every launch group (process-wide)
 * and clears earlier records; 0 stops recording. Adds host overhead: leave it off in
 * timed runs whose throughput is reported. */
void thc_cpd_profile(int enable);

/* Fills out[0..min(max_classes,7)) (waits for the recorded events); returns the count
 * filled or -1 on a CUDA error. */
int thc_cpd_profile_read(thc_cpd_kstat* out, int max_classes);

/* C (M x N) = A (M x K) B (N x K)^T to FP64 accuracy on the BF16 tensor cores (the
 * contraction behind THC_CPD_LDL_EMULATED, exposed for testing and reuse; the paper's
 * solves are FP64, Sec. 2.1 and 3). Every row of A and of B is scaled by a power of two and
 * cut into 7 signed 8-bit integer digits (an error-free splitting after Ozaki, Ogita, Oishi
 * and Rump, Numer. Algorithms 59, 2012); the digit products are exact on the tensor cores
 * (FP32 accumulation of integers below 2^24, K in chunks of 128) and are recombined exactly
 * in 64-bit integers, then rounded once to FP64. Error: about 2^-53 |C| + 2^-55 K
 * max_k |A_ik| max_k |B_jk|. Row-major FP64 device arrays (lda, ldb, ldc in elements).
 * Shapes: 1 <= M, N <= 4096, K >= 1. Synchronises. */
thc_cpd_status thc_cpd_emulated_gemm(int M, int N, int K, const double* A, int lda, const double* B,
                                     int ldb, double* C, int ldc, const thc_cpd_opts* opts);

/* The CPD+THC LT-MP2 exchange energy (Sec. 2.2), the consumer of the CP factors: with
 * the Laplace quadrature factors Lam (nalpha x o, occupied) and Gam (nalpha x v, virtual)
 * of Eq. mp1_t, amplitudes t[i,a,j,b] = Lam_i Gam_a Lam_j Gam_b X[i,a,j,b] and the
 * exchange pairing K(T, Y) = -sum_alpha sum_iajb t(T)[i,a,j,b] Y[i,b,j,a]:
 *   e_single = K(G, Gt)  (Eq. cpd_single_k, factor form O(R_thc^2 R) per point),
 *   e_double = K(Gt, Gt) (the double-CPD term, O((o + v) R^2) per point),
 *   e_robust = 2 e_single - e_double (Eq. rob_K; no error of first order in G - Gt),
 * G the THC block (Eq. THC) and Gt = sum_r lam_r A1 A2 A3 A4 (Eq. cp4). Device inputs as for
 * thc_cpd_loss (lam may not be NULL); the three energies are returned in host memory (each
 * pointer may be NULL). The contractions are FP64 GEMMs on the FP64 pipes, or with
 * opts->ldl = THC_CPD_LDL_EMULATED the FP64-accurate emulated products of the tensor cores;
 * the reductions run in a fixed order. 1 <= nalpha <= 1024. Synchronises. */
thc_cpd_status thc_cpd_exchange(int o, int v, int Rt, int R, int nalpha, const double* Xo,
                                const double* Xv, const double* Z, const double* const A[4],
                                const double* lam, const double* Lam, const double* Gam,
                                double* e_single, double* e_double, double* e_robust,
                                const thc_cpd_opts* opts);

/* THC core least-squares fit (Sec. 3, Computational Details): the core Z (R_thc x R_thc)
 * minimising f(Z) = 1/2 || G_DF - G_THC(Z) ||^2, where G_DF[i,a,j,b] = sum_X B[X,i,a] B[X,j,b]
 * is the (o,v,o,v) block of density-fitted integrals and G_THC(Z) the THC block of Eq. THC
 * on the given grid factors. Solves the normal equations S Z S = E^T E, S = (Xo^T Xo) o
 * (Xv^T Xv), E[X,P] = sum_ia B[X,i,a] Xo[i,P] Xv[a,P], as Z = F^T F with F = E S^-1 (LDL^T of
 * S, pseudo-inverse of S when a pivot fails: *used_pinv = 1). The result is symmetric.
 * Xo (o x Rt), Xv (v x Rt), B (naux x o x v, row-major), Z (Rt x Rt, written): device FP64.
 * loss: NULL, or host double receiving ||G_DF - G_THC(Z)||^2 (no 1/2) in factor form.
 * 1 <= R_thc <= 2048; o * v, naux * o, naux * R_thc and naux^2 below 2^31. The GEMMs run on the
 * FP64 pipes, or with opts->ldl = THC_CPD_LDL_EMULATED as the FP64-accurate emulated products
 * of the tensor cores (the solve then uses the emulated two-level LDL^T as well).
 * Allocates its workspace (about 256 MiB plus 2 naux R_thc doubles, plus naux o v and naux^2
 * doubles with loss) with cudaMallocAsync on opts->stream. Synchronises. */
thc_cpd_status thc_cpd_core_fit(int o, int v, int Rt, int naux, const double* Xo, const double* Xv,
                                const double* B, double* Z, double* loss, int* used_pinv,
                                const thc_cpd_opts* opts);

/* DF-driven CP-ALS (Sec. 2.1, Eq. df_loss), the prior-work variant the THC-driven method
 * replaces: CP-ALS of G_DF[i,a,j,b] = sum_X B[X,i,a] B[X,j,b] with every MTTKRP formed from
 * the order-3 DF tensor B (naux x o x v, device, row-major) at O(naux o v R) per mode (four
 * GEMMs of 2 naux o v R flop per sweep), the same normal-equation solve, normalisation, loss
 * and stopping rule as thc_cpd_als: A[4] (o x R, v x R, o x R, v x R) start factors in, final
 * unit-column factors out; lam (R) out; sweeps_done and fit_host (host) out, each may be NULL.
 * opts->precision must be THC_CPD_FP64; opts->ldl = THC_CPD_LDL_EMULATED runs the GEMMs and the
 * solve on the emulated FP64 tensor-core path. opts->history: NULL or 2 * max_sweeps host
 * doubles (loss, fit per sweep). opts->flags_out bit 0: a pseudo-inverse solve was used.
 * Workspace: about (2 o v + max(o, v) R + 3 R) naux + naux^2 + 5 R^2 doubles (cudaMallocAsync).
 * 1 <= R <= 2048, 1 <= o, v <= 4096. Synchronises once per sweep. */
thc_cpd_status thc_cpd_df_als(int o, int v, int naux, int R, const double* B, double* const A[4],
                              double* lam, int max_sweeps, double tol, int* sweeps_done,
                              double* fit_host, thc_cpd_opts* opts);

/* THC-driven CP-ALS of an order-d THC-like tensor (Conclusions; the order-4 block of Eq. THC
 * is the case d = 4, dL = 2, X = (Xo, Xv, Xo, Xv)):
 *   G[i_0..i_{d-1}] = sum_{P,Q} prod_{k < dL} X_k[i_k,P] Z[P,Q] prod_{k >= dL} X_k[i_k,Q],
 * CPD Gt = sum_r lam_r prod_k A_k[i_k,r]. dims: host array of the d mode sizes; X, A: host
 * arrays of d device pointers (X_k dims[k] x Rt, A_k dims[k] x R, row-major FP64); Z: device
 * Rt x Rt (need not be symmetric). 2 <= d <= 8, 1 <= dL <= d - 1, 1 <= dims[k] <= 4096,
 * 1 <= R <= 2048. Precision FP64 only; opts->ldl = THC_CPD_LDL_EMULATED runs the GEMMs and the
 * solve on the emulated FP64 tensor-core path.
 * thc_cpd_nd_mttkrp: M (dims[mode] x R, device) = the mode-`mode` MTTKRP (lam not applied).
 * thc_cpd_nd_als: A in/out (unit columns out), lam out, sweeps_done / fit_host host (may be
 * NULL); solve, normalisation, loss, stopping rule, history and flags_out as thc_cpd_df_als.
 * Allocate their workspace with cudaMallocAsync; synchronise (the ALS once per sweep). */
thc_cpd_status thc_cpd_nd_mttkrp(int d, int dL, const int* dims, int Rt, int R, const double* const* X,
                                 const double* Z, const double* const* A, int mode, double* M,
                                 const thc_cpd_opts* opts);
thc_cpd_status thc_cpd_nd_als(int d, int dL, const int* dims, int Rt, int R, const double* const* X,
                              const double* Z, double* const* A, double* lam, int max_sweeps, double tol,
                              int* sweeps_done, double* fit_host, thc_cpd_opts* opts);

/* Measured FP64 FMA throughput of the device (TFLOP/s, 2 flop per FMA) from a probe kernel
 * of independent FMA chains on every SM (64 warps per SM, best of three timed launches):
 * the roofline denominator of the FP64 kernels (Gram, solve, loss). Synchronises. */
thc_cpd_status thc_cpd_fp64_fma_rate(double* tflops_host, const thc_cpd_opts* opts);

/* thc_cpd_mttkrp without any device allocation (the paper has no counterpart: this is
 * a service for callers that may not allocate device memory while they run, such as a
 * host whose own pool allocator owns all device memory, or code that must not call
 * cudaMalloc because it can synchronise the device).
 * Same arguments and result as thc_cpd_mttkrp, FP64 only (opts->precision must be
 * THC_CPD_FP64 or opts NULL). The caller still provides Xo, Xv, Z, A and M; all scratch
 * comes from one 32 MiB array in the library's device memory, which every GPU that loads
 * the library keeps until the process exits. Problems whose 4 * R_thc * R_cp doubles do
 * not fit in it are rejected with THC_CPD_ERR_SHAPE (message in thc_cpd_last_error()).
 * Arguments are checked exactly as thc_cpd_mttkrp checks them (same statuses and messages).
 * The first call on a device, with that device current, looks up the array's device
 * address (cudaGetSymbolAddress); make it before any stream capture. Under CUDA's default
 * lazy module loading that first call is also what creates the 32 MiB array on the device
 * (with CUDA_MODULE_LOADING=EAGER, process start does): make it before another pool
 * allocator claims the device's memory; if no memory is left then, it returns
 * THC_CPD_ERR_CUDA with that explanation. The address is cached per device ordinal and
 * belongs to the device's primary context: it stays valid for the process's lifetime, not
 * across a cudaDeviceReset or in another context. Calls only enqueue
 * work on opts->stream (no synchronisation); M is ready when the stream reaches that
 * point. All calls on a device share the array, which keeps the last call's contents:
 * calls whose GPU work overlaps race on it and must be serialised by the caller. */
thc_cpd_status thc_cpd_mttkrp_noalloc(int o, int v, int Rt, int R,
                                      const double* Xo, const double* Xv, const double* Z,
                                      const double* const A[4], int mode, double* M,
                                      const thc_cpd_opts* opts);

/* Normal-equation solve of one ALS mode update (Sec. 2.1, the textbook CP-ALS update the
 * paper's ALS follows): A (n x R) with A H = M for the symmetric positive (semi)definite
 * H (R x R, full matrix, lower triangle read) and M (n x R), by the dataflow LDL^T with the
 * M rows carried along and the backward solve, exactly as inside thc_cpd_als. A pivot
 * <= R * eps * max_i H_ii switches to the pseudo-inverse (symmetric eigendecomposition,
 * eigenvalues <= R * eps * max |w| dropped); *used_pinv (host, may be NULL) says so.
 * H, M and A are device arrays owned by the caller; H and M are not modified.
 * tasks: NULL for the library's own schedule, or a caller-built off-path task list in the
 * format of thc_cpd_ldl_schedule (host, 4 shorts per task, ntasks tasks). A caller list is
 * checked for index ranges only (THC_CPD_ERR_ARG otherwise) and used as given: a list that
 * lacks a task some other task or the pivot chain waits for makes those waits run out
 * after opts->wait_limit_s and the call return THC_CPD_ERR_TIMEOUT; the device stays usable.
 * Shapes: 1 <= R <= 2048, 1 <= n <= 4096. Synchronises the stream. */
thc_cpd_status thc_cpd_ldl_solve(int R, int n, const double* H, const double* M, double* A,
                                 const short* tasks, int ntasks, int* used_pinv,
                                 const thc_cpd_opts* opts);

/* Task list of the dataflow LDL^T of the normal-equation solve (host only, no device
 * work; Sec. 2.1's normal equations, solved by LDL^T with the M rows carried along).
 * For an R x R matrix with n appended rows and 16 x 16 tiles, writes the off-path tasks in
 * the order worker groups claim them, 4 shorts per task: type (0 = substitution S(t, k) of
 * row tile t with diagonal tile k, 1 = trailing update U(t, j, k) of tile (t, j) with panel
 * k), then t, j, k. Row tiles 0..ceil(R/16)-1 are rows of H, the next ones rows of M. The
 * diagonal chain (S(s, s-1), U(s, s, s-1) and the factorisation of tile (s, s)) is not in
 * the list. out: caller-owned host array of cap tasks (4 * cap shorts), or NULL to query
 * the count; at most cap tasks are written. Returns the number of tasks, or -1 when R < 1,
 * n < 0, the shape is beyond the dataflow path (more than 256 tiles a side: the blocked
 * factorisation runs instead) or the order fails its check that every task comes after
 * all tasks it waits for. No counterpart in the paper: it exposes the schedule to tests. */
int thc_cpd_ldl_schedule(int R, int n, short* out, int cap);

/* Message for the last non-OK status returned on this host thread. */
const char* thc_cpd_last_error(void);

/* Library version string. */
const char* thc_cpd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* THC_CPD_H */
