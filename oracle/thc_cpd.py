"""FP64 oracle for the order-4 CPD of a THC-factorised integral block (CPU, numpy).

TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and bench.py's CPU
baseline; the library never imports it.

Objects (paper notation -> names here):
  THC block   G_iajb = sum_PQ Xo_iP Xv_aP Z_PQ Xo_jQ Xv_bQ
              (Eq. THC with U split into occupied / virtual blocks, Sec. 2.1, and the
              THC target of Eq. lossF restricted to the (o,v,o,v) block).
  CPD         Gt_iajb = sum_r lam_r A1_ir A2_ar A3_jr A4_br   (Eq. cp4; the two
              particle factors A, B of Eq. cp4 split into occupied/virtual parts
              give four independent factors, one per mode i, a, j, b).
  loss        ||G - Gt||_F^2   (Eq. loss / Eq. lossF without the 1/2 factor).
  fit         1 - ||G - Gt|| / ||G||, relerr = ||G - Gt|| / ||G|| (Sec. 3 defines
              the ratio ||T - Tt|| / ||T|| and stops on its change).

Everything is FP64. Library primitives used as steps: numpy matmul / einsum,
numpy.linalg.cholesky, scipy.linalg.solve_triangular, numpy.linalg.eigh.

Readings where the paper is silent (the ALS cost breakdown sits in the missing
supplement) follow textbook CP-ALS (Kolda & Bader 2009, cited in Sec. 2.1):
  * sweep order i, a, j, b (modes 0..3), Gauss-Seidel;
  * the mode-k update solves A_k H_k = M_k with H_k the Hadamard product of the other
    three Gram matrices and M_k the MTTKRP of the other (unscaled) factors, which
    absorbs lam; then lam_r = ||A_k[:, r]||_2 and the columns are normalised
    (a zero column keeps lam_r = 0 and is left as is);
  * Cholesky of H_k; if a pivot d_j <= R * eps * max_i H_ii (or is not finite),
    the pseudo-inverse from the symmetric eigendecomposition is used instead, with
    eigenvalues <= R * eps * max|w| dropped;
  * after each sweep loss and fit are evaluated in factor form; convergence when
    |fit_s - fit_{s-1}| < tol.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

EPS = np.finfo(np.float64).eps


# --------------------------------------------------------------------------------------
# explicit tensors (tiny sizes only)
# --------------------------------------------------------------------------------------
def thc_tensor(Xo, Xv, Z):
    """G[i,a,j,b] = sum_PQ Xo[i,P] Xv[a,P] Z[P,Q] Xo[j,Q] Xv[b,Q]   (Eq. THC, Eq. lossF).

    Written as T Z T^T with the particle-pair matrix T[(i,a), P] = Xo[i,P] Xv[a,P].
    """
    o, Rt = Xo.shape
    v = Xv.shape[0]
    T = (Xo[:, None, :] * Xv[None, :, :]).reshape(o * v, Rt)
    return (T @ Z @ T.T).reshape(o, v, o, v)


def thc_tensor_full(U, Z):
    """Full-orbital THC g_pqrs = sum_PQ U_pP U_qP Z_PQ U_rQ U_sQ (Eq. THC with U = [Uo; Uv]).

    Index order follows G: (p, q) belong to particle 1 (grid index P), (r, s) to particle 2.
    """
    n, Rt = U.shape
    T = (U[:, None, :] * U[None, :, :]).reshape(n * n, Rt)
    return (T @ Z @ T.T).reshape(n, n, n, n)


def cpd_tensor(A, lam=None):
    """Gt[i,a,j,b] = sum_r lam_r A1[i,r] A2[a,r] A3[j,r] A4[b,r]   (Eq. cp4)."""
    A1, A2, A3, A4 = A
    R = A1.shape[1]
    lam = np.ones(R) if lam is None else np.asarray(lam, dtype=np.float64)
    return np.einsum("r,ir,ar,jr,br->iajb", lam, A1, A2, A3, A4, optimize=False)


def mttkrp_explicit(G, A, mode):
    """Standard MTTKRP of the explicit 4-way tensor: the mode-`mode` unfolding of G times
    the Khatri-Rao product of the other three factors (lam not applied)."""
    A1, A2, A3, A4 = A
    if mode == 0:
        return np.einsum("iajb,ar,jr,br->ir", G, A2, A3, A4, optimize=False)
    if mode == 1:
        return np.einsum("iajb,ir,jr,br->ar", G, A1, A3, A4, optimize=False)
    if mode == 2:
        return np.einsum("iajb,ir,ar,br->jr", G, A1, A2, A4, optimize=False)
    if mode == 3:
        return np.einsum("iajb,ir,ar,jr->br", G, A1, A2, A3, optimize=False)
    raise ValueError("mode must be 0..3")


def frobenius2(T):
    return float(np.sum(T * T))


# --------------------------------------------------------------------------------------
# matrix-free forms through the THC factors (Sec. 2.1: gradients of Eq. lossF without
# forming the N^4 tensor)
# --------------------------------------------------------------------------------------
def project(Xo, Xv, A):
    """Grid projections W_k = X_k^T A_k with X = (Xo, Xv, Xo, Xv) for modes (i, a, j, b)."""
    X = (Xo, Xv, Xo, Xv)
    return tuple(X[k].T @ A[k] for k in range(4))


def mttkrp(Xo, Xv, Z, A, mode):
    """Matrix-free MTTKRP, obtained by substituting Eq. THC into the MTTKRP and summing
    the three free orbital indices inside out:

      M1 = Xo (W2 o (Z   (W3 o W4)))      M2 = Xv (W1 o (Z   (W3 o W4)))
      M3 = Xo (W4 o (Z^T (W1 o W2)))      M4 = Xv (W3 o (Z^T (W1 o W2)))

    with W_k = X_k^T A_k and o the Hadamard product. lam is not applied.
    """
    W1, W2, W3, W4 = project(Xo, Xv, A)
    if mode in (0, 1):
        Y = Z @ (W3 * W4)
        return Xo @ (W2 * Y) if mode == 0 else Xv @ (W1 * Y)
    if mode in (2, 3):
        Y = Z.T @ (W1 * W2)
        return Xo @ (W4 * Y) if mode == 2 else Xv @ (W3 * Y)
    raise ValueError("mode must be 0..3")


def thc_norm2(Xo, Xv, Z):
    """||G||^2 = sum_PQ Z[P,Q] (S Z S)[P,Q] with S = (Xo^T Xo) o (Xv^T Xv).

    Same contraction pattern as the O(R_THC^3) J-term of Eq. thc_Ej: expanding G^2 pairs
    grid indices P,P' (particle 1) and Q,Q' (particle 2) through the Grams of Xo and Xv.
    """
    S = (Xo.T @ Xo) * (Xv.T @ Xv)
    return float(np.sum(Z * (S @ Z @ S)))


def grams(A):
    return tuple(a.T @ a for a in A)


def cpd_norm2(A, lam):
    """||Gt||^2 = lam^T (G1 o G2 o G3 o G4) lam   (Eq. cp4, Gram form)."""
    G1, G2, G3, G4 = grams(A)
    return float(lam @ ((G1 * G2 * G3 * G4) @ lam))


def inner_thc_cpd(Xo, Xv, Z, A, lam):
    """<G, Gt> = sum_{P,Q,r} lam_r (W1 o W2)[P,r] Z[P,Q] (W3 o W4)[Q,r]."""
    W1, W2, W3, W4 = project(Xo, Xv, A)
    return float(np.sum(lam[None, :] * (W1 * W2) * (Z @ (W3 * W4))))


def loss_factor_form(Xo, Xv, Z, A, lam, normG2=None):
    """||G - Gt||^2 = ||G||^2 - 2 <G, Gt> + ||Gt||^2, all in factor form."""
    lam = np.asarray(lam, dtype=np.float64)
    nG2 = thc_norm2(Xo, Xv, Z) if normG2 is None else normG2
    return nG2 - 2.0 * inner_thc_cpd(Xo, Xv, Z, A, lam) + cpd_norm2(A, lam)


def fit_from_loss(loss, normG2):
    """fit = 1 - ||G - Gt|| / ||G||; negative round-off losses clamp to 0."""
    return 1.0 - np.sqrt(max(loss, 0.0)) / np.sqrt(normG2)


def loss_explicit(Xo, Xv, Z, A, lam):
    G = thc_tensor(Xo, Xv, Z)
    Gt = cpd_tensor(A, lam)
    return frobenius2(G - Gt)


# --------------------------------------------------------------------------------------
# ALS (textbook CP-ALS applied to Eq. lossF)
# --------------------------------------------------------------------------------------
def hadamard_of_grams(A, k):
    """H_k = Hadamard product of A_m^T A_m over the three modes m != k."""
    R = A[0].shape[1]
    H = np.ones((R, R))
    for m in range(4):
        if m != k:
            H = H * (A[m].T @ A[m])
    return H


def solve_normal_equations(M, H):
    """A = M H^{-1} for symmetric positive semidefinite H.

    Cholesky H = L L^T, then two triangular solves. If a pivot is <= R*eps*max diag(H)
    (or not finite) the pseudo-inverse from eigh(H) is used: eigenvalues at or below
    R*eps*max|w| are dropped. Returns (A, used_pinv).
    """
    R = H.shape[0]
    tau = R * EPS * float(np.max(np.diag(H))) if R else 0.0
    ok = np.all(np.isfinite(H))
    L = None
    if ok:
        try:
            L = np.linalg.cholesky(H)
        except np.linalg.LinAlgError:
            L = None
    if L is not None:
        piv = np.diag(L) ** 2
        if not (np.all(np.isfinite(piv)) and np.all(piv > tau)):
            L = None
    if L is not None:
        # A H = M  <=>  L (L^T A^T) = M^T
        Yt = sla.solve_triangular(L, M.T, lower=True)
        At = sla.solve_triangular(L.T, Yt, lower=False)
        return At.T, False
    w, V = np.linalg.eigh(H)
    cut = R * EPS * float(np.max(np.abs(w))) if R else 0.0
    keep = w > cut
    inv = np.zeros_like(w)
    inv[keep] = 1.0 / w[keep]
    Hp = (V * inv[None, :]) @ V.T
    return M @ Hp, True


def normalise_columns(A):
    """lam_r = ||A[:, r]||_2, A[:, r] /= lam_r (zero columns keep lam_r = 0)."""
    lam = np.sqrt(np.sum(A * A, axis=0))
    safe = np.where(lam > 0.0, lam, 1.0)
    return A / safe[None, :], lam


def als_mode_update(Xo, Xv, Z, A, k):
    """One ALS block update of mode k. Returns (new factor list, lam, used_pinv, M, H)."""
    M = mttkrp(Xo, Xv, Z, A, k)
    H = hadamard_of_grams(A, k)
    Ak, used_pinv = solve_normal_equations(M, H)
    Ak, lam = normalise_columns(Ak)
    A = list(A)
    A[k] = Ak
    return tuple(A), lam, used_pinv, M, H


def als_sweep(Xo, Xv, Z, A, lam=None, normG2=None):
    """One ALS sweep over modes 0..3; returns (A, lam, loss, fit, pinv_flags)."""
    nG2 = thc_norm2(Xo, Xv, Z) if normG2 is None else normG2
    flags = []
    for k in range(4):
        A, lam, used, _, _ = als_mode_update(Xo, Xv, Z, A, k)
        flags.append(used)
    loss = loss_factor_form(Xo, Xv, Z, A, lam, nG2)
    return A, lam, loss, fit_from_loss(loss, nG2), flags


def als(Xo, Xv, Z, A, max_sweeps, tol=0.0, lam=None):
    """CP-ALS driven by the THC factors. Stops after max_sweeps or when
    |fit_s - fit_{s-1}| < tol (tol <= 0: run all sweeps).

    Returns dict(A, lam, losses, fits, pinv, sweeps, normG2)."""
    nG2 = thc_norm2(Xo, Xv, Z)
    R = A[0].shape[1]
    lam = np.ones(R) if lam is None else lam
    losses, fits, pinv = [], [], []
    prev = None
    s = 0
    for s in range(1, max_sweeps + 1):
        A, lam, loss, fit, flags = als_sweep(Xo, Xv, Z, A, lam, nG2)
        losses.append(loss)
        fits.append(fit)
        pinv.append(any(flags))
        if tol > 0 and prev is not None and abs(fit - prev) < tol:
            break
        prev = fit
    return dict(A=A, lam=lam, losses=losses, fits=fits, pinv=pinv, sweeps=s, normG2=nG2)


# --------------------------------------------------------------------------------------
# extrapolated ALS step (learned line search; the accept rule is the exact loss)
# --------------------------------------------------------------------------------------
def extrapolate(A_prev, lam_prev, A_new, lam_new, alpha):
    """Trial point on lam-absorbed factors: B_k = P_k + alpha (N_k - P_k), where the last
    mode carries lam (A4 * lam); the trial is re-normalised column-wise afterwards."""
    P = [a.copy() for a in A_prev]
    N = [a.copy() for a in A_new]
    P[3] = P[3] * lam_prev[None, :]
    N[3] = N[3] * lam_new[None, :]
    B = [p + alpha * (n - p) for p, n in zip(P, N)]
    lam = np.ones(B[0].shape[1])
    out = []
    for b in B:
        b, l = normalise_columns(b)
        out.append(b)
        lam = lam * l
    return tuple(out), lam
