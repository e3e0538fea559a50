"""FP64 oracle of THC-driven CP-ALS for order-d THC-like tensors (Conclusions: the
decomposition strategy applies to any THC-like tensor network of order d, at O(N R^2)
per gradient instead of O(N^d R_thc)).

TEST INFRASTRUCTURE ONLY: used by tests/ (nothing in the library imports it).

Reading (the paper states the generalisation but not its form): the d modes are split
into a left group L = {0 .. dL-1} bound to one grid index P and a right group
R = {dL .. d-1} bound to Q, each mode k with its own grid factor X_k (n_k x R_thc):
    G[i_0 .. i_{d-1}] = sum_{P,Q} prod_{k in L} X_k[i_k,P] Z[P,Q] prod_{k in R} X_k[i_k,Q].
The order-4 block of Eq. THC is d = 4, dL = 2, X = (Xo, Xv, Xo, Xv). The CPD is
Gt = sum_r lam_r prod_k A_k[i_k, r] (Eq. cp4 with d factors).
Matrix-free MTTKRP (substitute G into the standard MTTKRP and sum every mode except k
inside out), with the projections W_m = X_m^T A_m (R_thc x R) and o the Hadamard product:
    k in L:  M_k = X_k ( (o_{m in L, m != k} W_m) o (Z (o_{m in R} W_m)) )
    k in R:  M_k = X_k ( (o_{m in R, m != k} W_m) o (Z^T (o_{m in L} W_m)) )
(an empty Hadamard product is all ones). Norms and inner product in factor form:
    ||G||^2 = sum Z o (S_L Z S_R),  S_L = o_{m in L} X_m^T X_m,  S_R = o_{m in R} X_m^T X_m
    <G, Gt> = sum_r lam_r sum_{P,Q} (o_L W)[P,r] Z[P,Q] (o_R W)[Q,r]
    ||Gt||^2 = lam^T (o_k A_k^T A_k) lam.
ALS steps as in oracle/thc_cpd.py (normal equations with H_k = o_{m != k} A_m^T A_m,
Cholesky with the pseudo-inverse fallback, column normalisation, Gauss-Seidel over
k = 0 .. d-1, factor-form loss, |fit change| < tol), whose solve and normalisation this
module calls.
"""
from __future__ import annotations

import string

import numpy as np

from .thc_cpd import fit_from_loss, normalise_columns, solve_normal_equations


def _hadamard(mats, shape):
    out = np.ones(shape)
    for m in mats:
        out = out * m
    return out


def nd_tensor(X, Z, dL):
    """Explicit order-d THC-like tensor (tiny sizes)."""
    d = len(X)
    letters = string.ascii_lowercase
    left = ",".join(f"{letters[k]}P" for k in range(dL))
    right = ",".join(f"{letters[k]}Q" for k in range(dL, d))
    spec = f"{left},PQ,{right}->{letters[:d]}"
    return np.einsum(spec, *X[:dL], Z, *X[dL:], optimize=True)


def nd_cpd_tensor(A, lam=None):
    """Gt = sum_r lam_r prod_k A_k[i_k, r] (explicit)."""
    d = len(A)
    R = A[0].shape[1]
    lam = np.ones(R) if lam is None else np.asarray(lam)
    letters = string.ascii_lowercase
    spec = "z," + ",".join(f"{letters[k]}z" for k in range(d)) + f"->{letters[:d]}"
    return np.einsum(spec, lam, *A, optimize=True)


def nd_mttkrp_explicit(G, A, k):
    """Standard MTTKRP of an explicit order-d tensor: unfold mode k and multiply by the
    Khatri-Rao product of the other factors (in mode order)."""
    d = G.ndim
    others = [m for m in range(d) if m != k]
    Gk = np.moveaxis(G, k, 0).reshape(G.shape[k], -1)
    R = A[0].shape[1]
    KR = np.ones((1, R))
    for m in others:
        KR = (KR[:, None, :] * A[m][None, :, :]).reshape(-1, R)
    return Gk @ KR


def nd_project(X, A):
    return [x.T @ a for x, a in zip(X, A)]


def nd_mttkrp(X, Z, dL, A, k):
    """Matrix-free MTTKRP of mode k (lam not applied)."""
    d = len(X)
    W = nd_project(X, A)
    shape = W[0].shape
    if k < dL:
        own = _hadamard([W[m] for m in range(dL) if m != k], shape)
        Y = Z @ _hadamard([W[m] for m in range(dL, d)], shape)
    else:
        own = _hadamard([W[m] for m in range(dL, d) if m != k], shape)
        Y = Z.T @ _hadamard([W[m] for m in range(dL)], shape)
    return X[k] @ (own * Y)


def nd_norm2(X, Z, dL):
    Rt = Z.shape[0]
    SL = _hadamard([x.T @ x for x in X[:dL]], (Rt, Rt))
    SR = _hadamard([x.T @ x for x in X[dL:]], (Rt, Rt))
    return float(np.sum(Z * (SL @ Z @ SR)))


def nd_inner(X, Z, dL, A, lam):
    W = nd_project(X, A)
    shape = W[0].shape
    PL = _hadamard(W[:dL], shape)
    PR = _hadamard(W[dL:], shape)
    return float(np.sum(np.asarray(lam)[None, :] * PL * (Z @ PR)))


def nd_cpd_norm2(A, lam):
    R = A[0].shape[1]
    H = _hadamard([a.T @ a for a in A], (R, R))
    lam = np.asarray(lam)
    return float(lam @ H @ lam)


def nd_loss(X, Z, dL, A, lam, normG2=None):
    nG2 = nd_norm2(X, Z, dL) if normG2 is None else normG2
    return nG2 - 2.0 * nd_inner(X, Z, dL, A, lam) + nd_cpd_norm2(A, lam)


def nd_als(X, Z, dL, A, max_sweeps, tol=0.0, lam=None):
    """Order-d THC-driven CP-ALS; returns dict(A, lam, losses, fits, pinv, sweeps, normG2)."""
    d = len(X)
    nG2 = nd_norm2(X, Z, dL)
    R = A[0].shape[1]
    lam = np.ones(R) if lam is None else lam
    A = list(A)
    losses, fits, pinv = [], [], []
    prev = None
    s = 0
    for s in range(1, max_sweeps + 1):
        flags = []
        for k in range(d):
            M = nd_mttkrp(X, Z, dL, A, k)
            H = _hadamard([A[m].T @ A[m] for m in range(d) if m != k], (R, R))
            Ak, used = solve_normal_equations(M, H)
            A[k], lam = normalise_columns(Ak)
            flags.append(used)
        loss = nd_loss(X, Z, dL, A, lam, nG2)
        fit = fit_from_loss(loss, nG2)
        losses.append(loss)
        fits.append(fit)
        pinv.append(any(flags))
        if tol > 0 and prev is not None and abs(fit - prev) < tol:
            break
        prev = fit
    return dict(A=tuple(A), lam=lam, losses=losses, fits=fits, pinv=pinv, sweeps=s, normG2=nG2)
