"""FP64 oracle of DF-driven CP-ALS, the prior-work variant of the paper (Sec. 2.1, Eq. df_loss):
CP-ALS of the (o,v,o,v) block of density-fitted integrals
    G_DF[i,a,j,b] = sum_X B[X,i,a] B[X,j,b]
with its gradients (MTTKRPs) formed matrix-free from the order-3 DF tensor B (naux x o x v)
at O(naux o v R) per mode, instead of from THC factors at O((o + v) R_thc R + R_thc^2 R).

TEST INFRASTRUCTURE ONLY: used by tests/ (nothing in the library imports it).

MTTKRP in DF form (substitute G_DF into the standard MTTKRP and sum the particle-2 pair
first): with the pair projections
    V12[X,r] = sum_{i,a} B[X,i,a] A1[i,r] A2[a,r],   V34[X,r] = sum_{j,b} B[X,j,b] A3[j,r] A4[b,r]
    M1[i,r] = sum_X (sum_a B[X,i,a] A2[a,r]) V34[X,r]      M2[a,r] = sum_X (sum_i B[X,i,a] A1[i,r]) V34[X,r]
    M3[j,r] = sum_X (sum_b B[X,j,b] A4[b,r]) V12[X,r]      M4[b,r] = sum_X (sum_j B[X,j,b] A3[j,r]) V12[X,r]
Loss in factor form: ||G_DF||^2 = ||D D^T||_F^2 (D[X,(i,a)] = B[X,i,a]),
<G_DF, Gt> = sum_r lam_r sum_X V12[X,r] V34[X,r], ||Gt||^2 = lam^T (G1 o G2 o G3 o G4) lam.
The ALS steps (normal equations, Cholesky with the pseudo-inverse fallback, column
normalisation, Gauss-Seidel order, fit and stopping rule) are those of the THC-driven oracle
(oracle/thc_cpd.py), which this module calls; only the MTTKRP and the loss differ.
"""
from __future__ import annotations

import numpy as np

from .thc_cpd import (cpd_norm2, fit_from_loss, hadamard_of_grams, normalise_columns,
                      solve_normal_equations)


def df_tensor(B):
    """G_DF[i,a,j,b] = sum_X B[X,i,a] B[X,j,b] (explicit; tiny sizes)."""
    return np.einsum("xia,xjb->iajb", B, B, optimize=False)


def pair_projection(B, Ap, Aq):
    """V[X,r] = sum_{i,a} B[X,i,a] Ap[i,r] Aq[a,r] (the first index of B with Ap)."""
    return np.einsum("xia,ir,ar->xr", B, Ap, Aq, optimize=True)


def df_mttkrp(B, A, mode):
    """DF-form MTTKRP of G_DF with the other three factors (lam not applied)."""
    A1, A2, A3, A4 = A
    if mode in (0, 1):
        V = pair_projection(B, A3, A4)
        if mode == 0:
            T = np.einsum("xia,ar->xir", B, A2, optimize=True)
        else:
            T = np.einsum("xia,ir->xar", B, A1, optimize=True)
    else:
        V = pair_projection(B, A1, A2)
        if mode == 2:
            T = np.einsum("xjb,br->xjr", B, A4, optimize=True)
        else:
            T = np.einsum("xjb,jr->xbr", B, A3, optimize=True)
    return np.einsum("xnr,xr->nr", T, V, optimize=True)


def df_norm2(B):
    """||G_DF||^2 = ||D D^T||_F^2 with D the (naux x o v) matricisation of B."""
    D = B.reshape(B.shape[0], -1)
    Q = D @ D.T
    return float(np.sum(Q * Q))


def df_inner(B, A, lam):
    """<G_DF, Gt> = sum_r lam_r sum_X V12[X,r] V34[X,r]."""
    A1, A2, A3, A4 = A
    return float(np.sum(np.asarray(lam)[None, :] * pair_projection(B, A1, A2) * pair_projection(B, A3, A4)))


def df_loss(B, A, lam, normG2=None):
    """||G_DF - Gt||^2 in factor form."""
    nG2 = df_norm2(B) if normG2 is None else normG2
    return nG2 - 2.0 * df_inner(B, A, lam) + cpd_norm2(A, lam)


def df_als_sweep(B, A, lam, normG2):
    """One DF-driven ALS sweep over modes 0..3: (A, lam, loss, fit, pinv_flags)."""
    flags = []
    for k in range(4):
        M = df_mttkrp(B, A, k)
        H = hadamard_of_grams(A, k)
        Ak, used = solve_normal_equations(M, H)
        Ak, lam = normalise_columns(Ak)
        A = list(A)
        A[k] = Ak
        A = tuple(A)
        flags.append(used)
    loss = df_loss(B, A, lam, normG2)
    return A, lam, loss, fit_from_loss(loss, normG2), flags


def df_als(B, A, max_sweeps, tol=0.0, lam=None):
    """DF-driven CP-ALS; same stopping rule and return dict as oracle.thc_cpd.als."""
    nG2 = df_norm2(B)
    R = A[0].shape[1]
    lam = np.ones(R) if lam is None else lam
    losses, fits, pinv = [], [], []
    prev = None
    s = 0
    for s in range(1, max_sweeps + 1):
        A, lam, loss, fit, flags = df_als_sweep(B, A, lam, nG2)
        losses.append(loss)
        fits.append(fit)
        pinv.append(any(flags))
        if tol > 0 and prev is not None and abs(fit - prev) < tol:
            break
        prev = fit
    return dict(A=A, lam=lam, losses=losses, fits=fits, pinv=pinv, sweeps=s, normG2=nG2)
