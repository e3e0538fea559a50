"""FP64 oracle of the CPD+THC LT-MP2 exchange energy (Sec. 2.2, Eq. thc_Ek, Eq. cpd_single_k,
the double-CPD term after it, and Eq. rob_K).

TEST INFRASTRUCTURE ONLY: used by tests/ (and nothing in the library imports it).

Objects, in the index order of the THC block G[i, a, j, b] = (ia|jb) used everywhere here
(i, j occupied; a, b virtual):
  Laplace quadrature (Eq. lt_D) with points t_alpha, weights w_alpha; per point the
    occupied and virtual factors (the Gamma / Lambda matrices after Eq. mp1_t)
      Lam[alpha, i] = |w|^(1/4) exp((eps_i - eps_f) t / 2)
      Gam[alpha, a] = |w|^(1/4) exp((eps_f - eps_a) t / 2)
  amplitudes (Eq. mp1_t) of a tensor X:  t_alpha[i,a,j,b] = Lam_i Gam_a Lam_j Gam_b X[i,a,j,b]
  exchange of amplitudes T and integrals Y (Eq. thc_Ek):
      K(T, Y) = - sum_alpha sum_{iajb} t_alpha[i,a,j,b] Y[i,b,j,a]   (a and b swapped)
  with the THC block G and the CPD Gt (Eq. cp4):
      E_THC    = K(G, G)            the THC exchange, O(N^4) or O(N^2 R_thc^2)
      E_single = K(G, Gt)           Eq. cpd_single_k, one tensor replaced by its CPD
      E_double = K(Gt, Gt)          both replaced
      E_robust = 2 E_single - E_double                                  (Eq. rob_K)
Because w is symmetric in a and b, K is a symmetric bilinear form, so with Gt = G - D:
      E_robust - E_THC = - K(D, D)
(the robust form has no error of first order in the CPD error D). The tests pin that
identity, the explicit forms against brute force and the factor forms against the explicit
ones.

Factor forms (matrix-free, the paper's contraction orders), per quadrature point:
  single:  U1 = (Lam o Xo)^T A1, U4 = (Gam o Xv)^T A4, U3 = (Lam o Xo)^T A3, U2 = (Gam o Xv)^T A2
           E_single = - sum_{P,r} lam_r (U1 o U4)[P, r] (Z (U3 o U2))[P, r]          O(R_thc^2 R)
  double:  M1 = A1^T diag(Lam) A1, M3 = A3^T diag(Lam) A3, N = A2^T diag(Gam) A4
           E_double = - lam^T (M1 o N o M3 o N^T) lam                             O(N R^2)
"""
from __future__ import annotations

import numpy as np

from .thc_cpd import cpd_tensor, thc_tensor


def lt_factors(eps_occ, eps_vir, t, w):
    """Lam (n_alpha x o) and Gam (n_alpha x v) of the Laplace quadrature (t, w), with eps_f
    midway between the highest occupied and the lowest virtual level."""
    eps_occ = np.asarray(eps_occ, dtype=np.float64)
    eps_vir = np.asarray(eps_vir, dtype=np.float64)
    eps_f = 0.5 * (np.max(eps_occ) + np.min(eps_vir))
    t = np.asarray(t, dtype=np.float64)[:, None]
    q = np.abs(np.asarray(w, dtype=np.float64))[:, None] ** 0.25
    Lam = q * np.exp((eps_occ[None, :] - eps_f) * t / 2.0)
    Gam = q * np.exp((eps_f - eps_vir[None, :]) * t / 2.0)
    return Lam, Gam


def exchange_explicit(T, Y, Lam, Gam):
    """K(T, Y) = - sum_alpha sum_{iajb} Lam_i Gam_a Lam_j Gam_b T[i,a,j,b] Y[i,b,j,a]."""
    Ys = np.transpose(Y, (0, 3, 2, 1))  # Ys[i,a,j,b] = Y[i,b,j,a]
    e = 0.0
    for al in range(Lam.shape[0]):
        w = np.einsum("i,a,j,b->iajb", Lam[al], Gam[al], Lam[al], Gam[al], optimize=False)
        e -= float(np.sum(w * T * Ys))
    return e


def exchange_energies_explicit(Xo, Xv, Z, A, lam, Lam, Gam):
    """(E_THC, E_single, E_double, E_robust) from the explicit tensors (tiny sizes)."""
    G = thc_tensor(Xo, Xv, Z)
    Gt = cpd_tensor(A, lam)
    e_thc = exchange_explicit(G, G, Lam, Gam)
    e1 = exchange_explicit(G, Gt, Lam, Gam)
    e2 = exchange_explicit(Gt, Gt, Lam, Gam)
    return e_thc, e1, e2, 2.0 * e1 - e2


def exchange_single(Xo, Xv, Z, A, lam, Lam, Gam):
    """E_single in factor form (Eq. cpd_single_k, contraction order of the paper)."""
    A1, A2, A3, A4 = A
    lam = np.asarray(lam, dtype=np.float64)
    e = 0.0
    for al in range(Lam.shape[0]):
        XoL = Lam[al][:, None] * Xo
        XvG = Gam[al][:, None] * Xv
        U1, U3 = XoL.T @ A1, XoL.T @ A3
        U2, U4 = XvG.T @ A2, XvG.T @ A4
        e -= float(np.sum(lam[None, :] * (U1 * U4) * (Z @ (U3 * U2))))
    return e


def exchange_double(A, lam, Lam, Gam):
    """E_double in factor form (the double-CPD term of Sec. 2.2)."""
    A1, A2, A3, A4 = A
    lam = np.asarray(lam, dtype=np.float64)
    e = 0.0
    for al in range(Lam.shape[0]):
        M1 = A1.T @ (Lam[al][:, None] * A1)
        M3 = A3.T @ (Lam[al][:, None] * A3)
        N = A2.T @ (Gam[al][:, None] * A4)
        e -= float(lam @ ((M1 * N * M3 * N.T) @ lam))
    return e


def exchange_robust(Xo, Xv, Z, A, lam, Lam, Gam):
    """(E_single, E_double, E_robust = 2 E_single - E_double)   (Eq. rob_K)."""
    e1 = exchange_single(Xo, Xv, Z, A, lam, Lam, Gam)
    e2 = exchange_double(A, lam, Lam, Gam)
    return e1, e2, 2.0 * e1 - e2
