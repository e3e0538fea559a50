"""FP64 oracle of the THC core least-squares fit f(Z) (Sec. 3, Computational Details).

TEST INFRASTRUCTURE ONLY: used by tests/ (nothing in the library imports it).

Inputs: THC grid factors Xo (o x Rt) and Xv (v x Rt) and a density-fitting tensor B
(naux x o x v). The (o,v,o,v) block of the DF integrals (the target of f(Z), the same
product of DF factors as in Eq. df_loss) is
    G_DF[i,a,j,b] = sum_X B[X,i,a] B[X,j,b]
and the THC block on the given factors (Eq. THC) is G_THC(Z) = K Z K^T with the
particle-pair matrix K[(i,a),P] = Xo[i,P] Xv[a,P]. The fit minimises
    f(Z) = 1/2 || G_DF - G_THC(Z) ||^2.
Writing D[X,(i,a)] = B[X,i,a], G_DF = D^T D, and setting the gradient
K^T (K Z K^T - D^T D) K to zero gives the normal equations
    S Z S = E^T E,   S = K^T K = (Xo^T Xo) o (Xv^T Xv),   E = D K,
    E[X,P] = sum_{i,a} B[X,i,a] Xo[i,P] Xv[a,P],
so for S positive definite the minimiser is Z* = S^-1 (E^T E) S^-1 (symmetric).
The loss is reported without the 1/2 (the convention of the CP-ALS loss here):
    ||G_DF - G_THC(Z)||^2 = ||D D^T||_F^2 - 2 <E^T E, Z> + <Z, S Z S>.

Library primitives used as steps: numpy matmul / einsum, scipy's Cholesky factor and solve,
numpy's least squares (the explicit reference only).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def pair_matrix(Xo, Xv):
    """K[(i,a), P] = Xo[i,P] Xv[a,P]  ((o v) x Rt, row index i * v + a)."""
    o, Rt = Xo.shape
    v = Xv.shape[0]
    return (Xo[:, None, :] * Xv[None, :, :]).reshape(o * v, Rt)


def df_tensor(B):
    """G_DF[i,a,j,b] = sum_X B[X,i,a] B[X,j,b] (explicit; tiny sizes)."""
    return np.einsum("xia,xjb->iajb", B, B, optimize=False)


def core_fit_explicit(Xo, Xv, B):
    """argmin_Z ||G_DF - K Z K^T||_F by least squares on the vectorised problem
    (K kron K) vec(Z) = vec(G_DF) (row-major vec; tiny sizes)."""
    K = pair_matrix(Xo, Xv)
    Rt = K.shape[1]
    ov = K.shape[0]
    G = df_tensor(B).reshape(ov * ov)
    z, *_ = np.linalg.lstsq(np.kron(K, K), G, rcond=None)
    return z.reshape(Rt, Rt)


def core_normal_terms(Xo, Xv, B):
    """(S, E): S = (Xo^T Xo) o (Xv^T Xv) (Rt x Rt), E[X,P] = sum_ia B[X,i,a] Xo[i,P] Xv[a,P]."""
    S = (Xo.T @ Xo) * (Xv.T @ Xv)
    naux, o, v = B.shape
    T = (B.reshape(naux * o, v) @ Xv).reshape(naux, o, -1)   # contract the virtual index
    E = np.einsum("xip,ip->xp", T, Xo, optimize=False)       # then the occupied one
    return S, E


def core_fit(Xo, Xv, B):
    """Z* solving the normal equations S Z S = E^T E (Cholesky of S, one solve per side)."""
    S, E = core_normal_terms(Xo, Xv, B)
    rhs = E.T @ E
    c = sla.cho_factor(S, lower=True)
    Y = sla.cho_solve(c, rhs)          # S^-1 (E^T E)
    return sla.cho_solve(c, Y.T).T     # (S^-1 Y^T)^T = S^-1 E^T E S^-1


def core_loss(Xo, Xv, B, Z):
    """||G_DF - G_THC(Z)||^2 in factor form (any Z)."""
    S, E = core_normal_terms(Xo, Xv, B)
    naux = B.shape[0]
    D = B.reshape(naux, -1)
    Q = D @ D.T
    return float(np.sum(Q * Q) - 2.0 * np.sum((E.T @ E) * Z) + np.sum(Z * (S @ Z @ S)))


def core_loss_explicit(Xo, Xv, B, Z):
    """||G_DF - K Z K^T||^2 from the explicit tensors (tiny sizes)."""
    K = pair_matrix(Xo, Xv)
    ov = K.shape[0]
    R = df_tensor(B).reshape(ov, ov) - K @ Z @ K.T
    return float(np.sum(R * R))
