"""Pins of the THC core-fit oracle (oracle/corefit.py) against what the mathematics fixes:
the least-squares solution of the vectorised problem by numpy's lstsq, exact recovery of a
core that generated the DF tensor, stationarity of the explicit residual, the factor-form
loss against the explicit tensors, and planted slips that must miss these pins."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import corefit as C
from thc_inputs import make_df


def _tiny(seed=0, o=2, v=3, Rt=4, naux=5, noise=0.3):
    return make_df(o, v, Rt, naux, seed=seed, noise=noise)


@pytest.mark.parametrize("seed,o,v,Rt,naux", [(0, 2, 3, 4, 5), (1, 3, 2, 5, 4), (2, 2, 4, 6, 7)])
def test_normal_equations_match_least_squares(seed, o, v, Rt, naux):
    Xo, Xv, B = _tiny(seed, o, v, Rt, naux)
    Z = C.core_fit(Xo, Xv, B)
    Zl = C.core_fit_explicit(Xo, Xv, B)
    assert np.max(np.abs(Z - Zl)) <= 1e-9 * np.max(np.abs(Zl))
    assert np.max(np.abs(Z - Z.T)) <= 1e-10 * np.max(np.abs(Z))


def test_exact_recovery_of_a_generating_core():
    # B = CPD(C, Xo, Xv) exactly -> G_DF = K (C^T C) K^T, so Z* = C^T C when K has full rank
    Xo, Xv, B = make_df(3, 5, 6, 8, seed=3, noise=0.0)
    rng = np.random.default_rng([3, 0xDF])
    Cg = rng.standard_normal((8, 6)) / np.sqrt(6)
    Z = C.core_fit(Xo, Xv, B)
    assert np.allclose(Z, Cg.T @ Cg, rtol=0, atol=1e-9 * np.max(np.abs(Cg.T @ Cg)))
    assert C.core_loss_explicit(Xo, Xv, B, Z) <= 1e-20 * np.sum(C.df_tensor(B) ** 2)


def test_stationarity_and_minimum():
    Xo, Xv, B = _tiny(4, 3, 4, 5, 6)
    Z = C.core_fit(Xo, Xv, B)
    K = C.pair_matrix(Xo, Xv)
    ov = K.shape[0]
    resid = C.df_tensor(B).reshape(ov, ov) - K @ Z @ K.T
    g = K.T @ resid @ K
    assert np.max(np.abs(g)) <= 1e-10 * np.max(np.abs(K.T @ C.df_tensor(B).reshape(ov, ov) @ K))
    f0 = C.core_loss_explicit(Xo, Xv, B, Z)
    rng = np.random.default_rng(9)
    for _ in range(5):
        d = rng.standard_normal(Z.shape) * 1e-3
        assert C.core_loss_explicit(Xo, Xv, B, Z + d) > f0


@pytest.mark.parametrize("seed", [0, 1])
def test_factor_form_loss_matches_explicit(seed):
    Xo, Xv, B = _tiny(seed, 3, 4, 5, 6)
    rng = np.random.default_rng(seed + 7)
    Z = rng.standard_normal((5, 5))  # any Z, not symmetric
    le = C.core_loss_explicit(Xo, Xv, B, Z)
    lf = C.core_loss(Xo, Xv, B, Z)
    assert abs(le - lf) <= 1e-10 * (np.sum(C.df_tensor(B) ** 2) + le)


def test_normal_terms_against_brute_force():
    Xo, Xv, B = _tiny(5, 2, 3, 4, 3)
    S, E = C.core_normal_terms(Xo, Xv, B)
    naux, o, v = B.shape
    Rt = Xo.shape[1]
    Sb = np.zeros((Rt, Rt))
    Eb = np.zeros((naux, Rt))
    for P in range(Rt):
        for Q in range(Rt):
            Sb[P, Q] = sum(Xo[i, P] * Xv[a, P] * Xo[i, Q] * Xv[a, Q] for i in range(o) for a in range(v))
        for X in range(naux):
            Eb[X, P] = sum(B[X, i, a] * Xo[i, P] * Xv[a, P] for i in range(o) for a in range(v))
    assert np.allclose(S, Sb, rtol=1e-13, atol=0)
    assert np.allclose(E, Eb, rtol=1e-13, atol=1e-15)


def test_planted_slips_miss_the_pins():
    Xo, Xv, B = _tiny(0)
    Zl = C.core_fit_explicit(Xo, Xv, B)
    S, E = C.core_normal_terms(Xo, Xv, B)
    rhs = E.T @ E
    tol = 1e-6 * np.max(np.abs(Zl))
    # S applied on one side only
    assert np.max(np.abs(np.linalg.solve(S, rhs) - Zl)) > tol
    # matrix product of the Grams instead of their Hadamard product
    S2 = (Xo.T @ Xo) @ (Xv.T @ Xv)
    S2 = 0.5 * (S2 + S2.T) + 10 * np.eye(S2.shape[0])
    Y = np.linalg.solve(S2, rhs)
    assert np.max(np.abs(np.linalg.solve(S2, Y.T).T - Zl)) > tol
    # E with the occupied factor contracted twice (Xv dropped)
    Eb = np.einsum("xia,ip->xp", B, Xo)
    c = sla.cho_factor(S, lower=True)
    Zb = sla.cho_solve(c, sla.cho_solve(c, Eb.T @ Eb).T).T
    assert np.max(np.abs(Zb - Zl)) > tol
