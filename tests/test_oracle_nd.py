"""Pins of the order-d THC-driven CP-ALS oracle (oracle/nd.py): the explicit tensor by brute
force, the matrix-free MTTKRP, norm and loss against the explicit tensor for d = 2 .. 6 and
every split of the modes, the order-4 case against the order-4 oracle (Eq. THC), exact
recovery of a planted order-6 CPD, and planted slips."""
import itertools

import numpy as np
import pytest

from oracle import nd as N
from oracle import thc_cpd as O
from thc_inputs import make_factors, make_nd, make_problem

CASES = [((3, 4), 1), ((2, 3, 4), 1), ((2, 3, 4), 2), ((2, 3, 2, 3), 2), ((3, 2, 2, 3), 1),
         ((2, 2, 3, 2, 2), 2), ((2, 3, 2, 2, 3, 2), 3), ((2, 2, 2, 3, 2, 2), 4)]


def _nonsym(Z, seed):
    rng = np.random.default_rng(seed)
    return Z + 0.3 * rng.standard_normal(Z.shape) * np.max(np.abs(Z))


def test_explicit_tensor_brute_force():
    X, Z, _ = make_nd((2, 3, 2), 4, 2, seed=1)
    Z = _nonsym(Z, 1)
    G = N.nd_tensor(X, Z, 2)
    for i, a, j in itertools.product(range(2), range(3), range(2)):
        ref = sum(X[0][i, P] * X[1][a, P] * Z[P, Q] * X[2][j, Q] for P in range(4) for Q in range(4))
        assert abs(G[i, a, j] - ref) < 1e-14


@pytest.mark.parametrize("dims,dL", CASES)
def test_mttkrp_matches_explicit(dims, dL):
    X, Z, A = make_nd(dims, 5, 3, seed=len(dims) + dL)
    Z = _nonsym(Z, dL)
    G = N.nd_tensor(X, Z, dL)
    for k in range(len(dims)):
        Me = N.nd_mttkrp_explicit(G, A, k)
        Mf = N.nd_mttkrp(X, Z, dL, A, k)
        assert np.max(np.abs(Mf - Me)) <= 1e-12 * np.max(np.abs(Me))


@pytest.mark.parametrize("dims,dL", CASES)
def test_norm_and_loss_match_explicit(dims, dL):
    X, Z, A = make_nd(dims, 5, 3, seed=7 + dL)
    Z = _nonsym(Z, 7)
    lam = np.random.default_rng(3).uniform(0.5, 2.0, 3)
    G = N.nd_tensor(X, Z, dL)
    Gt = N.nd_cpd_tensor(A, lam)
    g2 = float(np.sum(G * G))
    assert abs(N.nd_norm2(X, Z, dL) - g2) <= 1e-12 * g2
    le = float(np.sum((G - Gt) ** 2))
    assert abs(N.nd_loss(X, Z, dL, A, lam) - le) <= 1e-11 * (g2 + float(np.sum(Gt * Gt)))


def test_order4_reduces_to_the_thc_block():
    p = make_problem(3, 7, 12, 9, seed=4)
    X = [p.Xo, p.Xv, p.Xo, p.Xv]
    Z = _nonsym(p.Z, 4)
    for k in range(4):
        assert np.allclose(N.nd_mttkrp(X, Z, 2, p.A, k), O.mttkrp(p.Xo, p.Xv, Z, p.A, k), rtol=1e-12, atol=0)
    rn = N.nd_als(X, p.Z, 2, p.A, 6)
    rt = O.als(p.Xo, p.Xv, p.Z, p.A, 6)
    assert np.max(np.abs(np.array(rn["fits"]) - np.array(rt["fits"]))) <= 1e-12
    for a, b in zip(rn["A"], rt["A"]):
        assert np.max(np.abs(a - b)) <= 1e-10


def test_planted_order6_cpd_is_recovered():
    # X_k = A*_k and Z = I: G = sum_P prod_k A*_k[i_k, P], an exact rank-4 order-6 CPD
    dims, r = (3, 4, 3, 4, 3, 4), 4
    rng = np.random.default_rng(8)
    As = [rng.standard_normal((n, r)) for n in dims]
    A0 = [a * (1.0 + 0.1 * rng.standard_normal(a.shape)) for a in As]
    res = N.nd_als(As, np.eye(r), 3, A0, 200, tol=0.0)
    assert res["fits"][-1] > 1.0 - 1e-8


def test_planted_slips_miss_the_explicit_mttkrp():
    X, Z, A = make_nd((2, 3, 2, 3, 2), 5, 3, seed=9)
    Z = _nonsym(Z, 9)
    G = N.nd_tensor(X, Z, 2)
    k = 3  # a right-group mode
    Me = N.nd_mttkrp_explicit(G, A, k)
    W = N.nd_project(X, A)
    own = W[2] * W[4]
    slip = X[k] @ (own * (Z @ (W[0] * W[1])))  # Z instead of Z^T
    assert np.max(np.abs(slip - Me)) > 1e-3 * np.max(np.abs(Me))
    slip2 = X[k] @ (W[2] * W[3] * W[4] * (Z.T @ (W[0] * W[1])))  # own projection not left out
    assert np.max(np.abs(slip2 - Me)) > 1e-3 * np.max(np.abs(Me))
