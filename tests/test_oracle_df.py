"""Pins of the DF-driven CP-ALS oracle (oracle/df_cpd.py): MTTKRP, norm and loss against the
explicit DF tensor by brute force, exact rank-1 recovery, and the cross-check that makes the
two drivers meet: a DF tensor that is exactly an order-3 CPD on the THC grid gives
G_DF = G_THC with Z = C^T C, so DF-driven and THC-driven ALS must follow the same
trajectory from the same start."""
import numpy as np
import pytest

from oracle import df_cpd as D
from oracle import thc_cpd as O
from thc_inputs import make_df, make_factors


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("seed,o,v,naux,R", [(0, 2, 3, 4, 3), (1, 3, 5, 2, 4)])
def test_df_mttkrp_matches_explicit(mode, seed, o, v, naux, R):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((naux, o, v))
    A = make_factors((o, v, o, v), R, seed)
    G = D.df_tensor(B)
    Me = O.mttkrp_explicit(G, A, mode)
    Mf = D.df_mttkrp(B, A, mode)
    assert np.max(np.abs(Mf - Me)) <= 1e-12 * np.max(np.abs(Me))


def test_df_tensor_brute_force():
    rng = np.random.default_rng(3)
    B = rng.standard_normal((3, 2, 3))
    G = D.df_tensor(B)
    for i in range(2):
        for a in range(3):
            for j in range(2):
                for b in range(3):
                    assert abs(G[i, a, j, b] - sum(B[x, i, a] * B[x, j, b] for x in range(3))) < 1e-13


def test_df_norm_and_loss_match_explicit():
    rng = np.random.default_rng(4)
    B = rng.standard_normal((4, 3, 5))
    A = make_factors((3, 5, 3, 5), 4, 4)
    lam = rng.uniform(0.5, 2.0, 4)
    G = D.df_tensor(B)
    assert abs(D.df_norm2(B) - np.sum(G * G)) <= 1e-12 * np.sum(G * G)
    Gt = O.cpd_tensor(A, lam)
    le = float(np.sum((G - Gt) ** 2))
    assert abs(D.df_loss(B, A, lam) - le) <= 1e-11 * (np.sum(G * G) + np.sum(Gt * Gt))


def test_rank_one_df_block_is_recovered():
    # naux = 1 and B[0] = u v^T: G_DF = u o v o u o v, an exact rank-1 CPD
    rng = np.random.default_rng(5)
    u, w = rng.standard_normal(4), rng.standard_normal(6)
    B = np.outer(u, w)[None, :, :]
    A = make_factors((4, 6, 4, 6), 1, 5)
    r = D.df_als(B, A, 30, tol=0.0)
    assert r["fits"][-1] > 1.0 - 1e-7


def test_df_and_thc_drivers_follow_one_trajectory():
    o, v, Rt, naux, R = 3, 6, 8, 10, 5
    Xo, Xv, B = make_df(o, v, Rt, naux, seed=2, noise=0.0)
    rng = np.random.default_rng([2, 0xDF])
    C = rng.standard_normal((naux, Rt)) / np.sqrt(Rt)
    Z = C.T @ C
    assert abs(D.df_norm2(B) - O.thc_norm2(Xo, Xv, Z)) <= 1e-12 * D.df_norm2(B)
    A = make_factors((o, v, o, v), R, 7)
    rd = D.df_als(B, A, 8)
    rt = O.als(Xo, Xv, Z, A, 8)
    assert np.max(np.abs(np.array(rd["fits"]) - np.array(rt["fits"]))) <= 1e-10
    for a, b in zip(rd["A"], rt["A"]):
        assert np.max(np.abs(a - b)) <= 1e-8


def test_planted_slip_misses_the_explicit_mttkrp():
    rng = np.random.default_rng(6)
    B = rng.standard_normal((4, 3, 5))
    A = make_factors((3, 5, 3, 5), 3, 6)
    Me = O.mttkrp_explicit(D.df_tensor(B), A, 0)
    # mode 0 with the wrong pair projection (its own particle's V12 instead of V34)
    T = np.einsum("xia,ar->xir", B, A[1])
    slip = np.einsum("xir,xr->ir", T, D.pair_projection(B, A[0], A[1]))
    assert np.max(np.abs(slip - Me)) > 1e-3 * np.max(np.abs(Me))
    # the contraction of the right index of B for mode 1 (a) replaced by the left one
    V = D.pair_projection(B, A[2], A[3])
    T2 = np.einsum("xia,ir->xar", B, A[0])
    good = np.einsum("xar,xr->ar", T2, V)
    Me1 = O.mttkrp_explicit(D.df_tensor(B), A, 1)
    assert np.max(np.abs(good - Me1)) <= 1e-12 * np.max(np.abs(Me1))
