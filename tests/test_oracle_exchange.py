"""Pins for the exchange-energy oracle (oracle/exchange.py; Sec. 2.2, Eq. thc_Ek,
Eq. cpd_single_k, the double-CPD term and Eq. rob_K): brute force on tiny inputs, the
factor forms against the explicit tensors, the exact second-order identity of the robust
form, exact CPDs, and planted mistakes."""
import itertools

import numpy as np
import pytest

from oracle import exchange as X
from oracle import thc_cpd as O
from thc_inputs import make_lt, make_planted


def _tiny(seed=0, o=2, v=3, Rt=3, R=2, na=2):
    rng = np.random.default_rng(seed)
    Xo, Xv = rng.standard_normal((o, Rt)), rng.standard_normal((v, Rt))
    Z = rng.standard_normal((Rt, Rt))
    A = tuple(rng.standard_normal((n, R)) for n in (o, v, o, v))
    lam = rng.uniform(0.5, 2.0, R)
    eo, ev, t, w = make_lt(o, v, na, seed)
    Lam, Gam = X.lt_factors(eo, ev, t, w)
    return Xo, Xv, Z, A, lam, Lam, Gam


def _brute_K(T, Y, Lam, Gam):
    o, v = T.shape[0], T.shape[1]
    e = 0.0
    for al in range(Lam.shape[0]):
        for i, a, j, b in itertools.product(range(o), range(v), range(o), range(v)):
            e -= Lam[al, i] * Gam[al, a] * Lam[al, j] * Gam[al, b] * T[i, a, j, b] * Y[i, b, j, a]
    return e


def test_exchange_explicit_matches_brute_force():
    Xo, Xv, Z, A, lam, Lam, Gam = _tiny(1)
    G = O.thc_tensor(Xo, Xv, Z)
    Gt = O.cpd_tensor(A, lam)
    for T, Y in ((G, G), (G, Gt), (Gt, Gt), (Gt, G)):
        assert abs(X.exchange_explicit(T, Y, Lam, Gam) - _brute_K(T, Y, Lam, Gam)) <= 1e-12 * (1 + abs(_brute_K(T, Y, Lam, Gam)))


@pytest.mark.parametrize("seed,shape", [(2, (2, 3, 3, 2, 2)), (3, (3, 5, 7, 4, 3)), (4, (4, 6, 9, 5, 4))])
def test_factor_forms_equal_explicit(seed, shape):
    # non-symmetric Z: a Z / Z^T slip in the single-CPD contraction fails here
    o, v, Rt, R, na = shape
    Xo, Xv, Z, A, lam, Lam, Gam = _tiny(seed, o, v, Rt, R, na)
    _, e1x, e2x, erx = X.exchange_energies_explicit(Xo, Xv, Z, A, lam, Lam, Gam)
    e1, e2, er = X.exchange_robust(Xo, Xv, Z, A, lam, Lam, Gam)
    for got, want in ((e1, e1x), (e2, e2x), (er, erx)):
        assert abs(got - want) <= 1e-12 * (1.0 + abs(want))


def test_robust_error_is_exactly_second_order():
    # Gt = G - D:  E_robust - E_THC = -K(D, D)  (K symmetric: w is symmetric in a, b)
    Xo, Xv, Z, A, lam, Lam, Gam = _tiny(5, 3, 4, 5, 3, 3)
    G = O.thc_tensor(Xo, Xv, Z)
    Gt = O.cpd_tensor(A, lam)
    e_thc, e1, e2, er = X.exchange_energies_explicit(Xo, Xv, Z, A, lam, Lam, Gam)
    D = G - Gt
    assert abs((er - e_thc) - (-X.exchange_explicit(D, D, Lam, Gam))) <= 1e-11 * (1 + abs(e_thc))
    # and the first-order terms do not cancel in the single and double forms alone
    assert abs(e1 - e_thc) > 1e-6 and abs(e2 - e_thc) > 1e-6
    # shrinking the CPD error by s shrinks the robust error by s^2, the single one by s
    for s in (0.1, 0.01):
        Gs = G - s * D
        er_s = 2 * X.exchange_explicit(G, Gs, Lam, Gam) - X.exchange_explicit(Gs, Gs, Lam, Gam)
        e1_s = X.exchange_explicit(G, Gs, Lam, Gam)
        assert abs((er_s - e_thc) / (er - e_thc) - s * s) <= 1e-8
        assert abs((e1_s - e_thc) / (e1 - e_thc) - s) <= 1e-8


def test_exact_cpd_gives_the_thc_exchange_in_every_form():
    p, planted = make_planted(3, 5, 4, 4, seed=7, independent=True)
    eo, ev, t, w = make_lt(3, 5, 4, seed=7)
    Lam, Gam = X.lt_factors(eo, ev, t, w)
    G = O.thc_tensor(p.Xo, p.Xv, p.Z)
    e_thc = X.exchange_explicit(G, G, Lam, Gam)
    e1, e2, er = X.exchange_robust(p.Xo, p.Xv, p.Z, planted, np.ones(4), Lam, Gam)
    for e in (e1, e2, er):
        assert abs(e - e_thc) <= 1e-11 * abs(e_thc)


def test_laplace_quadrature_reproduces_the_denominator():
    # generator check: sum_alpha Lam_i Gam_a Lam_j Gam_b = sum w exp(-t D) ~ 1 / D
    eo, ev, t, w = make_lt(4, 7, 12, seed=3)
    Lam, Gam = X.lt_factors(eo, ev, t, w)
    for i, a, j, b in ((0, 0, 0, 0), (3, 6, 1, 2), (2, 4, 3, 5)):
        D = ev[a] + ev[b] - eo[i] - eo[j]
        s = float(np.sum(Lam[:, i] * Gam[:, a] * Lam[:, j] * Gam[:, b]))
        assert abs(s * D - 1.0) < 1e-3


def test_exchange_planted_mistakes_are_caught():
    Xo, Xv, Z, A, lam, Lam, Gam = _tiny(8, 3, 4, 5, 3, 2)
    G = O.thc_tensor(Xo, Xv, Z)
    Gt = O.cpd_tensor(A, lam)
    good = X.exchange_explicit(G, Gt, Lam, Gam)
    no_swap = -sum(float(np.sum(np.einsum("i,a,j,b->iajb", Lam[al], Gam[al], Lam[al], Gam[al]) * G * Gt))
                   for al in range(Lam.shape[0]))          # Coulomb-like pairing, not exchange
    assert abs(no_swap - good) > 1e-6 * abs(good)
    A1, A2, A3, A4 = A
    e = 0.0
    for al in range(Lam.shape[0]):                         # weights on the wrong factors
        XoL, XvG = Gam[al][:1].sum() * Xo, Lam[al][:1].sum() * Xv
        U1, U3, U2, U4 = XoL.T @ A1, XoL.T @ A3, XvG.T @ A2, XvG.T @ A4
        e -= float(np.sum(lam * (U1 * U4) * (Z @ (U3 * U2))))
    assert abs(e - good) > 1e-6 * abs(good)
    e1, e2, er = X.exchange_robust(Xo, Xv, Z, A, lam, Lam, Gam)
    assert abs((e1 - e2) - er) > 1e-9 * abs(er)            # robust = 2 single - double
