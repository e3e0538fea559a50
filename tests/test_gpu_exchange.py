"""The CPD+THC exchange energy (thc_cpd_exchange; Sec. 2.2, Eq. cpd_single_k, the
double-CPD term, Eq. rob_K) on the GPU, with FP64-pipe and emulated tensor-core products,
against the FP64 oracle (oracle/exchange.py, pinned against the explicit tensors)."""
import numpy as np
import pytest

from oracle import exchange as X
from oracle import thc_cpd as O
from tests._util import to_dev
from thc_inputs import make_lt, make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2502_17683_gb300 import api as a
    return a


def _case(o, v, Rt, R, na, seed):
    p = make_problem(o, v, Rt, R, seed=seed)
    rng = np.random.default_rng(seed)
    lam = rng.uniform(0.5, 2.0, R)
    eo, ev, t, w = make_lt(o, v, na, seed)
    Lam, Gam = X.lt_factors(eo, ev, t, w)
    return p, lam, Lam, Gam


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("emulated", [False, True])
@pytest.mark.parametrize("shape", [(2, 3, 5, 4, 2), (5, 15, 60, 80, 6), (7, 33, 97, 131, 5),
                                   (20, 100, 480, 720, 12)])
def test_exchange_matches_oracle(api, shape, emulated):
    o, v, Rt, R, na = shape
    p, lam, Lam, Gam = _case(o, v, Rt, R, na, seed=o + R)
    Z = p.Z + 0.2 * np.triu(p.Z, 1)  # non-symmetric core: Z and Z^T must not be mixed up
    d = to_dev(p, torch)
    e1, e2, er = api.thc_cpd_exchange(d["Xo"], d["Xv"], _dev(Z), d["A"], _dev(lam), _dev(Lam),
                                      _dev(Gam), emulated=emulated)
    r1, r2, rr = X.exchange_robust(p.Xo, p.Xv, Z, p.A, lam, Lam, Gam)
    # each energy is a sum of terms of either sign: compare against the size of the terms
    s1 = abs(X.exchange_single(np.abs(p.Xo), np.abs(p.Xv), np.abs(Z), [np.abs(a) for a in p.A], lam, Lam, Gam))
    s2 = abs(X.exchange_double([np.abs(a) for a in p.A], lam, Lam, Gam))
    assert abs(e1 - r1) <= 1e-12 * s1
    assert abs(e2 - r2) <= 1e-12 * s2
    assert abs(er - rr) <= 1e-12 * (2 * s1 + s2)


def test_exchange_of_an_als_cpd_is_robust_to_first_order(api):
    # the consumer on a CPD the library fitted: the robust energy differs from the THC
    # exchange only at second order in the CPD error (the identity of the oracle pins),
    # checked on the explicit tensors at o=3, v=6
    from oracle import exchange as XX
    o, v, Rt, R, na = 3, 6, 12, 14, 4
    p = make_problem(o, v, Rt, R, seed=5)
    d = to_dev(p, torch)
    lam = torch.ones(R, dtype=torch.float64, device="cuda")
    api.thc_cpd_als(d["Xo"], d["Xv"], d["Z"], d["A"], lam, 200, 0.0)
    A = [a.cpu().numpy() for a in d["A"]]
    lh = lam.cpu().numpy()
    eo, ev, t, w = make_lt(o, v, na, 5)
    Lam, Gam = XX.lt_factors(eo, ev, t, w)
    e1, e2, er = api.thc_cpd_exchange(d["Xo"], d["Xv"], d["Z"], d["A"], lam, _dev(Lam), _dev(Gam))
    e_thc, x1, x2, xr = XX.exchange_energies_explicit(p.Xo, p.Xv, p.Z, A, lh, Lam, Gam)
    G = O.thc_tensor(p.Xo, p.Xv, p.Z)
    D = G - O.cpd_tensor(A, lh)
    assert abs(er - xr) <= 1e-11 * abs(e_thc)
    assert abs((er - e_thc) + XX.exchange_explicit(D, D, Lam, Gam)) <= 1e-11 * abs(e_thc)
    assert abs(er - e_thc) < abs(e1 - e_thc)


@pytest.mark.parametrize("emulated", [False, True])
def test_exchange_at_full_size(api, emulated):
    # (50, 250, 1200, 1800), the decomposition's bench size, two of the 12 quadrature points
    p, lam, Lam, Gam = _case(50, 250, 1200, 1800, 12, seed=7)
    Lam, Gam = Lam[[0, 11]], Gam[[0, 11]]
    d = to_dev(p, torch)
    e1, e2, er = api.thc_cpd_exchange(d["Xo"], d["Xv"], d["Z"], d["A"], _dev(lam), _dev(Lam), _dev(Gam),
                                      emulated=emulated)
    r1, r2, rr = X.exchange_robust(p.Xo, p.Xv, p.Z, p.A, lam, Lam, Gam)
    s1 = abs(X.exchange_single(np.abs(p.Xo), np.abs(p.Xv), np.abs(p.Z), [np.abs(a) for a in p.A], lam, Lam, Gam))
    s2 = abs(X.exchange_double([np.abs(a) for a in p.A], lam, Lam, Gam))
    assert abs(e1 - r1) <= 1e-12 * s1
    assert abs(e2 - r2) <= 1e-12 * s2
    assert abs(er - rr) <= 1e-12 * (2 * s1 + s2)
