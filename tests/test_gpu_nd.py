"""Order-d THC-driven CP-ALS on the GPU (thc_cpd_nd_mttkrp, thc_cpd_nd_als; Conclusions)
with FP64-pipe and emulated tensor-core products, against the FP64 oracle (oracle/nd.py,
pinned against explicit tensors and, at d = 4, against the order-4 oracle). Tolerances as
for the order-4 path: MTTKRP 1e-12 of its largest entry, fits 1e-10, 1000 sampled CPD
entries 1e-10 of the largest."""
import numpy as np
import pytest

from oracle import nd as N
from tests._util import sample_idx
from thc_inputs import make_nd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2502_17683_gb300 import api as a
    return a


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _nonsym(Z, seed):
    rng = np.random.default_rng(seed)
    return Z + 0.3 * rng.standard_normal(Z.shape) * np.max(np.abs(Z))


def _sample(A, lam, idx):
    out = np.array(lam, dtype=np.float64)[None, :].repeat(len(idx[0]), 0)
    for a, i in zip(A, idx):
        out = out * a[i]
    return out.sum(axis=1)


@pytest.mark.parametrize("emulated", [False, True])
@pytest.mark.parametrize("dims,dL,Rt,R", [((1, 1), 1, 1, 1), ((3, 5, 4), 1, 9, 7), ((3, 5, 4), 2, 9, 7),
                                          ((5, 15, 5, 15), 2, 60, 80), ((4, 9, 6, 9, 4), 3, 50, 70),
                                          ((7, 33, 7, 33, 7, 33), 3, 131, 97)])
def test_nd_mttkrp_matches_oracle(api, dims, dL, Rt, R, emulated):
    X, Z, A = make_nd(dims, Rt, R, seed=len(dims) + Rt)
    Z = _nonsym(Z, Rt)
    Xd, Ad, Zd = [_dev(x) for x in X], [_dev(a) for a in A], _dev(Z)
    for k in range(len(dims)):
        M = api.thc_cpd_nd_mttkrp(Xd, Zd, Ad, dL, k, emulated=emulated).cpu().numpy()
        ref = N.nd_mttkrp(X, Z, dL, A, k)
        assert np.max(np.abs(M - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("emulated", [False, True])
@pytest.mark.parametrize("dims,dL,Rt,R,sweeps", [((3, 5, 4), 1, 9, 7, 8), ((5, 15, 5, 15), 2, 60, 80, 10),
                                                 ((4, 9, 6, 9, 4), 2, 50, 70, 6),
                                                 ((20, 100, 20, 100, 20, 100), 3, 480, 720, 2)])
def test_nd_trajectory_matches_oracle(api, dims, dL, Rt, R, sweeps, emulated):
    X, Z, A0 = make_nd(dims, Rt, R, seed=len(dims) + R)
    Xd, Zd = [_dev(x) for x in X], _dev(Z)
    A = [_dev(a) for a in A0]
    lam = torch.ones(R, dtype=torch.float64, device="cuda")
    out = api.thc_cpd_nd_als(Xd, Zd, A, lam, dL, sweeps, emulated=emulated, history=True)
    ref = N.nd_als(X, Z, dL, A0, sweeps)
    assert out["sweeps"] == ref["sweeps"]
    assert np.max(np.abs(np.array(out["fits"]) - np.array(ref["fits"]))) <= 1e-10
    idx = sample_idx(dims, 1000, R)
    got = _sample([a.cpu().numpy() for a in A], lam.cpu().numpy(), idx)
    want = _sample(ref["A"], ref["lam"], idx)
    assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))


def test_nd_planted_order6_recovery(api):
    dims, r = (3, 4, 3, 4, 3, 4), 4
    rng = np.random.default_rng(8)
    As = [rng.standard_normal((n, r)) for n in dims]
    A0 = [a * (1.0 + 0.1 * rng.standard_normal(a.shape)) for a in As]
    A = [_dev(a) for a in A0]
    lam = torch.ones(r, dtype=torch.float64, device="cuda")
    out = api.thc_cpd_nd_als([_dev(a) for a in As], _dev(np.eye(r)), A, lam, 3, 200)
    assert out["fit"] > 1.0 - 1e-8


def test_nd_rejects_bad_arguments(api):
    from paper_2502_17683_gb300._lib import ThcCpdError
    X, Z, A = make_nd((3, 4, 5), 6, 2, seed=0)
    Xd, Zd, Ad = [_dev(x) for x in X], _dev(Z), [_dev(a) for a in A]
    with pytest.raises(ThcCpdError):
        api.thc_cpd_nd_mttkrp(Xd, Zd, Ad, 3, 0)  # dL = d
    with pytest.raises(ThcCpdError):
        api.thc_cpd_nd_mttkrp(Xd, Zd, Ad, 0, 0)  # dL = 0
    with pytest.raises(ThcCpdError):
        api.thc_cpd_nd_mttkrp(Xd, Zd, Ad, 1, 3)  # mode out of range
