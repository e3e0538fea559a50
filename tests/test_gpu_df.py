"""DF-driven CP-ALS (thc_cpd_df_als; Sec. 2.1, Eq. df_loss) on the GPU, with FP64-pipe and
emulated tensor-core GEMMs, against the FP64 oracle (oracle/df_cpd.py, pinned against the
explicit DF tensor and against the THC-driven oracle on a DF block that is exactly THC).
Fits within 1e-10 and 1000 sampled CPD entries within 1e-10 of max|Gt| along whole
trajectories, as for the THC-driven path."""
import numpy as np
import pytest

from oracle import df_cpd as D
from tests._util import sample_cpd_entries, sample_idx
from thc_inputs import make_df, make_factors

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


def _check(api, o, v, naux, R, sweeps, emulated, seed, tol=0.0):
    _, _, B = make_df(o, v, max(1, (o + v) * 2), naux, seed=seed)
    A0 = make_factors((o, v, o, v), R, seed)
    A = [_dev(a) for a in A0]
    lam = torch.ones(R, dtype=torch.float64, device="cuda")
    out = api.thc_cpd_df_als(_dev(B), A, lam, sweeps, tol, emulated=emulated, history=True)
    ref = D.df_als(B, A0, sweeps, tol)
    assert out["sweeps"] == ref["sweeps"]
    assert np.max(np.abs(np.array(out["fits"]) - np.array(ref["fits"]))) <= 1e-10
    idx = sample_idx((o, v, o, v), 1000, seed)
    got = sample_cpd_entries([a.cpu().numpy() for a in A], lam.cpu().numpy(), idx)
    want = sample_cpd_entries(ref["A"], ref["lam"], idx)
    scale = np.max(np.abs(want))
    assert np.max(np.abs(got - want)) <= 1e-10 * scale
    return out


@pytest.mark.parametrize("emulated", [False, True])
@pytest.mark.parametrize("shape,sweeps", [((1, 1, 1, 1), 3), ((2, 3, 4, 3), 6), ((5, 15, 60, 80), 10),
                                          ((7, 33, 97, 131), 5), ((20, 100, 480, 720), 3)])
def test_df_trajectory_matches_oracle(api, shape, sweeps, emulated):
    o, v, naux, R = shape
    _check(api, o, v, naux, R, sweeps, emulated, seed=o + R)


def test_df_tolerance_stop(api):
    # the oracle stops this run after 39 sweeps (|fit change| < 1e-4)
    out = _check(api, 5, 15, 60, 20, 60, False, seed=11, tol=1e-4)
    assert 2 <= out["sweeps"] < 60


def test_df_pinv_fallback(api):
    # two identical columns in every start factor: each normal matrix is singular
    o, v, naux, R = 4, 9, 30, 12
    _, _, B = make_df(o, v, 20, naux, seed=6)
    A0 = [a.copy() for a in make_factors((o, v, o, v), R, 6)]
    for a in A0:
        a[:, R - 1] = a[:, R - 2]
    A = [_dev(a) for a in A0]
    lam = torch.ones(R, dtype=torch.float64, device="cuda")
    out = api.thc_cpd_df_als(_dev(B), A, lam, 1, history=True)
    ref = D.df_als(B, tuple(A0), 1)
    assert ref["pinv"][0] and (out["flags"] & 1)
    assert abs(out["losses"][0] - ref["losses"][0]) <= 1e-9 * ref["normG2"]


def test_df_rejects_split_precision(api):
    from paper_2502_17683_gb300._lib import Opts, PTR4, ThcCpdError, check, load
    import ctypes
    _, _, B = make_df(2, 3, 4, 5, seed=0)
    A = [_dev(a) for a in make_factors((2, 3, 2, 3), 4, 0)]
    lam = torch.ones(4, dtype=torch.float64, device="cuda")
    opts = Opts()
    opts.precision = 1
    Bd = _dev(B)
    with pytest.raises(ThcCpdError):
        check(load().thc_cpd_df_als(2, 3, 5, 4, Bd.data_ptr(), PTR4(*[a.data_ptr() for a in A]),
                                    lam.data_ptr(), 1, 0.0, None, None, ctypes.byref(opts)))
