"""The THC core least-squares fit (thc_cpd_core_fit; Sec. 3, Computational Details) on the
GPU, with FP64-pipe and emulated tensor-core products, against the FP64 oracle
(oracle/corefit.py, pinned against lstsq on the vectorised problem).

Z is compared in the metric of S (Zs = diag(d) Z diag(d), d_P = sqrt(S_PP)): the grid
weights make the entries of Z span about 8 decades, and the normal equations fix each entry
only to about eps * cond(S / d d^T) of its own scale, so a comparison against max|Z| would
be loose for the small entries and one against each entry would ask for more than FP64
gives. Tolerance: 1e-11 of max|Zs| (the oracle's two solves and a one-solve F^T F form agree
to 1e-14 on these inputs; cond(S / d d^T) <= 2.2e2)."""
import numpy as np
import pytest

from oracle import corefit as C
from thc_inputs import make_df

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


def _scaled_err(Xo, Xv, Zg, Zr):
    d = np.sqrt(np.diag((Xo.T @ Xo) * (Xv.T @ Xv)))
    sc = lambda M: d[:, None] * M * d[None, :]
    return float(np.max(np.abs(sc(Zg) - sc(Zr))) / np.max(np.abs(sc(Zr))))


@pytest.mark.parametrize("emulated", [False, True])
@pytest.mark.parametrize("shape", [(1, 1, 1, 1), (3, 7, 10, 11), (5, 15, 60, 70), (7, 33, 131, 97),
                                   (20, 100, 480, 400)])
def test_core_fit_matches_oracle(api, shape, emulated):
    o, v, Rt, naux = shape
    Xo, Xv, B = make_df(o, v, Rt, naux, seed=o + Rt)
    Zg, loss, pinv = api.thc_cpd_core_fit(_dev(Xo), _dev(Xv), _dev(B), loss=True, emulated=emulated)
    Zg = Zg.cpu().numpy()
    Zr = C.core_fit(Xo, Xv, B)
    assert not pinv
    assert _scaled_err(Xo, Xv, Zg, Zr) <= 1e-11
    assert np.array_equal(Zg, Zg.T)  # F^T F: symmetric by construction
    Dm = B.reshape(naux, -1)
    g2 = float(np.sum((Dm @ Dm.T) ** 2))
    assert abs(loss - C.core_loss(Xo, Xv, B, Zr)) <= 1e-12 * g2


@pytest.mark.parametrize("emulated", [False, True])
def test_core_fit_at_full_size_recovers_the_generating_core(api, emulated):
    # (o, v, R_thc, naux) = (50, 250, 1200, 1200) with a noise-free DF tensor: the core that
    # generated it is the exact minimiser (loss 0 up to rounding)
    o, v, Rt, naux = 50, 250, 1200, 1200
    Xo, Xv, B = make_df(o, v, Rt, naux, seed=3, noise=0.0)
    rng = np.random.default_rng([3, 0xDF])
    Cg = rng.standard_normal((naux, Rt)) / np.sqrt(Rt)
    Zg, loss, pinv = api.thc_cpd_core_fit(_dev(Xo), _dev(Xv), _dev(B), loss=True, emulated=emulated)
    Zg = Zg.cpu().numpy()
    assert not pinv
    assert _scaled_err(Xo, Xv, Zg, Cg.T @ Cg) <= 1e-10
    Dm = B.reshape(naux, -1)
    g2 = float(np.sum((Dm @ Dm.T) ** 2))
    assert abs(loss) <= 1e-11 * g2


def test_core_fit_at_full_size_matches_oracle(api):
    o, v, Rt, naux = 50, 250, 1200, 1200
    Xo, Xv, B = make_df(o, v, Rt, naux, seed=1)
    Zr = C.core_fit(Xo, Xv, B)
    for emulated in (False, True):
        Zg, _, _ = api.thc_cpd_core_fit(_dev(Xo), _dev(Xv), _dev(B), emulated=emulated)
        assert _scaled_err(Xo, Xv, Zg.cpu().numpy(), Zr) <= 1e-11


def test_core_fit_rejects_bad_shapes(api):
    from paper_2502_17683_gb300._lib import ThcCpdError
    Xo, Xv, B = make_df(2, 3, 4, 5, seed=0)
    with pytest.raises(ThcCpdError):
        api.thc_cpd_core_fit(_dev(Xo), _dev(Xv), _dev(B[:, :, :2]))
    Xo, Xv, B = make_df(2, 3, 2049, 1, seed=0)
    with pytest.raises(ThcCpdError):
        api.thc_cpd_core_fit(_dev(Xo), _dev(Xv), _dev(B))
