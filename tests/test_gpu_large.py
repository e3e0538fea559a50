"""Parity at the large paper-shaped size, o=50 v=250 R_thc=1200 R_cp=1800 (decay scale 240),
through the same entry point and launch configuration as the benchmark (thc_cpd_als, CUDA
graph replay, automatic factorisation choice: the dataflow LDL^T at this R_cp), and with
the blocked factorisation the batched driver uses.

The oracle's full ALS sweep at this size takes seconds on the host cores, so the checks are
one sweep from identical inputs (fit, loss and sampled entries of the reconstructed tensor)
and one full MTTKRP."""
import numpy as np
import pytest

from oracle import thc_cpd as O
from tests._util import rel, sample_cpd_entries, sample_idx, to_dev
from thc_inputs import make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPE = (50, 250, 1200, 1800)


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2502_17683_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def case():
    o, v, Rt, R = SHAPE
    p = make_problem(o, v, Rt, R, seed=0, decay=240.0)
    nG2 = O.thc_norm2(p.Xo, p.Xv, p.Z)
    A_ref, lam_ref, loss_ref, fit_ref, flags = O.als_sweep(p.Xo, p.Xv, p.Z, p.A, normG2=nG2)
    return p, nG2, A_ref, lam_ref, loss_ref, fit_ref


@pytest.mark.parametrize("ldl", ["auto", "blocked", "emulated"])
def test_fp64_sweep_at_full_size(api, case, ldl):
    p, nG2, A_ref, lam_ref, loss_ref, fit_ref = case
    o, v, Rt, R = SHAPE
    d = to_dev(p, torch)
    lam = torch.ones(R, dtype=torch.float64, device="cuda")
    out = api.thc_cpd_als(d["Xo"], d["Xv"], d["Z"], d["A"], lam, 1, 0.0, ldl=ldl)
    assert out["sweeps"] == 1
    assert abs(out["loss"] - loss_ref) <= 1e-11 * nG2
    assert abs(out["fit"] - fit_ref) <= 1e-10
    idx = sample_idx((o, v, o, v), 1000, 3)
    got = sample_cpd_entries([a.cpu().numpy() for a in d["A"]], lam.cpu().numpy(), idx)
    ref = sample_cpd_entries(A_ref, lam_ref, idx)
    assert rel(got, ref) <= 1e-9


def test_bf16x3_sweep_at_full_size(api, case):
    # each mode update is an exact block minimiser, so the split MTTKRP's error moves the
    # fit only at second order: 1e-6 relative, the mixed path's stated parity
    p, nG2, A_ref, lam_ref, loss_ref, fit_ref = case
    R = SHAPE[3]
    d = to_dev(p, torch)
    lam = torch.ones(R, dtype=torch.float64, device="cuda")
    out = api.thc_cpd_als(d["Xo"], d["Xv"], d["Z"], d["A"], lam, 1, 0.0, precision="bf16x3")
    assert abs(out["fit"] - fit_ref) <= 1e-6 * abs(fit_ref)


def test_fp64_mttkrp_at_full_size(api, case):
    p = case[0]
    d = to_dev(p, torch)
    for mode in (1, 2):  # a virtual (v x R_cp) and an occupied mode, both Z orientations
        M = api.thc_cpd_mttkrp(d["Xo"], d["Xv"], d["Z"], d["A"], mode).cpu().numpy()
        ref = O.mttkrp(p.Xo, p.Xv, p.Z, p.A, mode)
        assert np.max(np.abs(M - ref)) <= 1e-12 * np.max(np.abs(ref))
