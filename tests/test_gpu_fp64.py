"""FP64 GPU path vs the FP64 CPU oracle, through the C ABI.

Tolerances (FP64 path): MTTKRP and ||G||^2 elementwise within 1e-12 of the largest
entry; loss within 1e-12 * (||G||^2 + ||Gt||^2), the size of the terms whose difference
it is; fit and sampled CPD entries within 1e-10 relative."""
import numpy as np
import pytest

from oracle import thc_cpd as O
from tests._util import rel, sample_cpd_entries, sample_idx, to_dev
from thc_inputs import make_planted, make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [
    (1, 1, 1, 1),
    (2, 3, 5, 4),
    (5, 15, 60, 80),      # the small paper-shaped workload
    (7, 33, 97, 131),     # ragged: no dimension a multiple of a tile
    (20, 100, 480, 720),  # the bench workload
]


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2502_17683_gb300 import api as a
    return a


@pytest.mark.parametrize("shape", SHAPES)
def test_thc_norm2(api, shape):
    o, v, Rt, R = shape
    p = make_problem(o, v, Rt, R, seed=1)
    d = to_dev(p, torch)
    got = api.thc_cpd_thc_norm2(d["Xo"], d["Xv"], d["Z"])
    ref = O.thc_norm2(p.Xo, p.Xv, p.Z)
    assert abs(got - ref) <= 1e-12 * ref


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_mttkrp(api, shape, mode):
    o, v, Rt, R = shape
    p = make_problem(o, v, Rt, R, seed=2)
    Z = p.Z + 0.3 * np.triu(p.Z, 1)  # non-symmetric core: catches a Z / Z^T slip
    d = to_dev(p, torch)
    Zd = torch.from_numpy(np.ascontiguousarray(Z)).cuda()
    M = api.thc_cpd_mttkrp(d["Xo"], d["Xv"], Zd, d["A"], mode)
    ref = O.mttkrp(p.Xo, p.Xv, Z, p.A, mode)
    assert rel(M.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("shape", SHAPES)
def test_loss(api, shape):
    o, v, Rt, R = shape
    p = make_problem(o, v, Rt, R, seed=3)
    d = to_dev(p, torch)
    lam = np.random.default_rng(3).uniform(0.5, 1.5, R)
    loss, fit = api.thc_cpd_loss(d["Xo"], d["Xv"], d["Z"], d["A"], torch.from_numpy(lam).cuda())
    nG2 = O.thc_norm2(p.Xo, p.Xv, p.Z)
    ref = O.loss_factor_form(p.Xo, p.Xv, p.Z, p.A, lam, nG2)
    assert abs(loss - ref) <= 1e-12 * (nG2 + O.cpd_norm2(p.A, lam))
    assert abs(fit - O.fit_from_loss(ref, nG2)) <= 1e-10 * max(1.0, abs(fit))


@pytest.mark.parametrize("shape", SHAPES)
def test_one_sweep_identical_inputs(api, shape):
    o, v, Rt, R = shape
    p = make_problem(o, v, Rt, R, seed=4)
    d = to_dev(p, torch)
    lam = torch.ones(R, dtype=torch.float64, device="cuda")
    out = api.thc_cpd_als_sweep(d["Xo"], d["Xv"], d["Z"], d["A"], lam)
    A_ref, lam_ref, loss_ref, fit_ref, flags = O.als_sweep(p.Xo, p.Xv, p.Z, p.A)
    nG2 = O.thc_norm2(p.Xo, p.Xv, p.Z)
    assert out["flags"] & 1 == int(any(flags))
    assert abs(out["loss"] - loss_ref) <= 1e-11 * nG2
    assert abs(out["fit"] - fit_ref) <= 1e-10
    idx = sample_idx((o, v, o, v), 500, 0)
    got = sample_cpd_entries([a.cpu().numpy() for a in d["A"]], lam.cpu().numpy(), idx)
    ref = sample_cpd_entries(A_ref, lam_ref, idx)
    assert rel(got, ref) <= 1e-9


@pytest.mark.parametrize("ldl", ["dataflow", "blocked", "emulated"])
@pytest.mark.parametrize("name,shape,sweeps", [("c1", (5, 15, 60, 80), 25),
                                               ("c2", (20, 100, 480, 720), 50)])
def test_trajectory(api, name, shape, sweeps, ldl):
    o, v, Rt, R = shape
    p = make_problem(o, v, Rt, R, seed=0, decay=Rt / 5)
    d = to_dev(p, torch)
    lam = torch.ones(R, dtype=torch.float64, device="cuda")
    out = api.thc_cpd_als(d["Xo"], d["Xv"], d["Z"], d["A"], lam, sweeps, 0.0, history=True,
                          ldl=ldl)
    ref = O.als(p.Xo, p.Xv, p.Z, p.A, sweeps)
    assert out["sweeps"] == sweeps
    fits = np.array(out["fits"])
    assert np.max(np.abs(fits - np.array(ref["fits"]))) <= 1e-10
    idx = sample_idx((o, v, o, v), 1000, 1)
    got = sample_cpd_entries([a.cpu().numpy() for a in d["A"]], lam.cpu().numpy(), idx)
    want = sample_cpd_entries(ref["A"], ref["lam"], idx)
    G = O.thc_tensor(p.Xo, p.Xv, p.Z) if o * v <= 4000 else None
    scale = np.max(np.abs(G)) if G is not None else np.max(np.abs(want))
    assert np.max(np.abs(got - want)) <= 1e-10 * scale


def test_convergence_tolerance_stops_early(api):
    p = make_problem(5, 15, 60, 80, seed=5)
    d = to_dev(p, torch)
    lam = torch.ones(80, dtype=torch.float64, device="cuda")
    out = api.thc_cpd_als(d["Xo"], d["Xv"], d["Z"], d["A"], lam, 500, 1e-4, history=True)
    ref = O.als(p.Xo, p.Xv, p.Z, p.A, 500, tol=1e-4)
    assert out["sweeps"] == ref["sweeps"] < 500


def test_planted_recovery_gpu(api):
    p, planted = make_planted(5, 15, 12, 12, seed=0, independent=True)
    d = to_dev(p, torch)
    lam = torch.ones(12, dtype=torch.float64, device="cuda")
    out = api.thc_cpd_als(d["Xo"], d["Xv"], d["Z"], d["A"], lam, 1000, 0.0)
    # the factor-form loss cancels to ~eps ||G||^2, so its fit floors near sqrt(eps);
    # exact recovery is checked on the explicit tensor built from the returned factors
    assert 1.0 - out["fit"] < 1e-7
    A = [a.cpu().numpy() for a in d["A"]]
    G = O.thc_tensor(p.Xo, p.Xv, p.Z)
    relerr = np.linalg.norm(G - O.cpd_tensor(A, lam.cpu().numpy())) / np.linalg.norm(G)
    assert relerr < 1e-10


@pytest.mark.parametrize("ldl,R", [("dataflow", 6), ("blocked", 6), ("dataflow", 40),
                                   ("emulated", 200)])
def test_pinv_fallback_rollback(api, ldl, R):
    # two identical columns in every start factor make each H singular: the optimistic
    # sweep fails its LDL^T pivot test, is rolled back, and is replayed with the
    # pseudo-inverse (R = 40: the failing pivot sits in the dataflow kernel's third tile;
    # R = 200: in the second 128-column panel of the emulated two-level factorisation)
    p = make_problem(4, 9, 20, R, seed=6)
    A = [a.copy() for a in p.A]
    for a in A:
        a[:, R - 1] = a[:, R - 2]
    d = to_dev(p, torch)
    d["A"] = [torch.from_numpy(a).cuda() for a in A]
    lam = torch.ones(R, dtype=torch.float64, device="cuda")
    out = api.thc_cpd_als_sweep(d["Xo"], d["Xv"], d["Z"], d["A"], lam, ldl=ldl)
    A_ref, lam_ref, loss_ref, fit_ref, flags = O.als_sweep(p.Xo, p.Xv, p.Z, tuple(A))
    assert flags[0] and (out["flags"] & 1) and (out["flags"] & 2)
    nG2 = O.thc_norm2(p.Xo, p.Xv, p.Z)
    assert abs(out["loss"] - loss_ref) <= 1e-9 * nG2


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_pinv_fallback_in_a_fixed_length_run(api, prec):
    # the same singular start point over several sweeps of a fixed-length run: every sweep
    # fails its pivot test, while the next sweep is already queued; the queued sweep is
    # undone, the failed one rolled back and replayed, and the run goes on
    R, sweeps = 6, 5
    p = make_problem(4, 9, 20, R, seed=6)
    A = [a.copy() for a in p.A]
    for a in A:
        a[:, R - 1] = a[:, R - 2]
    d = to_dev(p, torch)
    d["A"] = [torch.from_numpy(a).cuda() for a in A]
    lam = torch.ones(R, dtype=torch.float64, device="cuda")
    out = api.thc_cpd_als(d["Xo"], d["Xv"], d["Z"], d["A"], lam, sweeps, 0.0, precision=prec,
                          loss_every=1, history=True)
    ref = O.als(p.Xo, p.Xv, p.Z, tuple(A), sweeps)
    assert out["sweeps"] == sweeps
    assert (out["flags"] & 1) and (out["flags"] & 2)
    nG2 = ref["normG2"]
    tol = 1e-9 if prec == "fp64" else 1e-5
    for got, want in zip(out["losses"], ref["losses"]):
        assert abs(got - want) <= tol * nG2


def test_bad_arguments_raise(api):
    from paper_2502_17683_gb300._lib import ThcCpdError
    p = make_problem(3, 4, 5, 6, seed=7)
    d = to_dev(p, torch)
    with pytest.raises(ThcCpdError):
        api.thc_cpd_mttkrp(d["Xo"], d["Xv"], d["Z"], d["A"], 5)
    with pytest.raises(ThcCpdError):
        api.thc_cpd_mttkrp(d["Xo"], d["Xv"], d["Z"], d["A"][:3], 0)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_graph_replay_is_bit_identical_to_direct_launches(api, prec, monkeypatch):
    # every kernel is deterministic (fixed-order reductions, no atomics on data), so the
    # CUDA-graph replay of a sweep and direct launches give the same bits
    p = make_problem(7, 33, 97, 131, seed=8)
    outs = []
    for no_graph in (False, True):
        if no_graph:
            monkeypatch.setenv("THC_CPD_NO_GRAPH", "1")
        d = to_dev(p, torch)
        lam = torch.ones(131, dtype=torch.float64, device="cuda")
        out = api.thc_cpd_als(d["Xo"], d["Xv"], d["Z"], d["A"], lam, 6, 0.0, precision=prec)
        outs.append((out["fit"], [a.cpu().numpy() for a in d["A"]], lam.cpu().numpy()))
    assert outs[0][0] == outs[1][0]
    for a, b in zip(outs[0][1], outs[1][1]):
        assert np.array_equal(a, b)
    assert np.array_equal(outs[0][2], outs[1][2])


def test_dataflow_and_blocked_ldl_agree_and_reproduce(api):
    # the two factorisations run the same LDL^T in different rounding orders; each is
    # bit-reproducible (tiles get their updates in a fixed order, whatever the schedule)
    p = make_problem(20, 100, 480, 720, seed=9)
    runs = {}
    for ldl in ("dataflow", "dataflow", "blocked"):
        d = to_dev(p, torch)
        lam = torch.ones(720, dtype=torch.float64, device="cuda")
        out = api.thc_cpd_als(d["Xo"], d["Xv"], d["Z"], d["A"], lam, 5, 0.0, ldl=ldl)
        runs.setdefault(ldl, []).append((out["fit"], [a.cpu().numpy() for a in d["A"]]))
    (f0, A0), (f1, A1) = runs["dataflow"]
    assert f0 == f1 and all(np.array_equal(a, b) for a, b in zip(A0, A1))
    fb, Ab = runs["blocked"][0]
    assert abs(f0 - fb) <= 1e-12
    for a, b in zip(A0, Ab):
        assert rel(a, b) <= 1e-8


def test_unknown_ldl_variant_rejected(api):
    from paper_2502_17683_gb300._lib import ThcCpdError
    p = make_problem(3, 4, 5, 6, seed=7)
    d = to_dev(p, torch)
    lam = torch.ones(6, dtype=torch.float64, device="cuda")
    with pytest.raises(ThcCpdError):
        api.thc_cpd_als(d["Xo"], d["Xv"], d["Z"], d["A"], lam, 1, ldl="cholesky")
