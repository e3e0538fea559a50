"""Batched ALS of independent problems of uneven shapes (one CUDA graph per sweep for all
problems) against the single-problem driver and the FP64 oracle."""
import numpy as np
import pytest

from oracle import thc_cpd as O
from tests._util import to_dev
from thc_inputs import batched_shapes, make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2502_17683_gb300 import api as a
    return a


def _problems(shapes, seed0):
    out = []
    for i, (o, v, Rt, R) in enumerate(shapes):
        p = make_problem(o, v, Rt, R, seed=seed0 + i)
        d = to_dev(p, torch)
        d["lam"] = torch.ones(R, dtype=torch.float64, device="cuda")
        d["host"] = p
        out.append(d)
    return out


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_batched_equals_single_problem_runs(api, prec):
    shapes = batched_shapes(6, seed=3, o_lo=2, o_hi=9)
    assert len(set(shapes)) > 1  # uneven
    batch = _problems(shapes, 100)
    solo = _problems(shapes, 100)
    res = api.thc_cpd_als_batched(batch, 8, 0.0, precision=prec)
    for b, s_, r in zip(batch, solo, res):
        # the batched driver factorises with the blocked LDL^T; so does this reference run
        out = api.thc_cpd_als(s_["Xo"], s_["Xv"], s_["Z"], s_["A"], s_["lam"], 8, 0.0, precision=prec,
                              ldl="blocked")
        assert r["sweeps"] == out["sweeps"] == 8
        assert r["fit"] == out["fit"]  # same kernels in the same order: same bits
        for a, c in zip(b["A"], s_["A"]):
            assert torch.equal(a, c)


def test_batched_fp64_matches_oracle_and_stops_per_problem(api):
    shapes = [(3, 15, 48, 64), (5, 25, 96, 112), (2, 10, 48, 48)]
    batch = _problems(shapes, 7)
    res = api.thc_cpd_als_batched(batch, 200, 1e-5, precision="fp64")
    for d, r in zip(batch, res):
        p = d["host"]
        ref = O.als(p.Xo, p.Xv, p.Z, p.A, 200, tol=1e-5)
        assert r["sweeps"] == ref["sweeps"]
        nG2 = ref["normG2"]
        assert abs(r["loss"] - ref["losses"][-1]) <= 1e-10 * nG2
        # fit = 1 - sqrt(loss / ||G||^2): at an exact fit (loss at the rounding floor of the
        # factor form, ~eps ||G||^2) the square root turns a rounding-level loss into
        # ~sqrt(eps) of fit, so the fits are compared only above that floor
        if ref["losses"][-1] > 1e-12 * nG2:
            assert abs(r["fit"] - ref["fits"][-1]) <= 1e-10
    assert len({r["sweeps"] for r in res}) >= 1


def test_batched_autotune_keeps_results(api):
    shapes = batched_shapes(4, seed=5, o_lo=3, o_hi=8)
    batch = _problems(shapes, 300)
    ref = _problems(shapes, 300)
    res = api.thc_cpd_als_batched(batch, 5, 0.0, precision="bf16x3", autotune=True)
    res0 = api.thc_cpd_als_batched(ref, 5, 0.0, precision="bf16x3")
    for a, b in zip(res, res0):
        assert abs(a["fit"] - b["fit"]) <= 1e-6


def test_dataflow_factorisation_does_not_depend_on_the_grid(api):
    # Asked for the dataflow LDL^T, the batched driver runs it on at most 32 CTAs per problem
    # (problems share the GPU), a single call on one CTA per SM. Every tile gets its updates
    # in a fixed order whatever the schedule, so both give the same bits.
    shapes = [(8, 40, 192, 288), (9, 45, 216, 324)]  # 18 and 21 tile rows: thousands of tasks
    batch = _problems(shapes, 500)
    solo = _problems(shapes, 500)
    res = api.thc_cpd_als_batched(batch, 4, 0.0, precision="fp64", ldl="dataflow")
    for b, s_, r in zip(batch, solo, res):
        out = api.thc_cpd_als(s_["Xo"], s_["Xv"], s_["Z"], s_["A"], s_["lam"], 4, 0.0,
                              precision="fp64", ldl="dataflow")
        assert r["sweeps"] == out["sweeps"] == 4
        assert r["fit"] == out["fit"]
        for a, c in zip(b["A"], s_["A"]):
            assert torch.equal(a, c)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_batched_emulated_factorisation_equals_single_runs(api, prec):
    # From R_cp = 1024 the batched driver (ldl auto) factorises with the emulated two-level
    # LDL^T, its panels on at most 32 CTAs next to the other problems; a single call runs the
    # same panels on one CTA per SM. The panel kernel's result does not depend on its grid
    # and the emulated products are deterministic, so both give the same bits, and the
    # emulated problems sit next to a small problem on the blocked path.
    shapes = [(29, 145, 704, 1056), (4, 20, 96, 144)]
    batch = _problems(shapes, 600)
    solo = _problems(shapes, 600)
    res = api.thc_cpd_als_batched(batch, 3, 0.0, precision=prec)
    for (o, v, Rt, R), b, s_, r in zip(shapes, batch, solo, res):
        out = api.thc_cpd_als(s_["Xo"], s_["Xv"], s_["Z"], s_["A"], s_["lam"], 3, 0.0, precision=prec,
                              ldl="emulated" if R >= 1024 else "blocked")
        assert r["sweeps"] == out["sweeps"] == 3
        assert r["fit"] == out["fit"]
        for a, c in zip(b["A"], s_["A"]):
            assert torch.equal(a, c)
    # and the FP64 run follows the oracle
    if prec == "fp64":
        p = batch[0]["host"]
        ref = O.als(p.Xo, p.Xv, p.Z, p.A, 3)
        assert abs(res[0]["fit"] - ref["fits"][-1]) <= 1e-10
