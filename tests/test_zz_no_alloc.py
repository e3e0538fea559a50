"""The allocation-free MTTKRP entry point (thc_cpd_mttkrp_noalloc) against the ordinary
one (thc_cpd_mttkrp), through the C ABI.

Some callers cannot allocate device memory while they run (their own pool allocator owns
the device, or a cudaMalloc that may synchronise the device is not allowed where they
enqueue work). For them the library keeps one fixed scratch array per device; this file
checks that two calls in a row through it give the ordinary entry point's results, and
that a problem too large for the array is refused with a clear message. It is collected
last on purpose: it must pass both alone in a fresh process and after every other test."""
import numpy as np
import pytest

from tests._util import rel, to_dev
from thc_inputs import make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2502_17683_gb300 import api as a
    return a


def test_noalloc_matches_allocating_mttkrp_on_two_calls_in_a_row(api):
    # two consecutive calls with different shapes and modes: the second reuses the scratch
    # left by the first, so a buffer that should have been rewritten would show up here
    for shape, mode, seed in (((20, 100, 480, 720), 1, 21), ((7, 33, 97, 131), 2, 22)):
        o, v, Rt, R = shape
        p = make_problem(o, v, Rt, R, seed=seed)
        d = to_dev(p, torch)
        ref = api.thc_cpd_mttkrp(d["Xo"], d["Xv"], d["Z"], d["A"], mode)
        M = torch.full((p.dims[mode], R), np.nan, dtype=torch.float64, device="cuda")
        api.thc_cpd_mttkrp_noalloc(d["Xo"], d["Xv"], d["Z"], d["A"], mode, M)
        torch.cuda.synchronize()
        assert rel(M.cpu().numpy(), ref.cpu().numpy()) <= 1e-12


def test_noalloc_rejects_problems_beyond_its_scratch(api):
    from paper_2502_17683_gb300._lib import ERR_SHAPE, ThcCpdError
    o, v, Rt, R = 2, 3, 2048, 1800  # 4 * Rt * R doubles > 32 MiB
    t = lambda *s: torch.zeros(*s, dtype=torch.float64, device="cuda")
    A = [t(o, R), t(v, R), t(o, R), t(v, R)]
    with pytest.raises(ThcCpdError) as ei:
        api.thc_cpd_mttkrp_noalloc(t(o, Rt), t(v, Rt), t(Rt, Rt), A, 0, t(o, R))
    assert ei.value.status == ERR_SHAPE
    assert "scratch" in str(ei.value)
