"""The allocation-free MTTKRP entry point (thc_cpd_mttkrp_noalloc) against the ordinary
one (thc_cpd_mttkrp), through the C ABI.

Some callers cannot allocate device memory while they run (their own pool allocator owns
the device, or a cudaMalloc that may synchronise the device is not allowed where they
enqueue work). For them the library keeps one fixed scratch array per device; this file
checks that two calls in a row through it give the ordinary entry point's results in every
mode, that a call after the first allocates nothing (the default memory pool's high-water
mark stays at zero and the device's free memory does not move), that it checks its
arguments exactly as the ordinary entry point does, and that a problem too large for the
array is refused with a clear message. It is collected last on purpose: it must pass both
alone in a fresh process and after every other test."""
import ctypes

import numpy as np
import pytest

from tests._util import rel, to_dev
from thc_inputs import make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# driver-API memory pool attribute: high-water mark of the memory in use (bytes)
_CU_MEMPOOL_ATTR_USED_MEM_HIGH = 8


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2502_17683_gb300 import api as a
    return a


class _DefaultPool:
    """The current device's default stream-ordered memory pool, read through the driver
    API (the pool every cudaMallocAsync of the library draws from)."""

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int(0)
        assert self.cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def reset_high(self):
        z = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, _CU_MEMPOOL_ATTR_USED_MEM_HIGH,
                                             ctypes.byref(z)) == 0

    def high(self):
        v = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolGetAttribute(self.pool, _CU_MEMPOOL_ATTR_USED_MEM_HIGH,
                                             ctypes.byref(v)) == 0
        return int(v.value)


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_noalloc_matches_allocating_mttkrp_on_two_calls_in_a_row(api, mode):
    # two consecutive calls with different shapes: the second reuses the scratch left by the
    # first, so a buffer that should have been rewritten would show up here. Modes 0 and 1
    # use Z, modes 2 and 3 Z^T; each mode has its own Hadamard partner.
    for shape, seed in (((20, 100, 480, 720), 21 + mode), ((7, 33, 97, 131), 31 + mode)):
        o, v, Rt, R = shape
        p = make_problem(o, v, Rt, R, seed=seed)
        d = to_dev(p, torch)
        ref = api.thc_cpd_mttkrp(d["Xo"], d["Xv"], d["Z"], d["A"], mode)
        M = torch.full((p.dims[mode], R), np.nan, dtype=torch.float64, device="cuda")
        api.thc_cpd_mttkrp_noalloc(d["Xo"], d["Xv"], d["Z"], d["A"], mode, M)
        torch.cuda.synchronize()
        assert rel(M.cpu().numpy(), ref.cpu().numpy()) <= 1e-12


def test_noalloc_call_after_the_first_allocates_nothing(api):
    p = make_problem(20, 100, 480, 720, seed=41)
    d = to_dev(p, torch)
    M = torch.empty((p.v, 720), dtype=torch.float64, device="cuda")
    api.thc_cpd_mttkrp_noalloc(d["Xo"], d["Xv"], d["Z"], d["A"], 1, M)  # set-up call
    torch.cuda.synchronize()
    pool = _DefaultPool()
    # control: the ordinary entry point draws its workspace from the pool
    pool.reset_high()
    api.thc_cpd_mttkrp(d["Xo"], d["Xv"], d["Z"], d["A"], 1)
    torch.cuda.synchronize()
    assert pool.high() > 0
    # the allocation-free call: nothing from the pool, no change in free device memory
    pool.reset_high()
    free0 = torch.cuda.mem_get_info()[0]
    api.thc_cpd_mttkrp_noalloc(d["Xo"], d["Xv"], d["Z"], d["A"], 1, M)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert pool.high() == 0
    assert free1 == free0
    ref = api.thc_cpd_mttkrp(d["Xo"], d["Xv"], d["Z"], d["A"], 1)
    assert rel(M.cpu().numpy(), ref.cpu().numpy()) <= 1e-12


def test_noalloc_checks_arguments_like_the_allocating_entry_point(api):
    from paper_2502_17683_gb300._lib import PTR4, ThcCpdError, check, load
    lib = load()
    t = lambda *s: torch.zeros(*s, dtype=torch.float64, device="cuda")
    o, v, Rt, R = 2, 3, 4, 5
    X = [t(o, Rt), t(v, Rt), t(Rt, Rt)]
    A = [t(o, R), t(v, R), t(o, R), t(v, R)]
    M = t(o, R)
    ptr = lambda x: ctypes.c_void_p(x.data_ptr())
    good = dict(o=o, v=v, Rt=Rt, R=R, X=[ptr(x) for x in X], A=PTR4(*[a.data_ptr() for a in A]),
                mode=0, M=ptr(M))
    bad_cases = [
        dict(good, Rt=46341, R=1),           # R_thc^2 beyond 2^31
        dict(good, o=0),                     # non-positive dimension
        dict(good, A=PTR4(A[0].data_ptr(), None, A[2].data_ptr(), A[3].data_ptr())),
        dict(good, mode=4),
        dict(good, M=ctypes.c_void_p(None)),
    ]
    for case in bad_cases:
        outs = []
        for fn in (lib.thc_cpd_mttkrp, lib.thc_cpd_mttkrp_noalloc):
            st = fn(case["o"], case["v"], case["Rt"], case["R"], *case["X"], case["A"],
                    case["mode"], case["M"], None)
            outs.append((st, lib.thc_cpd_last_error().decode()))
        assert outs[0][0] != 0 and outs[0] == outs[1], outs
    with pytest.raises(ThcCpdError):
        check(outs[0][0])


def test_noalloc_rejects_problems_beyond_its_scratch(api):
    from paper_2502_17683_gb300._lib import ERR_SHAPE, ThcCpdError
    o, v, Rt, R = 2, 3, 2048, 1800  # 4 * Rt * R doubles > 32 MiB
    t = lambda *s: torch.zeros(*s, dtype=torch.float64, device="cuda")
    A = [t(o, R), t(v, R), t(o, R), t(v, R)]
    with pytest.raises(ThcCpdError) as ei:
        api.thc_cpd_mttkrp_noalloc(t(o, Rt), t(v, Rt), t(Rt, Rt), A, 0, t(o, R))
    assert ei.value.status == ERR_SHAPE
    assert "scratch" in str(ei.value)
