"""Guard canaries around every buffer the entry points write or read (a stand-in for a memory
checker, which this pool does not run): each tensor is the interior of a larger device
buffer whose guard regions before and after it hold a signalling-NaN bit pattern; after the
call the guards must hold that pattern bit for bit, and read-only inputs must be unchanged.
The shapes are ragged (no dimension a multiple of a tile) and exercise the paths with the
most index arithmetic: the split-precision MTTKRP, the emulated two-level LDL^T with its
dataflow tail, the backward solve split into column blocks with split-K coupling products,
and the emulated product over several K chunks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GUARD = 256  # doubles before and after each tensor (keeps the 2 KB alignment of the interior)
CANARY = np.array([0x7FF4DEADBEEF1234], dtype=np.int64).view(np.float64)[0]


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2502_17683_gb300 import api as a
    return a


class Guarded:
    """A device tensor of the given contents inside a canary-filled buffer."""

    def __init__(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        n = x.size
        host = np.full(GUARD + n + GUARD, CANARY, dtype=np.float64)  # bit-exact payload
        host[GUARD:GUARD + n] = x.ravel()
        self.buf = torch.from_numpy(host).cuda()
        self.t = self.buf[GUARD:GUARD + n].view(x.shape)
        self.orig = x.copy()

    def guards_intact(self):
        b = self.buf.cpu().numpy().view(np.int64)
        c = np.int64(np.array([CANARY]).view(np.int64)[0])
        n = self.orig.size
        return bool(np.all(b[:GUARD] == c) and np.all(b[GUARD + n:] == c))

    def unchanged(self):
        return bool(np.array_equal(self.t.cpu().numpy().view(np.int64), self.orig.view(np.int64)))


def _problem(o, v, Rt, R, seed):
    from thc_inputs import make_problem
    return make_problem(o, v, Rt, R, seed=seed)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_mttkrp_writes_only_its_output(api, prec, mode):
    p = _problem(7, 37, 101, 83, seed=mode)
    ins = [Guarded(x) for x in (p.Xo, p.Xv, p.Z)] + [Guarded(a) for a in p.A]
    n = (7, 37, 7, 37)[mode]
    M = Guarded(np.zeros((n, 83)))
    api.thc_cpd_mttkrp(ins[0].t, ins[1].t, ins[2].t, [g.t for g in ins[3:]], mode, M=M.t, precision=prec)
    torch.cuda.synchronize()
    assert M.guards_intact()
    for g in ins:
        assert g.guards_intact() and g.unchanged()
    assert np.all(np.isfinite(M.t.cpu().numpy()))


@pytest.mark.parametrize("prec,ldl", [("bf16x3", "emulated"), ("fp64", "emulated"), ("fp64", "dataflow")])
def test_als_writes_only_factors_and_lambda(api, prec, ldl):
    # R_cp = 900 >= 768 with v = 150 >= 128: the v modes' backward solve splits into column
    # blocks with emulated coupling products; the emulated LDL^T runs 256-column panels and a
    # dataflow tail
    p = _problem(13, 150, 230, 900, seed=5)
    ins = [Guarded(x) for x in (p.Xo, p.Xv, p.Z)]
    A = [Guarded(a) for a in p.A]
    lam = Guarded(np.ones(900))
    out = api.thc_cpd_als(ins[0].t, ins[1].t, ins[2].t, [g.t for g in A], lam.t, 3, 0.0,
                          precision=prec, ldl=ldl)
    torch.cuda.synchronize()
    assert np.isfinite(out["fit"])
    for g in A + [lam]:
        assert g.guards_intact()
    for g in ins:
        assert g.guards_intact() and g.unchanged()


def test_ldl_solve_writes_only_its_output(api):
    rng = np.random.default_rng(3)
    R, n = 1000, 170
    H = np.ones((R, R))
    for d in (9, 40, 9):
        a = rng.standard_normal((d, R))
        a /= np.linalg.norm(a, axis=0)
        H *= a.T @ a
    H += 1e-3 * np.eye(R)
    Hg, Mg = Guarded(H), Guarded(rng.standard_normal((n, R)))
    Ag = Guarded(np.zeros((n, R)))
    api.thc_cpd_ldl_solve(Hg.t, Mg.t, A=Ag.t, ldl="emulated")
    torch.cuda.synchronize()
    assert Ag.guards_intact()
    for g in (Hg, Mg):
        assert g.guards_intact() and g.unchanged()
    A = Ag.t.cpu().numpy()
    assert np.linalg.norm(A @ H - Mg.orig) / np.linalg.norm(Mg.orig) <= 1e-10


def test_emulated_gemm_writes_only_its_output(api):
    rng = np.random.default_rng(4)
    A = Guarded(rng.standard_normal((301, 389)))
    B = Guarded(rng.standard_normal((203, 389)))
    C = Guarded(np.zeros((301, 203)))
    api.thc_cpd_emulated_gemm(A.t, B.t, C=C.t)
    torch.cuda.synchronize()
    assert C.guards_intact()
    for g in (A, B):
        assert g.guards_intact() and g.unchanged()
    ref = A.orig @ B.orig.T
    assert np.max(np.abs(C.t.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
