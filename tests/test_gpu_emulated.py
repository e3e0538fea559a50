"""The FP64-accurate product on the BF16 tensor cores (thc_cpd_emulated_gemm: exact integer
digit slices, exact tensor-core digit products, exact 64-bit recombination, one rounding)
and the normal-equation solve whose trailing updates run on it (THC_CPD_LDL_EMULATED),
against FP64 references.

Bounds. Each row of A and of B keeps its digits down to 2^-55 of its largest entry, so the
truncation error of an entry of C is at most 2 * 2^-55 * K * max_k|A_ik| * max_k|B_jk|; the
recombination rounds once (2^-53 |C_ij|). numpy's own FP64 product, the reference, errs by
up to K * 2^-53 * (|A| |B|^T)_ij. The tests hold the sum of the three (with a factor 2)."""
import numpy as np
import pytest

from oracle import thc_cpd as O
from tests._util import rel

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


def _bound(A, B, C):
    K = A.shape[1]
    u = 2.0 ** -53
    rowmax = np.max(np.abs(A), axis=1)[:, None] * np.max(np.abs(B), axis=1)[None, :]
    return 2.0 * (u * np.abs(C) + 2 * K * 2.0 ** -55 * rowmax + K * u * (np.abs(A) @ np.abs(B).T))


@pytest.mark.parametrize("shape", [(1, 1, 1), (7, 5, 3), (128, 64, 128), (130, 65, 129),
                                   (300, 200, 500), (1922, 1672, 128)])
def test_emulated_gemm_is_fp64_accurate(api, shape):
    M, N, K = shape
    rng = np.random.default_rng(M + 3 * N + 7 * K)
    # rows of very different magnitude and entries spanning six decades inside a row
    A = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-3, 3, (M, 1)) * 10.0 ** rng.uniform(-6, 0, (M, K))
    B = rng.standard_normal((N, K)) * 10.0 ** rng.uniform(-3, 3, (N, 1))
    C = api.thc_cpd_emulated_gemm(_dev(A), _dev(B)).cpu().numpy()
    ref = A @ B.T
    err = np.abs(C - ref)
    assert np.all(err <= _bound(A, B, ref)), float(np.max(err / _bound(A, B, ref)))
    # far beyond any split-float product: within a few FP64 ulps of |A||B|^T
    assert np.max(err / (np.abs(A) @ np.abs(B).T)) < 2.0 ** -44


def test_emulated_gemm_is_exact_on_integers(api):
    # integer entries below 2^20, K = 300: every product and sum is exact in FP64, so the
    # emulated result must equal the exact one bit for bit (a lost digit or carry shows)
    rng = np.random.default_rng(2)
    A = rng.integers(-(1 << 20), 1 << 20, (200, 300)).astype(np.float64)
    B = rng.integers(-(1 << 12), 1 << 12, (150, 300)).astype(np.float64)
    C = api.thc_cpd_emulated_gemm(_dev(A), _dev(B)).cpu().numpy()
    assert np.array_equal(C, A @ B.T)


def test_emulated_gemm_zero_rows_and_powers_of_two(api):
    A = np.zeros((70, 40))
    A[1::3] = 2.0 ** np.arange(-20, 20)[None, :]
    B = np.ones((33, 40))
    B[5] = 0.0
    C = api.thc_cpd_emulated_gemm(_dev(A), _dev(B)).cpu().numpy()
    assert np.array_equal(C, A @ B.T)


def _normal_equations(R, n, seed, dims=(9, 40, 9)):
    rng = np.random.default_rng(seed)
    H = np.ones((R, R))
    for d in dims:
        a = rng.standard_normal((d, R))
        a /= np.linalg.norm(a, axis=0)
        H *= a.T @ a
    return H, rng.standard_normal((n, R))


# the backward solve splits blocks of >= 768 columns when n >= 128: (800, 200) and (1080, 150)
# once, (1800, 250) twice (quarters); (720, 200) stays whole
@pytest.mark.parametrize("R,n", [(129, 3), (300, 50), (300, 200), (720, 100), (720, 200), (800, 200),
                                 (1080, 150), (1800, 250)])
def test_emulated_ldl_solve_matches_oracle(api, R, n):
    H, M = _normal_equations(R, n, seed=R)
    Aref, used_ref = O.solve_normal_equations(M, H)
    assert not used_ref
    A, used = api.thc_cpd_ldl_solve(_dev(H), _dev(M), ldl="emulated")
    A = A.cpu().numpy()
    assert not used
    assert np.linalg.norm(A @ H - M) / np.linalg.norm(M) <= 1e-12
    assert rel(A, Aref) <= 1e-9


def test_emulated_and_dataflow_ldl_agree_in_als(api):
    from tests._util import to_dev
    from thc_inputs import make_problem
    p = make_problem(20, 100, 480, 720, seed=9)
    fits, facs = [], []
    for ldl in ("emulated", "emulated", "dataflow"):
        d = to_dev(p, torch)
        lam = torch.ones(720, dtype=torch.float64, device="cuda")
        out = api.thc_cpd_als(d["Xo"], d["Xv"], d["Z"], d["A"], lam, 5, 0.0, ldl=ldl)
        fits.append(out["fit"])
        facs.append([a.cpu().numpy() for a in d["A"]])
    # bit-reproducible run to run; the same factorisation as the FP64 dataflow kernel up to
    # rounding order
    assert fits[0] == fits[1] and all(np.array_equal(a, b) for a, b in zip(facs[0], facs[1]))
    assert abs(fits[0] - fits[2]) <= 1e-12
    for a, b in zip(facs[0], facs[2]):
        assert rel(a, b) <= 1e-8


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_split_path_fp64_loss_through_emulated_products(api, prec):
    # with the emulated path the split-precision run takes its FP64 loss (projections and
    # the Z product) and the Grams from emulated products: the reported fit must be the
    # exact FP64 fit of the returned factors, as computed by the FP64-pipe loss entry point
    from tests._util import to_dev
    from thc_inputs import make_problem
    p = make_problem(20, 100, 480, 720, seed=12)
    d = to_dev(p, torch)
    lam = torch.ones(720, dtype=torch.float64, device="cuda")
    out = api.thc_cpd_als(d["Xo"], d["Xv"], d["Z"], d["A"], lam, 3, 0.0, precision=prec,
                          ldl="emulated")
    loss, fit = api.thc_cpd_loss(d["Xo"], d["Xv"], d["Z"], d["A"], lam)
    nG2 = O.thc_norm2(p.Xo, p.Xv, p.Z)
    assert abs(out["loss"] - loss) <= 1e-12 * nG2
    assert abs(out["fit"] - fit) <= 1e-12
    # and the run itself matches the oracle's sweeps to the split path's per-sweep bound
    ref = O.als(p.Xo, p.Xv, p.Z, p.A, 3)
    assert abs(out["fit"] - ref["fits"][-1]) <= 1e-5
