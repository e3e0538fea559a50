"""The normal-equation solve of the ALS mode update (thc_cpd_ldl_solve: dataflow LDL^T with
the M rows carried along, backward solve, pseudo-inverse fallback) against the FP64 oracle,
and its bounded waits: a task list that lacks one task must end in THC_CPD_ERR_TIMEOUT after
the configured limit, with the device still usable for a correct solve afterwards."""
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


def _normal_equations(R, n, seed, dims=(7, 30, 7)):
    # H as in an ALS mode update: the Hadamard product of three Gram matrices
    rng = np.random.default_rng(seed)
    H = np.ones((R, R))
    for d in dims:
        a = rng.standard_normal((d, R))
        a /= np.linalg.norm(a, axis=0)
        H *= a.T @ a
    M = rng.standard_normal((n, R))
    return H, M


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("R,n", [(1, 1), (17, 3), (100, 20), (720, 100), (1080, 150)])
def test_ldl_solve_matches_oracle(api, R, n):
    H, M = _normal_equations(R, n, seed=R + n)
    Aref, used_ref = O.solve_normal_equations(M, H)
    assert not used_ref
    A, used = api.thc_cpd_ldl_solve(_dev(H), _dev(M))
    A = A.cpu().numpy()
    assert not used
    # backward error of the FP64 solve, and agreement with the oracle's Cholesky solve
    assert np.linalg.norm(A @ H - M) / np.linalg.norm(M) <= 1e-12
    assert rel(A, Aref) <= 1e-9


def test_ldl_solve_singular_takes_the_pseudo_inverse(api):
    R, n = 64, 10
    H, M = _normal_equations(R, n, seed=5)
    H[:, 7] = H[:, 3]
    H[7, :] = H[3, :]  # a repeated column: singular, the LDL^T meets a zero pivot
    Aref, used_ref = O.solve_normal_equations(M, H)
    assert used_ref
    A, used = api.thc_cpd_ldl_solve(_dev(H), _dev(M))
    assert used
    assert rel(A.cpu().numpy(), Aref) <= 1e-8


def test_missing_task_times_out_and_the_device_stays_usable(api):
    from paper_2502_17683_gb300._lib import ERR_TIMEOUT, ThcCpdError
    R, n = 100, 20
    H, M = _normal_equations(R, n, seed=9)
    sched = np.array(api.thc_cpd_ldl_schedule(R, n), dtype=np.int16)
    # drop U(5, 3, 0): the update U(5, 3, 1) waits for it, so a bounded wait must run out
    drop = [i for i, x in enumerate(sched) if tuple(x) == (1, 5, 3, 0)]
    assert len(drop) == 1
    doctored = np.delete(sched, drop[0], axis=0)
    dH, dM = _dev(H), _dev(M)
    with pytest.raises(ThcCpdError) as ei:
        api.thc_cpd_ldl_solve(dH, dM, tasks=doctored, wait_limit_s=0.005)
    assert ei.value.status == ERR_TIMEOUT
    # the same device, the full list (given explicitly) and the library's own: correct
    Aref, _ = O.solve_normal_equations(M, H)
    for tasks in (sched, None):
        A, used = api.thc_cpd_ldl_solve(dH, dM, tasks=tasks)
        assert not used
        assert rel(A.cpu().numpy(), Aref) <= 1e-9
