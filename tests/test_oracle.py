"""Pins for the FP64 CPU oracle: brute force on tiny inputs, closed forms, invariants,
hand-derived values and planted solutions. None of these re-types the oracle's own
formula; each compares it with something the mathematics fixes independently."""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import thc_cpd as O
from thc_inputs import make_planted, make_problem

HERE = os.path.dirname(os.path.abspath(__file__))


def _rand(shape, rng):
    return rng.standard_normal(shape)


def _tiny(seed=0, o=2, v=3, Rt=3, R=2, sym=False):
    rng = np.random.default_rng(seed)
    Xo, Xv, Z = _rand((o, Rt), rng), _rand((v, Rt), rng), _rand((Rt, Rt), rng)
    if sym:
        Z = Z + Z.T
    A = tuple(_rand((n, R), rng) for n in (o, v, o, v))
    lam = rng.uniform(0.5, 2.0, R)
    return Xo, Xv, Z, A, lam


def _brute_G(Xo, Xv, Z):
    o, Rt = Xo.shape
    v = Xv.shape[0]
    G = np.zeros((o, v, o, v))
    for i, a, j, b in itertools.product(range(o), range(v), range(o), range(v)):
        s = 0.0
        for P in range(Rt):
            for Q in range(Rt):
                s += Xo[i, P] * Xv[a, P] * Z[P, Q] * Xo[j, Q] * Xv[b, Q]
        G[i, a, j, b] = s
    return G


def _brute_Gt(A, lam):
    A1, A2, A3, A4 = A
    o, v, R = A1.shape[0], A2.shape[0], A1.shape[1]
    G = np.zeros((o, v, o, v))
    for i, a, j, b in itertools.product(range(o), range(v), range(o), range(v)):
        G[i, a, j, b] = sum(lam[r] * A1[i, r] * A2[a, r] * A3[j, r] * A4[b, r] for r in range(R))
    return G


def _brute_mttkrp(G, A, mode):
    dims = G.shape
    R = A[0].shape[1]
    M = np.zeros((dims[mode], R))
    for idx in itertools.product(*[range(d) for d in dims]):
        for r in range(R):
            p = G[idx]
            for m in range(4):
                if m != mode:
                    p *= A[m][idx[m], r]
            M[idx[mode], r] += p
    return M


def test_thc_tensor_matches_brute_force():
    Xo, Xv, Z, A, lam = _tiny(1)
    np.testing.assert_allclose(O.thc_tensor(Xo, Xv, Z), _brute_G(Xo, Xv, Z), rtol=1e-13, atol=1e-13)


def test_cpd_tensor_matches_brute_force():
    Xo, Xv, Z, A, lam = _tiny(2)
    np.testing.assert_allclose(O.cpd_tensor(A, lam), _brute_Gt(A, lam), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_mttkrp_brute_explicit_matrix_free(mode):
    # non-symmetric Z: a Z / Z^T mix-up in modes j, b fails here
    Xo, Xv, Z, A, lam = _tiny(3, sym=False)
    G = _brute_G(Xo, Xv, Z)
    Mb = _brute_mttkrp(G, A, mode)
    np.testing.assert_allclose(O.mttkrp_explicit(G, A, mode), Mb, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(O.mttkrp(Xo, Xv, Z, A, mode), Mb, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_mttkrp_matrix_free_equals_explicit_c1(mode):
    p = make_problem(5, 15, 60, 80, seed=4)
    G = O.thc_tensor(p.Xo, p.Xv, p.Z)
    Me = O.mttkrp_explicit(G, p.A, mode)
    Mf = O.mttkrp(p.Xo, p.Xv, p.Z, p.A, mode)
    assert np.max(np.abs(Mf - Me)) <= 1e-12 * np.max(np.abs(Me))


def test_rank_one_closed_form():
    # Rt = 1, R = 1: G = z (xo x xv x xo x xv) and M1[i] = z xo_i (xv.a2)(xo.a3)(xv.a4)
    rng = np.random.default_rng(5)
    xo, xv = rng.standard_normal(4), rng.standard_normal(6)
    z = 1.7
    a = [rng.standard_normal(n) for n in (4, 6, 4, 6)]
    A = tuple(x[:, None] for x in a)
    M = O.mttkrp(xo[:, None], xv[:, None], np.array([[z]]), A, 0)[:, 0]
    expect = z * xo * (xv @ a[1]) * (xo @ a[2]) * (xv @ a[3])
    np.testing.assert_allclose(M, expect, rtol=1e-14)
    M4 = O.mttkrp(xo[:, None], xv[:, None], np.array([[z]]), A, 3)[:, 0]
    np.testing.assert_allclose(M4, z * xv * (xo @ a[0]) * (xv @ a[1]) * (xo @ a[2]), rtol=1e-14)


def test_thc_norm2_closed_form_equals_sum_of_squares():
    for sym in (False, True):
        p = make_problem(5, 15, 60, 8, seed=6)
        Z = p.Z if sym else p.Z + np.triu(p.Z, 1)  # break symmetry for the second pass
        G = O.thc_tensor(p.Xo, p.Xv, Z)
        n2 = O.thc_norm2(p.Xo, p.Xv, Z)
        assert abs(n2 - O.frobenius2(G)) <= 1e-12 * n2


def test_loss_factor_form_equals_explicit():
    p = make_problem(5, 15, 60, 80, seed=7)
    lam = np.random.default_rng(7).uniform(0.1, 2.0, 80)
    Lf = O.loss_factor_form(p.Xo, p.Xv, p.Z, p.A, lam)
    Le = O.loss_explicit(p.Xo, p.Xv, p.Z, p.A, lam)
    assert abs(Lf - Le) <= 1e-11 * Le
    Xo, Xv, Z, A, lam = _tiny(8)
    Lb = float(np.sum((_brute_G(Xo, Xv, Z) - _brute_Gt(A, lam)) ** 2))
    assert abs(O.loss_factor_form(Xo, Xv, Z, A, lam) - Lb) <= 1e-12 * Lb


def test_inner_product_consistency_every_mode():
    # <G, Gt> = sum_{n,r} lam_r M_k[n,r] A_k[n,r] for every mode k
    p = make_problem(5, 15, 60, 30, seed=9)
    lam = np.random.default_rng(9).uniform(0.1, 2.0, 30)
    ref = float(np.sum(O.thc_tensor(p.Xo, p.Xv, p.Z) * O.cpd_tensor(p.A, lam)))
    for k in range(4):
        M = O.mttkrp(p.Xo, p.Xv, p.Z, p.A, k)
        assert abs(float(np.sum(lam[None, :] * M * p.A[k])) - ref) <= 1e-11 * abs(ref)
    assert abs(O.inner_thc_cpd(p.Xo, p.Xv, p.Z, p.A, lam) - ref) <= 1e-11 * abs(ref)


def test_full_orbital_symmetries_and_block():
    rng = np.random.default_rng(10)
    o, v, Rt = 2, 3, 4
    Xo, Xv = rng.standard_normal((o, Rt)), rng.standard_normal((v, Rt))
    U = np.concatenate([Xo, Xv], axis=0)
    Zs = rng.standard_normal((Rt, Rt))
    Zs = Zs + Zs.T
    g = O.thc_tensor_full(U, Zs)
    np.testing.assert_allclose(g, g.transpose(1, 0, 2, 3), rtol=0, atol=1e-13)  # within particle 1
    np.testing.assert_allclose(g, g.transpose(0, 1, 3, 2), rtol=0, atol=1e-13)  # within particle 2
    np.testing.assert_allclose(g, g.transpose(2, 3, 0, 1), rtol=0, atol=1e-12)  # particle swap, Z sym
    Zn = Zs + np.triu(rng.standard_normal((Rt, Rt)), 1)
    gn = O.thc_tensor_full(U, Zn)
    assert np.max(np.abs(gn - gn.transpose(2, 3, 0, 1))) > 1e-3  # not symmetric for non-sym Z
    G = O.thc_tensor(Xo, Xv, Zn)
    np.testing.assert_allclose(G, gn[:o, o:, :o, o:], rtol=1e-13, atol=1e-13)


def test_mode_equivariance_particle_swap():
    # swapping particles (A1,A2) <-> (A3,A4) and Z <-> Z^T maps M1<->M3, M2<->M4
    Xo, Xv, Z, A, lam = _tiny(11, o=3, v=4, Rt=5, R=3)
    As = (A[2], A[3], A[0], A[1])
    for k, ks in ((0, 2), (1, 3), (2, 0), (3, 1)):
        np.testing.assert_allclose(O.mttkrp(Xo, Xv, Z, A, k), O.mttkrp(Xo, Xv, Z.T, As, ks), rtol=1e-12)


def test_hand_golden_cases():
    with open(os.path.join(HERE, "golden", "hand_cases.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        Xo, Xv, Z = (np.array(c[k], dtype=float) for k in ("Xo", "Xv", "Z"))
        A = tuple(np.array(a, dtype=float) for a in c["A"])
        lam = np.array(c["lam"], dtype=float)
        np.testing.assert_allclose(O.thc_tensor(Xo, Xv, Z), np.array(c["G"]), rtol=1e-15)
        assert O.thc_norm2(Xo, Xv, Z) == pytest.approx(c["normG2"], rel=1e-15)
        assert O.loss_factor_form(Xo, Xv, Z, A, lam) == pytest.approx(c["loss"], rel=1e-14)
        for k in range(4):
            assert O.mttkrp(Xo, Xv, Z, A, k)[0, 0] == pytest.approx(c["mttkrp"][k], rel=1e-15)
        if "loss_after_mode0" in c:
            A2, lam2, used, _, _ = O.als_mode_update(Xo, Xv, Z, A, 0)
            np.testing.assert_allclose(lam2, c["lam_after_mode0"], rtol=1e-15)
            assert abs(O.loss_factor_form(Xo, Xv, Z, A2, lam2)) <= 1e-10


def test_als_update_is_exact_block_minimiser():
    p = make_problem(5, 15, 60, 20, seed=12)
    A = p.A
    nG2 = O.thc_norm2(p.Xo, p.Xv, p.Z)
    lam = np.ones(20)
    prev = O.loss_factor_form(p.Xo, p.Xv, p.Z, A, lam, nG2)
    for sweep in range(3):
        for k in range(4):
            A_new, lam, used, M, H = O.als_mode_update(p.Xo, p.Xv, p.Z, A, k)
            assert not used
            raw = A_new[k] * lam[None, :]
            # normal equations hold: raw H = M
            assert np.linalg.norm(raw @ H - M) <= 1e-9 * np.linalg.norm(M)
            A = A_new
            cur = O.loss_factor_form(p.Xo, p.Xv, p.Z, A, lam, nG2)
            assert cur <= prev * (1 + 1e-12) + 1e-14 * nG2
            prev = cur
    # normalised columns
    for k in range(3):
        np.testing.assert_allclose(np.linalg.norm(A[k], axis=0), 1.0, rtol=1e-13)


def test_pinv_fallback_min_norm_least_squares():
    rng = np.random.default_rng(13)
    B = rng.standard_normal((6, 5))
    B[:, 4] = B[:, 3]  # duplicated column -> singular Gram
    H = B.T @ B
    M = rng.standard_normal((3, 5))
    A, used = O.solve_normal_equations(M, H)
    assert used
    # minimum-norm solution of A H = M in the least-squares sense == lstsq on H^T
    ref = np.linalg.lstsq(H.T, M.T, rcond=None)[0].T
    np.testing.assert_allclose(A, ref, rtol=1e-8, atol=1e-10)
    # nonsingular H goes through Cholesky and matches a general solve
    H2 = H + np.eye(5)
    A2, used2 = O.solve_normal_equations(M, H2)
    assert not used2
    np.testing.assert_allclose(A2, np.linalg.solve(H2.T, M.T).T, rtol=1e-12)


def test_planted_rank12_exact_recovery():
    p, planted = make_planted(5, 15, 12, 12, seed=0, independent=True)
    # the THC block is exactly the planted CPD
    G = O.thc_tensor(p.Xo, p.Xv, p.Z)
    np.testing.assert_allclose(G, O.cpd_tensor(planted), rtol=1e-13, atol=1e-12)
    res = O.als(p.Xo, p.Xv, p.Z, p.A, max_sweeps=1000, tol=0.0)
    # factor-form fit is limited to ~sqrt(eps) by cancellation; the explicit tensor is not
    assert 1.0 - res["fits"][-1] < 1e-7
    relerr = np.linalg.norm(G - O.cpd_tensor(res["A"], res["lam"])) / np.linalg.norm(G)
    assert relerr < 1e-10
    # factors equal the planted ones up to permutation and scaling (Kruskal-unique)
    for k in range(4):
        Ak = res["A"][k] / np.linalg.norm(res["A"][k], axis=0)
        Pk = planted[k] / np.linalg.norm(planted[k], axis=0)
        C = np.abs(Ak.T @ Pk)
        used = set()
        for r in range(12):
            c = int(np.argmax([C[r, s] if s not in used else -1 for s in range(12)]))
            used.add(c)
            assert C[r, c] > 1 - 1e-8


def test_planted_overcomplete_fit_monotone():
    p, _ = make_planted(5, 15, 12, 80, seed=1, independent=False)
    res = O.als(p.Xo, p.Xv, p.Z, p.A, max_sweeps=40)
    fits = np.array(res["fits"])
    assert np.all(np.diff(fits) >= -1e-10)
    assert fits[-1] > 0.99


# --- planted mistakes: each plausible slip in the oracle must trip a pin above ---------
def test_planted_mistakes_are_caught():
    Xo, Xv, Z, A, lam = _tiny(14, o=2, v=3, Rt=3, R=2, sym=False)
    G = _brute_G(Xo, Xv, Z)
    W1, W2, W3, W4 = O.project(Xo, Xv, A)
    good = _brute_mttkrp(G, A, 2)
    wrong_transpose = Xo @ (W4 * (Z @ (W1 * W2)))       # Z instead of Z^T
    wrong_partner = Xo @ (W3 * (Z.T @ (W1 * W2)))       # wrong Hadamard partner
    dropped = Xo @ (Z.T @ (W1 * W2))                    # dropped Hadamard
    for bad in (wrong_transpose, wrong_partner, dropped):
        assert np.max(np.abs(bad - good)) > 1e-6
    S = (Xo.T @ Xo) * (Xv.T @ Xv)
    bad_norm = float(np.sum(Z * (S @ Z.T @ S)))          # transposed core in ||G||^2
    assert abs(bad_norm - O.frobenius2(G)) > 1e-6 * O.frobenius2(G)


# --- the extrapolated trial point of the learned step --------------------------------
# Hand case (R = 2, dims 1, 2, 1, 2, alpha = 2): P = previous point, N = ALS point, lam on
# the last mode. B_k = P_k + 2 (N_k - P_k) = 2 N_k - P_k, with mode 4 taken lam-absorbed:
#   B1 = 2[3 2] - [1 2] = [5 2]                    norms (5, 2)
#   B2 = 2[[1 1],[1 0]] - I = [[1 2],[2 -1]]       norms (sqrt5, sqrt5)
#   B3 = 2[2 3] - [2 1] = [2 5]                    norms (2, 5)
#   P4 lam_prev = [[2 0],[0 6]], N4 lam_new = [[0 2],[1 0]]
#   B4 = [[-2 4],[2 -6]]                           norms (2 sqrt2, 2 sqrt13)
# lam = product of the column norms = (5 sqrt5 2 2sqrt2, 2 sqrt5 5 2sqrt13) = (20 sqrt10, 20 sqrt65).
_EXT_PREV = ([[1.0, 2.0]], [[1.0, 0.0], [0.0, 1.0]], [[2.0, 1.0]], [[1.0, 0.0], [0.0, 2.0]])
_EXT_NEW = ([[3.0, 2.0]], [[1.0, 1.0], [1.0, 0.0]], [[2.0, 3.0]], [[0.0, 1.0], [1.0, 0.0]])
_EXT_LAM_PREV = [2.0, 3.0]
_EXT_LAM_NEW = [1.0, 2.0]
_S5, _S2, _S13 = np.sqrt(5.0), np.sqrt(2.0), np.sqrt(13.0)
_EXT_B = ([[1.0, 1.0]],
          [[1 / _S5, 2 / _S5], [2 / _S5, -1 / _S5]],
          [[1.0, 1.0]],
          [[-1 / _S2, 2 / _S13], [1 / _S2, -3 / _S13]])
_EXT_LAM = [20.0 * np.sqrt(10.0), 20.0 * np.sqrt(65.0)]


def _ext_inputs():
    a = lambda x: tuple(np.array(m, dtype=np.float64) for m in x)
    return a(_EXT_PREV), np.array(_EXT_LAM_PREV), a(_EXT_NEW), np.array(_EXT_LAM_NEW)


def _ext_matches(B, lam):
    return (all(np.allclose(b, np.array(e), rtol=0, atol=1e-14) for b, e in zip(B, _EXT_B))
            and np.allclose(lam, _EXT_LAM, rtol=1e-14, atol=0))


def test_extrapolate_hand_case():
    P, lp, N, ln = _ext_inputs()
    B, lam = O.extrapolate(P, lp, N, ln, 2.0)
    assert _ext_matches(B, lam)


def test_extrapolate_end_points_reproduce_the_two_tensors():
    # alpha = 0 gives back the previous point's tensor, alpha = 1 the ALS point's
    # (the definition of the step; normalisation leaves the CPD tensor unchanged)
    P, lp, N, ln = _ext_inputs()
    for alpha, (A, lam) in ((0.0, (P, lp)), (1.0, (N, ln))):
        B, lb = O.extrapolate(P, lp, N, ln, alpha)
        np.testing.assert_allclose(O.cpd_tensor(B, lb), _brute_Gt(A, lam), rtol=1e-13, atol=1e-13)
        for b in B:
            np.testing.assert_allclose(np.linalg.norm(b, axis=0), 1.0, rtol=1e-14)


def test_extrapolate_planted_mistakes_are_caught():
    # plausible slips: lam absorbed into mode 1 instead of mode 4, lam dropped, the new
    # point's lam used for both points; each misses the hand values
    P, lp, N, ln = _ext_inputs()

    def variant(mode_for_lam, lam_prev, lam_new):
        Pp = [p.copy() for p in P]
        Nn = [n.copy() for n in N]
        if mode_for_lam is not None:
            Pp[mode_for_lam] = Pp[mode_for_lam] * lam_prev[None, :]
            Nn[mode_for_lam] = Nn[mode_for_lam] * lam_new[None, :]
        B = [p + 2.0 * (n - p) for p, n in zip(Pp, Nn)]
        out, lam = [], np.ones(2)
        for b in B:
            nrm = np.linalg.norm(b, axis=0)
            out.append(b / nrm)
            lam = lam * nrm
        return out, lam

    assert _ext_matches(*variant(3, lp, ln))           # the reading itself passes
    assert not _ext_matches(*variant(0, lp, ln))       # lam on the first mode
    assert not _ext_matches(*variant(None, lp, ln))    # lam dropped
    assert not _ext_matches(*variant(3, ln, ln))       # stale lam on the previous point
