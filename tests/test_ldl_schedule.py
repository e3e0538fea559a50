"""Host-side checks of the dataflow LDL^T schedule (no GPU).

The normal equations of each ALS mode (Sec. 2.1) are solved by LDL^T with the rows of M
carried along. On the GPU, one CTA runs the diagonal chain (for tile s: substitution
S(s, s-1), update U(s, s, s-1), factorisation of tile (s, s)) and worker groups claim the
other tasks in list order, each waiting on per-tile progress counters. These tests take
the list from the library and check, independently of the C++ checker, that (1) it holds
every task exactly once, (2) every task comes after the tasks it waits for, and (3)
replayed with tile arithmetic under random worker schedules (counters as in the kernel),
it never deadlocks and reproduces L, D and Y = M L^-T D^-1 from numpy's Cholesky, also
when, as in the kernel, the tasks of row tile s on panels s-2 and s-3 (those that feed chain
step s) are taken out of the list and served in order by groups of their own.
"""
import random

import numpy as np
import pytest

FB = 16


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2502_17683_gb300 import api as a
    return a


def _tiles(R, n):
    return -(-R // FB), -(-n // FB)


def _expected(R, n):
    nT, nM = _tiles(R, n)
    s = set()
    for k in range(nT):
        for t in list(range(k + 2, nT)) + list(range(nT, nT + nM)):
            s.add((0, t, 0, k))
        for j in range(k + 1, nT):
            for t in list(range(j, nT)) + list(range(nT, nT + nM)):
                if not (t == j == k + 1):
                    s.add((1, t, j, k))
    return s


# ... and the shapes the emulated factorisation launches at R_cp = 1800: 256-column panels over
# the rows below them (up to 1794 with n = 250), 128-column ones, and the 520-column tail
@pytest.mark.parametrize("R,n", [(720, 20), (720, 100), (80, 5), (17, 1), (16, 3), (5, 4),
                                 (33, 40), (144, 20), (100, 0), (31, 33), (1800, 250),
                                 (256, 1794), (128, 1922), (520, 250), (520, 50)])
def test_schedule_complete_and_ordered(api, R, n):
    tasks = api.thc_cpd_ldl_schedule(R, n)
    nT, nM = _tiles(R, n)
    assert len(tasks) == len(set(tasks)) == len(_expected(R, n))
    assert set(tasks) == _expected(R, n)
    pos = {t: i for i, t in enumerate(tasks)}
    # chain step s waits for U(s, s-1, m) and U(s, s, m), m <= s - 2
    wmax = []
    w = -1
    for s in range(nT):
        for m in range(s - 1):
            w = max(w, pos[(1, s, s - 1, m)], pos[(1, s, s, m)])
        wmax.append(w)
    for i, (ty, t, j, k) in enumerate(tasks):
        if ty == 0:
            assert all(pos[(1, t, k, m)] < i for m in range(k))
            assert wmax[k] < i  # waits for the chain's factorisation of tile (k, k)
        else:
            for r in (t, j):
                if not (r < nT and r == k + 1):
                    assert pos[(0, r, 0, k)] < i
            if k:
                assert pos[(1, t, j, k - 1)] < i
            if j == k + 1:
                assert wmax[k + 1] < i  # waits for the chain's substitution of row tile k+1


def test_schedule_rejects_out_of_range(api):
    from paper_2502_17683_gb300._lib import ThcCpdError
    with pytest.raises(ThcCpdError):
        api.thc_cpd_ldl_schedule(0, 4)
    with pytest.raises(ThcCpdError):
        api.thc_cpd_ldl_schedule(16 * 257, 4)


def _critical(tk, nT):
    ty, t, j, k = tk
    return t < nT and k >= t - 3


def _replay(R, n, tasks, workers, seed, crit_workers=0):
    """Run the tasks with `workers` groups claiming tickets in order and a random choice,
    at every step, among the runnable actions (a group whose inputs are ready, or the
    chain). With crit_workers > 0 the critical tasks form a second list, claimed in order
    by that many groups of their own. Tile arithmetic as in the kernel; returns the final
    augmented matrix."""
    rng = np.random.default_rng(seed)
    pick = random.Random(seed)
    nT, nM = _tiles(R, n)
    B = rng.standard_normal((R + 3, R))
    H = B.T @ B + 0.1 * R * np.eye(R)
    M = rng.standard_normal((n, R))
    Hg = np.vstack([np.tril(H), M])
    P = np.zeros((R, R))
    dinv = np.zeros(R)

    def rows(t):
        if t < nT:
            return t * FB, min(R, t * FB + FB)
        return R + (t - nT) * FB, min(R + n, R + (t - nT) * FB + FB)

    def cols(k):
        return k * FB, min(R, k * FB + FB)

    def subst(t, k, L, dv):
        r0, r1 = rows(t)
        k0, k1 = cols(k)
        Bt = Hg[r0:r1, k0:k1]
        X = np.zeros_like(Bt)
        for c in range(k1 - k0):
            X[:, c] = Bt[:, c] - X[:, :c] @ L[c, :c]
        Hg[r0:r1, k0:k1] = X * dv
        if t < nT:
            P[r0:r1, k0:k1] = X

    def update(t, j, k):
        r0, r1 = rows(t)
        c0, c1 = cols(j)
        k0, k1 = cols(k)
        u = Hg[r0:r1, k0:k1] @ P[c0:c1, k0:k1].T
        Hg[r0:r1, c0:c1] -= np.tril(u) if t == j else u

    def factor(s):
        s0, s1 = cols(s)
        S = np.tril(Hg[s0:s1, s0:s1])
        S = S + np.tril(S, -1).T
        jb = s1 - s0
        L, d = np.eye(jb), np.zeros(jb)
        for c in range(jb):
            d[c] = S[c, c]
            L[c + 1:, c] = S[c + 1:, c] / d[c]
            S[c + 1:, c + 1:] -= np.outer(L[c + 1:, c], S[c, c + 1:])
        Hg[s0:s1, s0:s1] = np.tril(L, -1) + np.diag(d)
        dinv[s0:s1] = 1.0 / d

    cnt = np.zeros((nT + nM, nT), int)
    sdone = np.zeros(nT + nM, int)
    fdone = chain = 0
    if crit_workers:
        lists = [[x for x in tasks if not _critical(x, nT)], [x for x in tasks if _critical(x, nT)]]
        lanes = [0] * workers + [1] * crit_workers
    else:
        lists, lanes = [tasks], [0] * workers
    tickets = [0] * len(lists)
    held = [None] * len(lanes)

    def ready(tk):
        ty, t, j, k = tk
        if ty == 0:
            return fdone >= k + 1 and cnt[t, k] >= k
        return sdone[t] >= k + 1 and sdone[j] >= k + 1 and cnt[t, j] >= k

    while True:
        for w, lane in enumerate(lanes):
            if held[w] is None and tickets[lane] < len(lists[lane]):
                held[w] = lists[lane][tickets[lane]]
                tickets[lane] += 1
        acts = [w for w in range(len(lanes)) if held[w] is not None and ready(held[w])]
        if chain < nT and (chain == 0 or (cnt[chain, chain - 1] >= chain - 1 and
                                          cnt[chain, chain] >= chain - 1)):
            acts.append("chain")
        if not acts:
            assert chain == nT and all(tk == len(ls) for tk, ls in zip(tickets, lists)) and \
                all(h is None for h in held), "schedule deadlocked"
            return H, M, Hg
        a = pick.choice(acts)
        if a == "chain":
            s = chain
            if s:
                p0, p1 = cols(s - 1)
                subst(s, s - 1, np.tril(Hg[p0:p1, p0:p1], -1), dinv[p0:p1])
                sdone[s] = s
                update(s, s, s - 1)
            factor(s)
            fdone = chain = s + 1
        else:
            ty, t, j, k = held[a]
            if ty == 0:
                k0, k1 = cols(k)
                subst(t, k, np.tril(Hg[k0:k1, k0:k1], -1), dinv[k0:k1])
                sdone[t] = k + 1
            else:
                update(t, j, k)
                cnt[t, j] = k + 1
            held[a] = None


@pytest.mark.parametrize("R,n", [(70, 21), (64, 40), (33, 17), (129, 35)])
@pytest.mark.parametrize("workers,crit", [(1, 0), (3, 0), (64, 0), (1, 1), (3, 2), (64, 1)])
def test_schedule_replay_reproduces_ldlt(api, R, n, workers, crit):
    tasks = api.thc_cpd_ldl_schedule(R, n)
    for seed in (0, 1):
        H, M, Hg = _replay(R, n, tasks, workers, seed, crit)
        C = np.linalg.cholesky(H)
        d = np.diag(C) ** 2
        L = C / np.diag(C)
        Y = np.linalg.solve(L, M.T).T / d
        assert np.max(np.abs(np.tril(Hg[:R], -1) - np.tril(L, -1))) < 1e-12
        assert np.max(np.abs(np.diag(Hg[:R]) - d) / d) < 1e-12
        assert np.max(np.abs(Hg[R:] - Y)) <= 1e-12 * max(1.0, np.max(np.abs(Y)))
