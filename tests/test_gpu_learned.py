"""Learned ALS extrapolation: the network's GPU kernels against the FP64 oracle, the
recorded training data against the oracle's own trajectory, the accept rule, and the
gain of the trained network over plain ALS."""
import os

import numpy as np
import pytest

from oracle import mlp as N
from oracle import thc_cpd as O
from tests._util import to_dev
from thc_inputs import make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2502_17683_gb300 import api as a
    return a


def _bf16(x):
    """Round float32 values to BF16 (nearest even) and back, as the kernels do."""
    t = torch.from_numpy(np.asarray(x, dtype=np.float32))
    return t.to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


def _rounded_theta(theta):
    th = np.asarray(theta, dtype=np.float64).copy()
    p = N.unpack(th)
    for name in ("W1", "W2", "w3"):
        p[name] = _bf16(p[name])
    return N.pack(p)


def test_forward_and_gradient_match_oracle(api):
    rng = np.random.default_rng(0)
    theta = (N.init(3) + 0.05 * rng.standard_normal(N.NPARAM)).astype(np.float32)
    X = rng.standard_normal((96, 40)).astype(np.float32)
    y = rng.uniform(1, 4, 96).astype(np.float32)
    P = torch.from_numpy(theta).cuda()
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    alpha = api.thc_cpd_mlp_forward(P, Xd).cpu().numpy()
    th_r = _rounded_theta(theta)   # the kernels compute with BF16-rounded weights
    a_ref, _ = N.forward(th_r, X.astype(np.float64))
    assert np.max(np.abs(alpha - a_ref)) <= 1e-5
    g, loss = api.thc_cpd_mlp_grad(P, Xd, yd)
    l_ref, g_ref = N.loss_and_grad(th_r, X.astype(np.float64), y.astype(np.float64))
    g = g.cpu().numpy().astype(np.float64)
    assert abs(loss - l_ref) <= 1e-5 * max(1.0, l_ref)
    assert np.max(np.abs(g - g_ref)) <= 1e-4 * np.max(np.abs(g_ref))
    # against the unrounded FP64 network: within the BF16 weight rounding
    l_64, g_64 = N.loss_and_grad(theta.astype(np.float64), X.astype(np.float64), y.astype(np.float64))
    assert np.max(np.abs(g - g_64)) <= 2e-2 * np.max(np.abs(g_64))


def test_adam_step_matches_oracle(api):
    # the optimiser kernel that training applies after every batch, from nonzero moments at
    # step t = 7 (bias corrections and both decay rates matter), element by element
    rng = np.random.default_rng(5)
    theta = rng.standard_normal(N.NPARAM).astype(np.float32)
    grad = (rng.standard_normal(N.NPARAM) * 10.0 ** rng.uniform(-4, 0, N.NPARAM)).astype(np.float32)
    m = (0.1 * rng.standard_normal(N.NPARAM)).astype(np.float32)
    v = (0.01 * rng.uniform(0, 1, N.NPARAM)).astype(np.float32)
    t, lr = 7, 3e-3
    # the kernel holds lr, b1, b2 and eps as FP32 constants (1 - b2 is then 1 - fl32(0.999),
    # 1.3e-5 away from 0.001): the oracle step is taken with those values
    f = lambda x: float(np.float32(x))
    th_ref, m_ref, v_ref = N.adam_step(theta.astype(np.float64), grad.astype(np.float64),
                                       m.astype(np.float64), v.astype(np.float64), t, f(lr),
                                       b1=f(0.9), b2=f(0.999), eps=f(1e-8))
    d = lambda x: torch.from_numpy(x.copy()).cuda()
    P, G, Md, Vd = d(theta), d(grad), d(m), d(v)
    api.thc_cpd_mlp_adam(P, G, Md, Vd, t, lr)
    P, Md, Vd = (x.cpu().numpy().astype(np.float64) for x in (P, Md, Vd))
    # FP32 arithmetic: a few ulps of each quantity
    assert np.max(np.abs(Md - m_ref)) <= 1e-6 * np.max(np.abs(m_ref))
    assert np.max(np.abs(Vd - v_ref) / np.maximum(v_ref, 1e-30)) <= 1e-6
    assert np.max(np.abs(P - th_ref)) <= 1e-6 * np.max(np.abs(th_ref))
    # and the step is not the identity (lr * mh / (sqrt(vh) + eps) is well above rounding)
    assert np.max(np.abs(P - theta)) > 1e-3 * lr


def test_training_fits_a_teacher(api):
    rng = np.random.default_rng(1)
    teacher = N.init(7) * 2.0
    X = rng.standard_normal((2048, 40))
    y, _ = N.forward(teacher, X)
    P = api.thc_cpd_mlp_init(11)
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    yd = torch.from_numpy(y.astype(np.float32)).cuda()
    _, l0 = api.thc_cpd_mlp_grad(P, Xd, yd)
    l1 = api.thc_cpd_mlp_train(P, Xd, yd, epochs=60, batch=64, lr=3e-3, seed=5)
    assert l1 < 0.1 * l0


def _oracle_history(p, sweeps, alphas):
    """The oracle's plain trajectory: losses, change norms, and trial losses per sweep."""
    nG2 = O.thc_norm2(p.Xo, p.Xv, p.Z)
    A, lam = p.A, np.ones(p.R)
    losses = [O.loss_factor_form(p.Xo, p.Xv, p.Z, A, lam, nG2)]
    chg, feats, tls = [], [], []
    for _ in range(sweeps):
        An, lamn, loss, _, _ = O.als_sweep(p.Xo, p.Xv, p.Z, A, lam, nG2)
        ch = []
        for k in range(4):
            a = An[k] * (lamn if k == 3 else 1.0)
            b = A[k] * (lam if k == 3 else 1.0)
            ch.append(np.linalg.norm(a - b) / np.linalg.norm(a))
        chg.append(ch)
        feats.append(N.features(losses + [loss], chg))
        row = []
        for al in alphas:
            T, lamT = O.extrapolate(A, lam, An, lamn, al)
            row.append(O.loss_factor_form(p.Xo, p.Xv, p.Z, T, lamT, nG2))
        tls.append(row)
        losses.append(loss)
        A, lam = An, lamn
    return np.array(feats), np.array(tls), nG2


def test_trajectory_features_and_trial_losses_match_oracle(api):
    p = make_problem(4, 12, 40, 24, seed=31)
    d = to_dev(p, torch)
    lam = torch.ones(24, dtype=torch.float64, device="cuda")
    alphas = [1.0, 1.5, 2.0, 3.0]
    f, tl = api.thc_cpd_als_trajectory(d["Xo"], d["Xv"], d["Z"], d["A"], lam, 6, alphas)
    f_ref, tl_ref, nG2 = _oracle_history(p, 6, alphas)
    assert np.max(np.abs(f - f_ref)) <= 1e-5
    # the loss is a difference of terms of size ||G||^2 + ||Gt||^2 (the trial CPD can be far
    # larger than G right after the random start)
    assert np.all(np.abs(tl - tl_ref) <= 1e-12 * (nG2 + np.abs(tl_ref)))


def test_accept_rule_never_worse_than_plain_step(api):
    # a network that always proposes alpha = 1.5 (zero weights, b3 = log(1/5))
    theta = np.zeros(N.NPARAM, dtype=np.float32)
    theta[-1] = np.log(1.0 / 5.0)
    P = torch.from_numpy(theta).cuda()
    assert abs(api.thc_cpd_mlp_forward(P, torch.zeros(1, 40, device="cuda")).item() - 1.5) < 1e-6
    p = make_problem(5, 15, 60, 80, seed=41)
    d = to_dev(p, torch)
    lam = torch.ones(80, dtype=torch.float64, device="cuda")
    out = api.thc_cpd_als(d["Xo"], d["Xv"], d["Z"], d["A"], lam, 30, 0.0, mlp=P, history=True)
    losses = np.array(out["losses"])
    assert out["accepted"] > 0
    # ALS steps never raise the loss and accepted trials lower it further
    assert np.all(np.diff(losses) <= 1e-12 * losses[0])
    # the reported loss is the exact loss of the returned factors
    loss, _ = api.thc_cpd_loss(d["Xo"], d["Xv"], d["Z"], d["A"], lam)
    assert abs(loss - out["loss"]) <= 1e-12 * O.thc_norm2(p.Xo, p.Xv, p.Z)


def test_trained_network_gains_over_plain_als(api):
    from paper_2502_17683_gb300 import learned
    if not os.path.exists(learned.DEFAULT_PATH):
        pytest.fail("trained parameters missing: run python -m paper_2502_17683_gb300.learned")
    P = learned.load_params()
    rows = []
    for shape, seed in (((5, 15, 60, 80), 901), ((5, 15, 60, 80), 902), ((20, 100, 480, 720), 903)):
        o, v, Rt, R = shape
        p = make_problem(o, v, Rt, R, seed=seed)
        res = {}
        for name, mlp in (("plain", None), ("learned", P)):
            d = to_dev(p, torch)
            lam = torch.ones(R, dtype=torch.float64, device="cuda")
            res[name] = api.thc_cpd_als(d["Xo"], d["Xv"], d["Z"], d["A"], lam, 3000, 1e-6, mlp=mlp)
        rows.append((res["plain"]["sweeps"], res["learned"]["sweeps"], res["plain"]["fit"],
                     res["learned"]["fit"]))
    print("sweeps to |dfit| < 1e-6 (plain, learned, fit plain, fit learned):", rows)
    assert sum(r[1] for r in rows) < sum(r[0] for r in rows)


def test_trained_network_reaches_a_common_fit_in_less_wall_time(api):
    # o=30 v=150 R_thc=720 R_cp=1080 (the learned-extrapolation workload), split precision:
    # plain ALS runs 250 sweeps; its fit is the target the learned run must reach sooner
    import time
    from paper_2502_17683_gb300 import learned
    P = learned.load_params()
    p = make_problem(30, 150, 720, 1080, seed=904)
    R = 1080

    def run(mlp, sweeps, target=0.0):
        d = to_dev(p, torch)
        lam = torch.ones(R, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = api.thc_cpd_als(d["Xo"], d["Xv"], d["Z"], d["A"], lam, sweeps, 0.0,
                              precision="bf16x3", mlp=mlp, target_fit=target)
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    run(None, 3)  # warm-up (graphs, plans)
    plain, t_plain = run(None, 250)
    learned_out, t_learned = run(P, 250, target=plain["fit"])
    print(f"plain {plain['sweeps']} sweeps {t_plain:.2f} s fit {plain['fit']:.9f}; learned "
          f"{learned_out['sweeps']} sweeps {t_learned:.2f} s fit {learned_out['fit']:.9f}")
    assert learned_out["fit"] >= plain["fit"]
    assert learned_out["sweeps"] < plain["sweeps"]
    assert t_learned < t_plain
