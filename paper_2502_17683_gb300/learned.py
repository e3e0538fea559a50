"""Training of the ALS step proposer (learned extrapolation), end to end on the GPU.

Data: plain ALS trajectories that the library itself runs (thc_cpd_als_trajectory) on
synthetic THC problems of the paper-shaped sizes (o, v, R_thc, R_cp) =
(5, 15, 60, 80), (20, 100, 480, 720) and (50, 250, 1200, 1800) with several seeds. After
every sweep the library records the 40 history features and the exact FP64 losses of
the trial points P + alpha (P_ALS - P) on a grid of alpha; the label is the grid alpha
with the lowest loss (1 when no trial beats the ALS point).
Training: Adam on the mean squared error of alpha, by the library's own forward /
backward / update kernels (thc_cpd_mlp_train).

  python -m paper_2502_17683_gb300.learned [--quick] [--out PATH]
writes the parameters (6849 float32) to PATH (default: extrapolator.npy next to this
file), which thc_cpd_als uses through `mlp=`.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_PATH = os.path.join(HERE, "extrapolator.npy")
ALPHAS = np.round(np.arange(1.0, 4.0001, 0.25), 6)

# (o, v, R_thc, R_cp, seeds, sweeps) per training workload
TRAIN_SET = [
    (5, 15, 60, 80, range(100, 124), 80),
    (20, 100, 480, 720, range(200, 206), 60),
    (50, 250, 1200, 1800, range(300, 302), 25),
]
QUICK_SET = [
    (5, 15, 60, 80, range(100, 106), 40),
    (20, 100, 480, 720, range(200, 201), 20),
]


def labels_from_losses(trial_losses: np.ndarray) -> np.ndarray:
    """alpha with the lowest exact loss per sweep (column 0 is alpha = 1, the ALS point)."""
    best = np.argmin(trial_losses, axis=1)
    return ALPHAS[best].astype(np.float32)


def generate(train_set, precision="fp64", log=print):
    import torch
    from thc_inputs import make_problem
    from . import api
    Xs, ys = [], []
    for o, v, Rt, R, seeds, sweeps in train_set:
        for seed in seeds:
            p = make_problem(o, v, Rt, R, seed=seed, decay=Rt / 5.0)
            t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
            A = [t(a) for a in p.A]
            lam = torch.ones(R, dtype=torch.float64, device="cuda")
            f, tl = api.thc_cpd_als_trajectory(t(p.Xo), t(p.Xv), t(p.Z), A, lam, sweeps, ALPHAS,
                                               precision=precision)
            Xs.append(f[1:])  # from the second sweep on (one decrement exists)
            ys.append(labels_from_losses(tl[1:]))
        log(f"  trajectories o={o} v={v} R_thc={Rt} R_cp={R}: {len(seeds)} x {sweeps} sweeps")
    return np.concatenate(Xs).astype(np.float32), np.concatenate(ys).astype(np.float32)


def train(X, y, epochs=300, batch=64, lr=2e-3, seed=0):
    import torch
    from . import api
    params = api.thc_cpd_mlp_init(seed)
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    yd = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    _, l0 = api.thc_cpd_mlp_grad(params, Xd, yd)
    l1 = api.thc_cpd_mlp_train(params, Xd, yd, epochs, batch, lr, seed)
    return params, l0, l1


def load_params(path: str = DEFAULT_PATH):
    import torch
    return torch.from_numpy(np.load(path).astype(np.float32)).cuda()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_PATH)
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--epochs", type=int, default=300)
    args = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(HERE))
    t0 = time.time()
    X, y = generate(QUICK_SET if args.quick else TRAIN_SET)
    t1 = time.time()
    params, l0, l1 = train(X, y, epochs=args.epochs)
    np.save(args.out, params.cpu().numpy())
    info = {"samples": int(len(y)), "label_mean": float(y.mean()),
            "label_frac_gt1": float(np.mean(y > 1.0)), "mse_before": l0, "mse_after": l1,
            "data_s": round(t1 - t0, 1), "train_s": round(time.time() - t1, 1)}
    print(json.dumps(info))
    return 0


if __name__ == "__main__":
    sys.exit(main())
