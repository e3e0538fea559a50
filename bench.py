#!/usr/bin/env python
"""ALS sweeps/s of THC-driven matrix-free CP-ALS on one GB300.

Workload (one step): thc_cpd_als on the o=50, v=250, R_thc=1200, R_cp=1800 THC block
(synthetic THC factors with Z decay scale 240, seed 0; 100 sweeps, no early stop),
restarted from the same start factors every step. value = sweeps/s over all ranks (each
rank solves its own independent problem: weak scaling, no collective on the data path).
Beside it: the plain FP64 GPU path on the same workload, and the wall-time each form
(FP64, BF16x3, BF16x3 with the learned extrapolation) needs to reach one common fit.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|bf16x3|tf32x3]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores
  python bench.py --drift-report         # per-sweep fit differences from identical starts
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

W = dict(o=50, v=250, Rt=1200, R=1800, sweeps=100, seed=0, decay=240.0)
WORKLOAD = "THC-driven CP-ALS, o=50 v=250 R_thc=1200 R_cp=1800 (Z decay 240), 100 sweeps per step"
# other paper-shaped sizes, for profiling captures (the bench line uses the default)
CONFIGS = {
    "c1": dict(o=5, v=15, Rt=60, R=80, sweeps=25),
    "c2": dict(o=20, v=100, Rt=480, R=720, sweeps=50),
    "c3": dict(o=50, v=250, Rt=1200, R=1800, sweeps=100, decay=240.0),
    "c5": dict(o=30, v=150, Rt=720, R=1080, sweeps=50),
}
METRIC = "ALS sweeps/s"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweeps", type=int, default=None,
                    help="sweeps per step (profiling captures only; the bench line uses 100)")
    ap.add_argument("--config", default="c3", choices=sorted(CONFIGS),
                    help="workload size (profiling captures only; the bench line uses c3)")
    ap.add_argument("--ldl", default="auto", choices=["auto", "dataflow", "blocked", "emulated"],
                    help="factorisation of the normal equations (thc_cpd_opts.ldl)")
    ap.add_argument("--no-equal-fit", action="store_true",
                    help="skip the wall-time-to-a-common-fit comparison")
    ap.add_argument("--drift-report", action="store_true",
                    help="o=20 v=100 R_thc=480 R_cp=720, 50 sweeps: per-sweep |fit - fit_fp64| of "
                         "the split precisions and of FP64 runs from perturbed starts")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip timing the FP64 path beside the split precision")
    ap.add_argument("--learned-report", action="store_true",
                    help="o=30 v=150 R_thc=720 R_cp=1080, split precision: sweeps and wall-time "
                         "to a 1e-6 fit change, plain vs learned extrapolation")
    ap.add_argument("--profile-run", action="store_true",
                    help="run one step (--sweeps sweeps of --config) untimed and exit: the "
                         "command the ncu captures under profiles/ run")
    ap.add_argument("--rows-report", action="store_true",
                    help="the rows beyond the ALS hot path at the bench sizes: exchange energy, "
                         "THC core fit, DF- vs THC-driven ALS, order-6 ALS (GPU FP64 and emulated, "
                         "each beside its oracle on the host cores)")
    ap.add_argument("--batched", action="store_true",
                    help="64 uneven problems (o in [4,40], v=5o, R_thc=4(o+v), R_cp=6(o+v) "
                         "rounded up to 16), 40 sweeps each: batched graph vs one by one")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# nominal dense rates (TFLOP/s) used to carry the measured bf16 peak over to other dtypes
NOMINAL = {"bf16": 2250.0, "tf32": 1100.0, "fp64": 1.25}


def fp64_peaks(dev, sm_max_mhz):
    """FP64 roofline denominators: the FP64 FMA rate measured by the library's probe kernel,
    cuBLAS DGEMM (torch float64 matmul, 8192^3, best of 5) and the rate derived from the unit
    counts (SMs read from the device x 2 FP64 FMA per clock x 2 flop x the maximum SM clock)."""
    import torch
    from paper_2502_17683_gb300 import api
    probe = api.thc_cpd_fp64_fma_rate()
    n = 8192
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    best = 0.0
    for i in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        if i:
            best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) / 1e3) / 1e12)
    del a, b
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = sm_max_mhz or 2070.0
    return {"probe_tflops": probe, "dgemm_tflops": best, "nsm": nsm,
            "derived_tflops": nsm * 2 * 2 * mhz * 1e6 / 1e12, "sm_max_mhz": mhz}


# DRAM bytes per launch of k_ldl_flow (one launch per solve on the dataflow path, one per
# panel on the emulated path), keyed by (workload, path), from one ncu capture of
# one sweep of that workload (all of the sweep's launches averaged; ncu starts every launch
# from a flushed cache, so this is the cold-cache figure), and the SHA-256 of the kernel's
# sources (concatenated in this order) it was taken on: reported only while they are
# unchanged.
LDL_SOURCES = [os.path.join("paper_2502_17683_gb300", "csrc", f)
               for f in ("ldl_flow.cu", "ldl_common.cuh", "common.cuh", "oz_gemm.cu")]
LDL_TRAFFIC = {
    # 24 launches of sweep 1: 20 panels of 256 columns and 4 tails
    # (profiles/ldl_flow_panels_o50_v250_Rt1200_R1800_emulated.md)
    ("c3", "emulated"): {"bytes_per_launch": 2810539,
                         "sha256": "d4600829b64cd367ddca378d58a8afd98a7b436117a55d9636a58fae6d451452"},
}


def ldl_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for src in LDL_SOURCES:
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def ldl_traffic(config, path):
    rec = LDL_TRAFFIC.get((config, path))
    if not rec:
        return None
    try:
        sha = ldl_sources_sha256()
    except OSError:
        return None
    return rec["bytes_per_launch"] if sha == rec["sha256"] else None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, x in enumerate(r) if x.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over all ranks (barrier semantics); x itself without a process
    group. Works on any backend (NCCL with a CUDA device, gloo on the CPU)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, ms_per_rank: float, device=None):
    """Whole-job throughput of independent replicas: all ranks' units over the slowest
    rank's time (weak scaling)."""
    import torch.distributed as dist
    world = dist.get_world_size() if (dist.is_available() and dist.is_initialized()) else 1
    ms = max_over_ranks(ms_per_rank, device)
    return world * units_per_rank / (ms / 1000.0), ms


def oracle_sweeps_per_s(seconds: float, seed: int):
    """The FP64 CPU oracle as it stands, on the host cores, over a bounded number of sweeps
    of the same workload from the same start point."""
    from oracle import thc_cpd as O
    from thc_inputs import make_problem
    p = make_problem(W["o"], W["v"], W["Rt"], W["R"], seed=seed, decay=W.get("decay"))
    nG2 = O.thc_norm2(p.Xo, p.Xv, p.Z)
    A, lam = p.A, None
    t0 = time.perf_counter()
    A, lam, _, _, _ = O.als_sweep(p.Xo, p.Xv, p.Z, A, lam, nG2)
    t1 = time.perf_counter() - t0
    n = max(1, int(seconds / max(t1, 1e-6)) - 1)
    t0 = time.perf_counter()
    for _ in range(n):
        A, lam, _, _, _ = O.als_sweep(p.Xo, p.Xv, p.Z, A, lam, nG2)
    dt = time.perf_counter() - t0
    return n / dt, n, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    per_step = max(1.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sweeps_per_s(per_step / 4, W["seed"])
    vals, sweeps, secs = [], 0, 0.0
    for _ in range(args.steps):
        v, n, dt = oracle_sweeps_per_s(per_step, W["seed"])
        vals.append(v)
        sweeps += n
        secs += dt
    value = sweeps / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "sweeps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "o": W["o"], "v": W["v"], "R_thc": W["Rt"],
                   "R_cp": W["R"], "sweeps_per_step": W["sweeps"], "precision": "fp64",
                   "note": "each step is a bounded sample of sweeps of the workload"},
        "cpu_baseline": {"value": value, "unit": "sweeps/s", "cores": os.cpu_count(),
                         "kind": "oracle", "sample": f"{sweeps} sweeps over {args.steps} steps, "
                         "numpy/OpenBLAS FP64 matrix-free ALS"},
        "e2e": {"value": value, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def learned_report(args):
    """Wall-time and sweeps to |fit_s - fit_{s-1}| < 1e-6 at o=30 v=150 R_thc=720
    R_cp=1080 (split precision), plain ALS vs the trained step proposer, plus plain FP64."""
    import numpy as np
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2502_17683_gb300 import api, learned
    from thc_inputs import make_problem
    prec = args.precision or "bf16x3"
    P = learned.load_params()
    rows = {}
    for seed in (0, 1):
        p = make_problem(30, 150, 720, 1080, seed=seed)
        t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
        for name, mlp, pr in (("plain", None, prec), ("learned", P, prec), ("plain_fp64", None, "fp64")):
            A = [t(a) for a in p.A]
            lam = torch.ones(1080, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = api.thc_cpd_als(t(p.Xo), t(p.Xv), t(p.Z), A, lam, 5000, 1e-6, precision=pr, mlp=mlp)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            rows.setdefault(name, []).append({"seed": seed, "sweeps": out["sweeps"], "seconds": dt,
                                              "fit": out["fit"], "accepted": out.get("accepted", 0)})
    print(json.dumps({"report": "learned extrapolation", "workload":
                      "o=30 v=150 R_thc=720 R_cp=1080, stop at |dfit| < 1e-6", "precision": prec,
                      "rows": rows}))
    return 0


def batched_report(args):
    """64 uneven problems, 40 sweeps each, split precision: one batched call (one CUDA
    graph per sweep for all problems, autotuned tiles) vs the same problems one by one."""
    import numpy as np
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2502_17683_gb300 import api
    from thc_inputs import batched_shapes, make_problem
    prec = args.precision or "bf16x3"
    shapes = batched_shapes(64, seed=0)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    probs = [make_problem(o, v, Rt, R, seed=i) for i, (o, v, Rt, R) in enumerate(shapes)]
    dev = [dict(Xo=t(p.Xo), Xv=t(p.Xv), Z=t(p.Z), A0=[t(a) for a in p.A]) for p in probs]

    def fresh():
        out = []
        for d, p in zip(dev, probs):
            out.append(dict(Xo=d["Xo"], Xv=d["Xv"], Z=d["Z"], A=[a.clone() for a in d["A0"]],
                            lam=torch.ones(p.R, dtype=torch.float64, device="cuda")))
        return out
    sweeps = 40
    flops = 0.0
    for (o, v, Rt, R) in shapes:
        n = o + v
        flops += sweeps * (4 * Rt * Rt * R + 8 * n * Rt * R + 2 * n * R * R + 4 * R ** 3 / 3 + 4 * n * R * R)
    api.thc_cpd_als_batched(fresh(), 2, 0.0, precision=prec, autotune=True)  # warm-up + tuning
    torch.cuda.synchronize()
    res = {}
    for name in ("batched", "one_by_one"):
        best = 1e30
        for _ in range(2):
            pr = fresh()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if name == "batched":
                outs = api.thc_cpd_als_batched(pr, sweeps, 0.0, precision=prec)
            else:
                outs = [api.thc_cpd_als(d["Xo"], d["Xv"], d["Z"], d["A"], d["lam"], sweeps, 0.0,
                                        precision=prec) for d in pr]
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        res[name] = {"seconds": best, "problem_sweeps_per_s": 64 * sweeps / best,
                     "useful_tflops": flops / best / 1e12,
                     "mean_fit": float(np.mean([o["fit"] for o in outs]))}
    print(json.dumps({"report": "batched", "problems": 64, "sweeps": sweeps, "precision": prec,
                      "shapes": {"o_min": min(s[0] for s in shapes), "o_max": max(s[0] for s in shapes),
                                 "R_cp_max": max(s[3] for s in shapes)},
                      "rows": res, "speedup": res["one_by_one"]["seconds"] / res["batched"]["seconds"]}))
    return 0


def rows_report(args):
    """Exchange energy, THC core fit, DF-driven vs THC-driven ALS and order-6 ALS at the bench
    sizes (o=50 v=250 R_thc=1200 R_cp=1800, naux=1200; order 6: (20,100) x 3, R_thc=480,
    R_cp=720): GPU time per call (best of 3 after a warm-up; each call synchronises) with the
    FP64 pipes and with the emulated tensor-core products, the algorithmic FP64 flop rate, and
    the oracle's time on the host cores for one call (DF-driven and order-6 ALS: one sweep)."""
    import numpy as np
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2502_17683_gb300 import api
    from thc_inputs import make_df, make_factors, make_lt, make_nd, make_problem
    from oracle import corefit as OC, df_cpd as OD, exchange as OX, nd as ON
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    probe = None
    try:
        probe = api.thc_cpd_fp64_fma_rate()
    except Exception:
        probe = None

    def gpu_best(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        return best

    def cpu_once(fn):
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    def row(flops, t64, temu, tcpu, unit_note):
        out = {"fp64_s": t64, "emulated_s": temu, "oracle_s": tcpu, "flop": flops,
               "fp64_tflops": flops / t64 / 1e12, "emulated_tflops": flops / temu / 1e12,
               "emulated_speedup": t64 / temu, "vs_oracle": tcpu / temu, "unit": unit_note}
        if probe:
            out["fp64_frac_of_fma_rate"] = out["fp64_tflops"] / probe
        return out

    rows = {}
    o, v, Rt, R, naux = 50, 250, 1200, 1800, 1200
    nmax = max(o, v)
    # exchange energy (12 Laplace points) on the bench THC block and random CP factors
    p = make_problem(o, v, Rt, R, seed=0, decay=240.0)
    rng = np.random.default_rng(0)
    lam = rng.uniform(0.5, 2.0, R)
    eo, ev, tq, wq = make_lt(o, v, 12, 0)
    Lam, Gam = OX.lt_factors(eo, ev, tq, wq)
    dX = dict(Xo=d(p.Xo), Xv=d(p.Xv), Z=d(p.Z), A=[d(a) for a in p.A], lam=d(lam), Lam=d(Lam), Gam=d(Gam))
    ex = lambda emu: api.thc_cpd_exchange(dX["Xo"], dX["Xv"], dX["Z"], dX["A"], dX["lam"], dX["Lam"],
                                          dX["Gam"], emulated=emu)
    fl = 12 * (4.0 * (o + v) * Rt * R + 2.0 * Rt * Rt * R + 4.0 * o * R * R + 2.0 * v * R * R)
    tc = cpu_once(lambda: OX.exchange_robust(p.Xo, p.Xv, p.Z, p.A, lam, Lam[:1], Gam[:1])) * 12
    rows["exchange_energy"] = row(fl, gpu_best(lambda: ex(False)), gpu_best(lambda: ex(True)), tc,
                                  "one call, 12 quadrature points (oracle: 1 point x 12)")
    # THC core fit from a DF tensor
    Xo, Xv, B = make_df(o, v, Rt, naux, seed=1)
    dC = dict(Xo=d(Xo), Xv=d(Xv), B=d(B))
    cf = lambda emu: api.thc_cpd_core_fit(dC["Xo"], dC["Xv"], dC["B"], emulated=emu)
    fl = 2.0 * naux * o * v * Rt + 2.0 * naux * o * Rt + (o + v) * Rt * Rt + Rt ** 3 / 3 + 3.0 * naux * Rt * Rt
    tc = cpu_once(lambda: OC.core_fit(Xo, Xv, B))
    rows["core_fit"] = row(fl, gpu_best(lambda: cf(False)), gpu_best(lambda: cf(True)), tc, "one fit")
    # DF-driven vs THC-driven ALS, 3 sweeps from the same start
    A0 = make_factors((o, v, o, v), R, 2)
    dB = d(B)

    def df_run(emu):
        A = [d(a) for a in A0]
        lamd = torch.ones(R, dtype=torch.float64, device="cuda")
        api.thc_cpd_df_als(dB, A, lamd, 3, emulated=emu)
    fl = 3 * (8.0 * naux * o * v * R + 4 * R ** 3 / 3 + 4.0 * (o + v) * R * R)
    pc = make_df(20, 100, 480, 480, seed=1)[2]
    Ac = make_factors((20, 100, 20, 100), 720, 2)
    tc = cpu_once(lambda: OD.df_als(pc, Ac, 1))
    rows["df_als"] = row(fl, gpu_best(lambda: df_run(False), 2), gpu_best(lambda: df_run(True), 2), tc,
                         "3 sweeps at naux=1200 (oracle: 1 sweep at o=20 v=100 naux=480 R_cp=720)")
    rows["df_als"]["sweeps_per_s_fp64"] = 3 / rows["df_als"]["fp64_s"]
    rows["df_als"]["sweeps_per_s_emulated"] = 3 / rows["df_als"]["emulated_s"]
    pt = make_problem(o, v, Rt, R, seed=0, decay=240.0)
    dT = dict(Xo=d(pt.Xo), Xv=d(pt.Xv), Z=d(pt.Z))
    thc = {}
    for prec, ldl in (("fp64", "dataflow"), ("fp64", "emulated"), ("bf16x3", "emulated")):
        def th():
            A = [d(a) for a in A0]
            lamd = torch.ones(R, dtype=torch.float64, device="cuda")
            api.thc_cpd_als(dT["Xo"], dT["Xv"], dT["Z"], A, lamd, 3, 0.0, precision=prec, ldl=ldl)
        thc[f"{prec}+{ldl}"] = 3 / gpu_best(th, 2)
    rows["df_als"]["thc_driven_sweeps_per_s"] = thc
    # order-6 ALS
    dims, Rt6, R6 = (20, 100, 20, 100, 20, 100), 480, 720
    X6, Z6, A6 = make_nd(dims, Rt6, R6, seed=3)
    dX6, dZ6 = [d(x) for x in X6], d(Z6)

    def nd_run(emu):
        A = [d(a) for a in A6]
        lamd = torch.ones(R6, dtype=torch.float64, device="cuda")
        api.thc_cpd_nd_als(dX6, dZ6, A, lamd, 3, 3, emulated=emu)
    n6 = sum(dims)
    fl = 3 * (2.0 * (2 * n6) * Rt6 * R6 + 2 * 2.0 * Rt6 * Rt6 * R6 + n6 * R6 * R6 + 6 * R6 ** 3 / 3 + 2.0 * n6 * R6 * R6)
    tc = cpu_once(lambda: ON.nd_als(X6, Z6, 3, A6, 1))
    rows["order6_als"] = row(fl, gpu_best(lambda: nd_run(False), 2), gpu_best(lambda: nd_run(True), 2), tc * 3,
                             "3 sweeps (oracle: 1 sweep x 3)")
    rows["order6_als"]["sweeps_per_s_fp64"] = 3 / rows["order6_als"]["fp64_s"]
    rows["order6_als"]["sweeps_per_s_emulated"] = 3 / rows["order6_als"]["emulated_s"]
    print(json.dumps({"report": "rows beyond the ALS hot path", "fp64_fma_tflops": probe,
                      "sizes": {"o": o, "v": v, "R_thc": Rt, "R_cp": R, "naux": naux,
                                "order6": {"dims": dims, "R_thc": Rt6, "R_cp": R6}},
                      "rows": rows}))
    return 0


def drift_report(args):
    """Per-sweep |fit - fit_fp64| on o=20 v=100 R_thc=480 R_cp=720 over 50 sweeps from one
    start: the split precisions, and FP64 runs whose start factors carry a relative
    perturbation of 1e-9, 1e-7 and 1e-5 (how far ALS itself carries a perturbation of a given
    size along this unconverged trajectory). All fits are exact FP64 losses."""
    import numpy as np
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2502_17683_gb300 import api
    from thc_inputs import make_problem
    o, v, Rt, R, sweeps = 20, 100, 480, 720, 50
    p = make_problem(o, v, Rt, R, seed=0)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    Xo, Xv, Z = t(p.Xo), t(p.Xv), t(p.Z)

    def run(prec, eps=0.0):
        rng = np.random.default_rng(123)
        A = [t(a * (1.0 + eps * rng.standard_normal(a.shape))) for a in p.A]
        lam = torch.ones(R, dtype=torch.float64, device="cuda")
        out = api.thc_cpd_als(Xo, Xv, Z, A, lam, sweeps, 0.0, precision=prec, loss_every=1,
                              history=True)
        return np.array(out["fits"])

    ref = run("fp64")
    rows = {}
    for name, prec, eps in (("bf16x3", "bf16x3", 0.0), ("tf32x3", "tf32x3", 0.0),
                            ("fp64_start_1e-9", "fp64", 1e-9), ("fp64_start_1e-7", "fp64", 1e-7),
                            ("fp64_start_1e-5", "fp64", 1e-5)):
        d = np.abs(run(prec, eps) - ref)
        rows[name] = {"sweep": [1, 2, 5, 10, 20, 30, 40, 50],
                      "abs_fit_diff": [float(d[s - 1]) for s in (1, 2, 5, 10, 20, 30, 40, 50)],
                      "max": float(d.max())}
    print(json.dumps({"report": "drift", "workload": "o=20 v=100 R_thc=480 R_cp=720, 50 sweeps, seed 0",
                      "fp64_fit": [float(ref[s - 1]) for s in (1, 10, 50)], "rows": rows}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.learned_report:
        return learned_report(args)
    if args.batched:
        return batched_report(args)
    if args.drift_report:
        return drift_report(args)
    if args.rows_report:
        return rows_report(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__ as g
    g.build()
    from paper_2502_17683_gb300 import api
    from thc_inputs import make_problem

    precision = args.precision or "bf16x3"
    global WORKLOAD
    if args.config != "c3":
        W.update(CONFIGS[args.config])
        W["decay"] = CONFIGS[args.config].get("decay")
        WORKLOAD = (f"THC-driven CP-ALS, o={W['o']} v={W['v']} R_thc={W['Rt']} R_cp={W['R']}, "
                    f"{W['sweeps']} sweeps per step")
    if args.sweeps:
        W["sweeps"] = args.sweeps
    p = make_problem(W["o"], W["v"], W["Rt"], W["R"], seed=W["seed"] + rank, decay=W.get("decay"))
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    Xo, Xv, Z = t(p.Xo), t(p.Xv), t(p.Z)
    A0 = [t(a) for a in p.A]
    A = [a.clone() for a in A0]
    lam = torch.ones(W["R"], dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        return api.thc_cpd_als(Xo, Xv, Z, A, lam, W["sweeps"], 0.0, precision=precision, ldl=args.ldl)

    def reset():
        for a, a0 in zip(A, A0):
            a.copy_(a0)

    if args.profile_run:
        out = step()
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": WORKLOAD, "precision": precision, "fit": out["fit"]}))
        return

    for _ in range(args.warmup):
        reset()
        out = step()
    torch.cuda.synchronize()

    # ---- timed region (device time per step, L2 flushed between steps) ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = api.thc_cpd_launch_count()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            reset()
            ev[k][0].record(stream)
            out = step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    launches = api.thc_cpd_launch_count() - l0
    if world > 1:
        dist.barrier()
    value, ms = job_throughput(args.steps * W["sweeps"], sum(a.elapsed_time(b) for a, b in ev), dev)
    sweeps_total = world * args.steps * W["sweeps"]
    fit = out["fit"]

    # ---- end to end through the public API with host buffers ----
    hp = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    hXo, hXv, hZ = hp(p.Xo), hp(p.Xv), hp(p.Z)
    hA = [hp(a) for a in p.A]
    oA = [torch.empty_like(a).pin_memory() for a in hA]
    olam = torch.empty(W["R"], dtype=torch.float64).pin_memory()
    h2d = sum(x.numel() * 8 for x in [hXo, hXv, hZ] + hA)
    d2h = sum(x.numel() * 8 for x in oA) + olam.numel() * 8
    dXo, dXv, dZ = torch.empty_like(Xo), torch.empty_like(Xv), torch.empty_like(Z)

    def e2e_step():
        dXo.copy_(hXo, non_blocking=True)
        dXv.copy_(hXv, non_blocking=True)
        dZ.copy_(hZ, non_blocking=True)
        for a, h in zip(A, hA):
            a.copy_(h, non_blocking=True)
        api.thc_cpd_als(dXo, dXv, dZ, A, lam, W["sweeps"], 0.0, precision=precision, ldl=args.ldl)
        for o_, a in zip(oA, A):
            o_.copy_(a, non_blocking=True)
        olam.copy_(lam, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        ev2[k][0].record(stream)
        e2e_step()
        ev2[k][1].record(stream)
    torch.cuda.synchronize()
    e2e_value, ms2 = job_throughput(args.steps * W["sweeps"], sum(a.elapsed_time(b) for a, b in ev2), dev)

    # ---- the plain FP64 GPU path on the same workload, same protocol ----
    compare = None
    o64 = None
    nst = min(args.steps, 3)  # the FP64 path is timed on fewer steps (it is the slow arm)
    if precision != "fp64" and not args.no_compare:
        for _ in range(2):
            reset()
            api.thc_cpd_als(Xo, Xv, Z, A, lam, W["sweeps"], 0.0, precision="fp64", ldl=args.ldl)
        torch.cuda.synchronize()
        ev3 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(nst)]
        for k in range(nst):
            flush.zero_()
            reset()
            ev3[k][0].record(stream)
            o64 = api.thc_cpd_als(Xo, Xv, Z, A, lam, W["sweeps"], 0.0, precision="fp64", ldl=args.ldl)
            ev3[k][1].record(stream)
        torch.cuda.synchronize()
        v64, ms3 = job_throughput(nst * W["sweeps"], sum(a.elapsed_time(b) for a, b in ev3), dev)
        compare = {"fp64": {"value": v64, "fit": o64["fit"], "ms_per_step": ms3 / nst},
                   precision: {"value": value, "fit": fit, "ms_per_step": ms / args.steps},
                   "speedup_vs_fp64": value / v64,
                   "fit_diff_vs_fp64": fit - o64["fit"],
                   "note": "equal sweep count; both fits are exact FP64 losses of the returned factors"}

    # ---- equal fit: wall-time of each form to the FP64 run's fit after the step's sweeps ----
    equal_fit = None
    if precision != "fp64" and o64 is not None and not args.no_equal_fit and world == 1:
        from paper_2502_17683_gb300 import learned
        target = o64["fit"]
        rows = {"fp64": {"sweeps": W["sweeps"], "seconds": ms3 / nst / 1000.0, "fit": o64["fit"]}}
        arms = [(precision, None, 5), (precision + "+learned", learned.load_params(), 0)]
        for name, mlp, every in arms:
            reset()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = api.thc_cpd_als(Xo, Xv, Z, A, lam, 4 * W["sweeps"], 0.0, precision=precision,
                                mlp=mlp, loss_every=every, target_fit=target, ldl=args.ldl)
            e1.record(stream)
            torch.cuda.synchronize()
            rows[name] = {"sweeps": r["sweeps"], "seconds": e0.elapsed_time(e1) / 1000.0,
                          "fit": r["fit"], "reached": r["fit"] >= target}
            if mlp is not None:
                rows[name]["accepted_steps"] = r["accepted"]
        equal_fit = {"target_fit": target,
                     "target": f"the FP64 run's fit after {W['sweeps']} sweeps from the same start",
                     "rows": rows,
                     "speedup_vs_fp64": {k: rows["fp64"]["seconds"] / v["seconds"]
                                         for k, v in rows.items() if k != "fp64"},
                     "note": "split runs evaluate the exact FP64 loss every 5 sweeps (learned: every "
                             "sweep, its accept rule needs it) and stop at the first evaluated sweep "
                             "whose fit reaches the target; seconds by CUDA events around the call"}

    # ---- roofline: per-kernel-class CUDA events over one more profiled step ----
    pk, pk_kind = peaks()
    f64pk = fp64_peaks(dev, clk.summary().get("sm_max_mhz"))
    # the factorisation a single problem gets (thc_cpd_opts.ldl = auto): dataflow up to R = 2048
    reset()
    api.thc_cpd_profile(True)
    step()
    torch.cuda.synchronize()
    prof = api.thc_cpd_profile_read()
    api.thc_cpd_profile(False)
    # the factorisation that ran (thc_cpd_opts.ldl = auto decides by the problem's order)
    if args.ldl != "auto":
        ldl_path = args.ldl
    elif prof.get("tc_emulated", {"ms": 0.0})["ms"] > 0:
        ldl_path = "emulated"
    else:
        ldl_path = "dataflow" if W["R"] <= 2048 else "blocked"
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    achieved = d["flops"] / (d["ms"] / 1000.0) / 1e12 if d["ms"] > 0 else 0.0
    # the LDL^T is one launch per solve on the dataflow path; per launch = per solve
    kernel = {"cholesky": "k_ldl_flow (LDL^T + forward solve, one launch per mode)"
              if ldl_path == "dataflow" else
              ("k_ldl_flow panels of the emulated two-level LDL^T (one launch per 256 columns, one for the last 520)"
               if ldl_path == "emulated" else "blocked LDL^T launches (per mode)"),
              "backward_solve": "k_bsolve_slices", "fp64_gemm": "k_dgemm",
              "tc_gemm": "k_tc_gemm", "tc_zgemm": "k_tc_gemm (Z contraction)",
              "elementwise": "element-wise kernels",
              "tc_emulated": "k_oz_split + k_oz_update (emulated FP64 products)"}[dom]
    traffic = None
    if dom == "tc_gemm":
        bound, peak = "tensor", pk["bf16_tflops_sustained"]
        note = "bf16 sustained, " + pk_kind
    elif dom == "tc_emulated":
        # FP64-equivalent work; the tensor cores issue 28 BF16 products per FP64 product
        bound, peak = "tensor", pk["bf16_tflops_sustained"] / 28.0
        note = "bf16 sustained / 28 (slice products per emulated FP64 product), " + pk_kind
    elif dom == "elementwise":
        bound, peak, note = "hbm", None, pk_kind
    else:
        bound, peak = "alu", f64pk["probe_tflops"]
        note = (f"measured FP64 FMA rate (library probe kernel); cuBLAS DGEMM measures "
                f"{f64pk['dgemm_tflops']:.3f}, the unit counts give {f64pk['nsm']} SMs x 2 FMA/clk "
                f"x 2 flop x {f64pk['sm_max_mhz']:.0f} MHz = {f64pk['derived_tflops']:.3f}")
        if dom == "cholesky":
            traffic = ldl_traffic(args.config, ldl_path)  # the capture of this workload, if current
    roofline = {"bound": bound, "kernel": kernel, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": (achieved / peak) if peak else None,
                "traffic": traffic, "peak_source": note,
                "fp64_peaks": {k: (round(v, 4) if isinstance(v, float) else v)
                               for k, v in f64pk.items()},
                "frac_of_dgemm": (achieved / f64pk["dgemm_tflops"]) if bound == "alu" else None,
                "frac_of_derived": (achieved / f64pk["derived_tflops"]) if bound == "alu" else None,
                "classes_ms_per_step": {k: round(v["ms"], 3) for k, v in prof.items()}}
    te = prof.get("tc_emulated", {"ms": 0.0})
    if te["ms"] > 0:
        useful = te["flops"] / (te["ms"] / 1000.0) / 1e12
        roofline["emulated_fp64_products"] = {
            "fp64_equivalent_tflops": useful, "issued_bf16_tflops": 28.0 * useful,
            "frac_issued": 28.0 * useful / pk["bf16_tflops_sustained"],
            "vs_fp64_probe": useful / f64pk["probe_tflops"],
            "note": "k_oz_split + k_oz_update: Grams and LDL^T trailing updates as exact "
                    "integer-digit products (7 x 7 slices, 28 kept) on the BF16 tensor cores"}
    # the split MTTKRP: projections and back-projections (tc_gemm) and the Z contraction
    # (tc_zgemm), together and the Z contraction alone
    tcp = prof.get("tc_gemm", {"ms": 0.0, "flops": 0.0})
    tcz = prof.get("tc_zgemm", {"ms": 0.0, "flops": 0.0})
    if tcp["ms"] + tcz["ms"] > 0:
        pk16 = pk["bf16_tflops_sustained"]
        issued_peak = pk16 if precision == "bf16x3" else pk16 * NOMINAL["tf32"] / NOMINAL["bf16"]
        ms_all, fl_all = tcp["ms"] + tcz["ms"], tcp["flops"] + tcz["flops"]
        useful = fl_all / (ms_all / 1000.0) / 1e12
        roofline["mttkrp_tensor_core"] = {
            "useful_tflops": useful, "issued_tflops": 3.0 * useful, "peak": issued_peak,
            "frac_issued": 3.0 * useful / issued_peak,
            "peak_source": f"{pk_kind} bf16 sustained" + ("" if precision == "bf16x3" else
                                                          " x nominal tf32/bf16 ratio")}
        if tcz["ms"] > 0:
            uz = tcz["flops"] / (tcz["ms"] / 1000.0) / 1e12
            roofline["mttkrp_tensor_core"]["z_contraction"] = {
                "useful_tflops": uz, "issued_tflops": 3.0 * uz, "frac_issued": 3.0 * uz / issued_peak,
                "ms_per_sweep": tcz["ms"] / W["sweeps"],
                "note": "Y = Z (W o W) on the tensor cores, 2 R_thc^2 R_cp flop per launch, two per sweep"}

    line = {
        "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if precision == "fp64" else f"{precision}+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "o": W["o"], "v": W["v"], "R_thc": W["Rt"],
                   "R_cp": W["R"], "sweeps_per_step": W["sweeps"], "precision": precision,
                   "ldl": ldl_path,
                   "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{world}"},
        "fit": fit,
        "clocks": clk.summary(),
        "e2e": {"value": e2e_value, "unit": "sweeps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roofline,
    }
    if compare:
        line["compare"] = compare
    if equal_fit:
        line["equal_fit"] = equal_fit
    if rank == 0 and not args.no_cpu_baseline:
        v, n, dt = oracle_sweeps_per_s(args.cpu_seconds, W["seed"])
        line["cpu_baseline"] = {"value": v, "unit": "sweeps/s", "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": f"{n} sweeps of the same workload ({dt:.1f} s), "
                                          "numpy/OpenBLAS FP64, default thread count"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
