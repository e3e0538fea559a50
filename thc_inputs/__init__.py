"""Seeded synthetic inputs for THC-driven CP-ALS.

This module is shared by the CPU oracle, the tests and the benchmark. It only draws
random numbers and assembles input arrays; it holds none of the method's arithmetic
(no MTTKRP, no solve, no loss).

The paper's molecules (water clusters, the L7 set) and their THC factors are not
available, so synthetic THC factors with the paper's shape conventions stand in:
v/o = 5 (a virtual space five times the occupied one) and THC / CP ranks that are
multiples of the orbital count N = o + v (Sec. 4, rank choices R = kX).

Generator recipe (all FP64, numpy PCG64, draw order fixed below):
  1. w_P = 10**U(-2, 0) for each grid point P (one weight per THC column,
     shared by Xo and Xv).
  2. Xo[i,P] = N(0,1)/sqrt(Rt) * w_P ,  Xv[a,P] = N(0,1)/sqrt(Rt) * w_P.
  3. Z = L diag(exp(-k/s)) L^T with L[P,k] = N(0,1)/sqrt(Rt), k = 0..Rt-1 and
     decay scale s (Rt/5 by default: 12 at Rt=60, 240 at Rt=1200).
  4. Initial CP factors A1 (o x R), A2 (v x R), A3 (o x R), A4 (v x R), N(0,1)
     (or U[-1,1], the initialisation of Sec. 3), drawn from a second stream so that
     the THC inputs do not depend on R.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class THCProblem:
    """One THC-factorised integral block G_iajb and its CP-ALS start point."""
    o: int
    v: int
    Rt: int
    R: int
    Xo: np.ndarray  # o x Rt
    Xv: np.ndarray  # v x Rt
    Z: np.ndarray   # Rt x Rt
    A: tuple        # (A1 o x R, A2 v x R, A3 o x R, A4 v x R)

    @property
    def dims(self):
        return (self.o, self.v, self.o, self.v)


def make_thc(o: int, v: int, Rt: int, seed: int, decay: float | None = None):
    """Synthetic THC factors (Xo, Xv, Z) following the recipe in the module docstring."""
    rng = np.random.default_rng([seed, 0x7C])
    s = Rt / 5.0 if decay is None else float(decay)
    w = 10.0 ** rng.uniform(-2.0, 0.0, size=Rt)
    scale = 1.0 / math.sqrt(Rt)
    Xo = rng.standard_normal((o, Rt)) * scale * w[None, :]
    Xv = rng.standard_normal((v, Rt)) * scale * w[None, :]
    L = rng.standard_normal((Rt, Rt)) * scale
    d = np.exp(-np.arange(Rt) / s)
    Z = (L * d[None, :]) @ L.T
    Z = 0.5 * (Z + Z.T)  # exactly symmetric bytes
    return Xo, Xv, Z


def make_factors(dims, R: int, seed: int, init: str = "normal"):
    """Initial CP factors for modes (i, a, j, b); N(0,1) or U[-1,1]."""
    rng = np.random.default_rng([seed, 0xA1])
    out = []
    for n in dims:
        if init == "normal":
            out.append(rng.standard_normal((n, R)))
        elif init == "uniform":
            out.append(rng.uniform(-1.0, 1.0, size=(n, R)))
        else:
            raise ValueError(f"unknown init {init!r}")
    return tuple(out)


def make_problem(o: int, v: int, Rt: int, R: int, seed: int = 0,
                 decay: float | None = None, init: str = "normal") -> THCProblem:
    Xo, Xv, Z = make_thc(o, v, Rt, seed, decay)
    A = make_factors((o, v, o, v), R, seed, init)
    return THCProblem(o, v, Rt, R, Xo, Xv, Z, A)


def make_planted(o: int, v: int, rank: int, R: int, seed: int = 0,
                 independent: bool = True) -> tuple[THCProblem, tuple]:
    """A THC block that is exactly a rank-`rank` CPD with N(0,1) factors.

    independent=True : Xo = [A1*|A3*], Xv = [A2*|A4*], Z = [[0, I], [0, 0]]
                       (Rt = 2*rank), so G = sum_r A1*_ir A2*_ar A3*_jr A4*_br.
    independent=False: Xo = A1*, Xv = A2*, Z = I (Rt = rank), the particle-symmetric
                       CPD G = sum_r A1*_ir A2*_ar A1*_jr A2*_br.
    Returns the problem (with random start factors of rank R) and the planted factors.
    """
    rng = np.random.default_rng([seed, 0x91])
    A1 = rng.standard_normal((o, rank))
    A2 = rng.standard_normal((v, rank))
    A3 = rng.standard_normal((o, rank))
    A4 = rng.standard_normal((v, rank))
    if independent:
        Xo = np.concatenate([A1, A3], axis=1)
        Xv = np.concatenate([A2, A4], axis=1)
        Z = np.zeros((2 * rank, 2 * rank))
        Z[:rank, rank:] = np.eye(rank)
        planted = (A1, A2, A3, A4)
    else:
        Xo, Xv, Z = A1, A2, np.eye(rank)
        planted = (A1, A2, A1, A2)
    A = make_factors((o, v, o, v), R, seed + 1000)
    Rt = Xo.shape[1]
    return THCProblem(o, v, Rt, R, Xo, Xv, Z, A), planted


def make_planted_noisy(o: int, v: int, rank: int, noise_rank: int = 24, noise_scale: float = 10.0,
                       seed: int = 0, start_perturb: float = 0.3) -> tuple[THCProblem, tuple]:
    """A planted rank-`rank` CPD plus a THC-shaped perturbation, so that the best rank-`rank`
    CPD is a fixed point of ALS that is not exact (fit below 1):

      Xo = [A1*|A3*|Eo], Xv = [A2*|A4*|Ev], Z = blockdiag([[0, I], [0, 0]], s L L^T / m)

    with Eo, Ev, L ~ N(0,1)/sqrt(m) (m = noise_rank, L m x m) and s = noise_scale. The start
    factors are the planted ones with each entry scaled by (1 + start_perturb N(0,1)), so
    that ALS converges to the fixed point near the planted CPD. R_cp = rank.
    Returns the problem and the planted factors."""
    base, planted = make_planted(o, v, rank, rank, seed=seed, independent=True)
    rng = np.random.default_rng([seed, 0x5E])
    m = noise_rank
    Eo = rng.standard_normal((o, m)) / math.sqrt(m)
    Ev = rng.standard_normal((v, m)) / math.sqrt(m)
    L = rng.standard_normal((m, m))
    Xo = np.concatenate([base.Xo, Eo], axis=1)
    Xv = np.concatenate([base.Xv, Ev], axis=1)
    Rt = Xo.shape[1]
    Z = np.zeros((Rt, Rt))
    Z[:base.Rt, :base.Rt] = base.Z
    Z[base.Rt:, base.Rt:] = noise_scale * (L @ L.T) / m
    A = tuple(a * (1.0 + start_perturb * rng.standard_normal(a.shape)) for a in planted)
    return THCProblem(o, v, Rt, rank, Xo, Xv, Z, A), planted


def make_lt(o: int, v: int, n_alpha: int = 12, seed: int = 0):
    """Synthetic orbital energies and a Laplace quadrature for the LT-MP2 exchange energy
    (Eq. lt_D): occupied eps ~ U(-2, -0.5), virtual eps ~ U(0.2, 3); n_alpha Gauss-Legendre
    points x on [-1, 1] mapped to [0, inf) by s = tau (1 + x) / (1 - x), weights times the
    Jacobian 2 tau / (1 - x)^2, tau = 1 / (2 gap), gap = min eps_vir - max eps_occ, so that
    sum w exp(-D s) ~ 1/D. The Gamma / Lambda factors of the paper carry exp(+-eps t / 2), so
    the four of them multiply to exp(-D t / 2): the points are returned as t = 2 s (weights
    unchanged). Returns (eps_occ, eps_vir, t, w). (The paper uses 12 Legendre points; the
    mapping is this build's choice.)"""
    rng = np.random.default_rng([seed, 0x17])
    eps_occ = np.sort(rng.uniform(-2.0, -0.5, size=o))
    eps_vir = np.sort(rng.uniform(0.2, 3.0, size=v))
    gap = float(np.min(eps_vir) - np.max(eps_occ))
    tau = 1.0 / (2.0 * gap)
    x, om = np.polynomial.legendre.leggauss(n_alpha)
    s_pts = tau * (1.0 + x) / (1.0 - x)
    w = om * 2.0 * tau / (1.0 - x) ** 2
    return eps_occ, eps_vir, 2.0 * s_pts, w


def make_df(o: int, v: int, Rt: int, naux: int, seed: int = 0, noise: float = 1e-2,
            decay: float | None = None):
    """A synthetic density-fitting tensor B (naux x o x v) and THC grid factors (Xo, Xv) for it,
    built the way the paper builds its THC factors from the DF tensor's order-3 CPD (Sec. 3):
      Xo, Xv from make_thc (the same draws, so the same grid factors as make_problem),
      C[X,P] = N(0,1) / sqrt(Rt),
      B[X,i,a] = sum_P C[X,P] Xo[i,P] Xv[a,P] + noise * rms(that sum) * N(0,1),
    i.e. an order-3 CPD of rank Rt plus a relative Gaussian perturbation, so that the
    (o,v,o,v) DF block is close to, but not exactly, a THC block on these factors.
    Returns (Xo, Xv, B). naux is the auxiliary-basis size (3-4 x (o + v) is typical of DF
    bases). The CPD assembly is input construction (np.einsum); it is none of the
    core fit's or of DF-driven CP-ALS's arithmetic."""
    Xo, Xv, _ = make_thc(o, v, Rt, seed, decay)
    rng = np.random.default_rng([seed, 0xDF])
    C = rng.standard_normal((naux, Rt)) / math.sqrt(Rt)
    B = np.einsum("xp,ip,ap->xia", C, Xo, Xv, optimize=True)
    rms = float(np.sqrt(np.mean(B * B))) if B.size else 0.0
    B = B + noise * rms * rng.standard_normal(B.shape)
    return Xo, Xv, np.ascontiguousarray(B)


def make_nd(dims, Rt: int, R: int, seed: int = 0, decay: float | None = None):
    """Order-d THC-like inputs: grid factors X_k (dims[k] x Rt) and a core Z (Rt x Rt) by the
    recipe of make_thc (one weight w_P per grid point shared by every X_k; Z = L diag(exp(-k/s))
    L^T), and start factors A_k (dims[k] x R) N(0,1). Returns (X list, Z, A tuple)."""
    rng = np.random.default_rng([seed, 0x4D])
    s = Rt / 5.0 if decay is None else float(decay)
    w = 10.0 ** rng.uniform(-2.0, 0.0, size=Rt)
    scale = 1.0 / math.sqrt(Rt)
    X = [rng.standard_normal((n, Rt)) * scale * w[None, :] for n in dims]
    L = rng.standard_normal((Rt, Rt)) * scale
    d = np.exp(-np.arange(Rt) / s)
    Z = (L * d[None, :]) @ L.T
    Z = 0.5 * (Z + Z.T)
    return X, Z, make_factors(tuple(dims), R, seed)


def round_up(x: int, m: int) -> int:
    return ((x + m - 1) // m) * m


def batched_shapes(nprob: int = 64, seed: int = 0, o_lo: int = 4, o_hi: int = 40):
    """Shapes of the batched workload: o ~ U{o_lo..o_hi}, v = 5o,
    Rt = 4(o+v) and R = 6(o+v), both rounded up to a multiple of 16."""
    rng = np.random.default_rng([seed, 0xB4])
    os_ = rng.integers(o_lo, o_hi + 1, size=nprob)
    out = []
    for o in os_:
        o = int(o)
        v = 5 * o
        out.append((o, v, round_up(4 * (o + v), 16), round_up(6 * (o + v), 16)))
    return out


# Named workloads (sizes from the paper-shaped configurations).
CONFIGS = {
    "c1": dict(o=5, v=15, Rt=60, R=80, sweeps=25),
    "c2": dict(o=20, v=100, Rt=480, R=720, sweeps=50),
    "c3": dict(o=50, v=250, Rt=1200, R=1800, sweeps=100, decay=240.0),
    "c5": dict(o=30, v=150, Rt=720, R=1080, sweeps=200),
}


def make_config(name: str, seed: int = 0) -> THCProblem:
    c = CONFIGS[name]
    return make_problem(c["o"], c["v"], c["Rt"], c["R"], seed, c.get("decay"))
