"""Thin Python binding of the C ABI (include/thc_cpd.h) over torch CUDA tensors.

Functions carry the C names and only marshal arguments: every step of the method runs
in the library's CUDA kernels. Tensors must be contiguous float64 tensors on one CUDA
device; factor tensors are updated in place where the C ABI says so.
"""
from __future__ import annotations

import ctypes

import torch

from ._lib import (ERR_ARG, KCLASS_NAMES, LDL_VARIANTS, MLP_NPARAM, PRECISIONS, PTR4, KStat,
                   Opts, Problem, ThcCpdError, check, load)

__all__ = ["thc_cpd_thc_norm2", "thc_cpd_mttkrp", "thc_cpd_loss", "thc_cpd_als_sweep",
           "thc_cpd_als", "thc_cpd_version", "thc_cpd_launch_count", "thc_cpd_profile",
           "thc_cpd_profile_read", "thc_cpd_split_gemm", "thc_cpd_mttkrp_noalloc",
           "thc_cpd_als_batched", "thc_cpd_mlp_init", "thc_cpd_mlp_forward", "thc_cpd_mlp_grad",
           "thc_cpd_mlp_train", "thc_cpd_als_trajectory", "thc_cpd_ldl_solve", "thc_cpd_mlp_adam", "thc_cpd_fp64_fma_rate",
           "thc_cpd_emulated_gemm", "thc_cpd_exchange", "thc_cpd_core_fit", "thc_cpd_df_als", "thc_cpd_nd_mttkrp", "thc_cpd_nd_als", "Opts"]


def _dev(t: torch.Tensor, name: str, shape=None) -> int:
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
        raise ThcCpdError(ERR_ARG, f"{name} must be a float64 CUDA tensor")
    if not t.is_contiguous():
        raise ThcCpdError(ERR_ARG, f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ThcCpdError(ERR_ARG, f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


def _fdev(t: torch.Tensor, name: str, shape=None) -> int:
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_cuda:
        raise ThcCpdError(ERR_ARG, f"{name} must be a float32 CUDA tensor")
    if not t.is_contiguous():
        raise ThcCpdError(ERR_ARG, f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ThcCpdError(ERR_ARG, f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


def _opts(precision="fp64", stream=None, loss_every=0, history=None, polish_sweeps=0,
          autotune=False, ldl="auto", wait_limit_s=0.0) -> Opts:
    o = Opts()
    o.wait_limit_s = float(wait_limit_s)
    if ldl not in LDL_VARIANTS:
        raise ThcCpdError(ERR_ARG, f"unknown ldl variant {ldl!r}")
    o.ldl = LDL_VARIANTS[ldl]
    o.polish_sweeps = int(polish_sweeps)
    o.autotune = 1 if autotune else 0
    if isinstance(precision, str):
        if precision not in PRECISIONS:
            raise ThcCpdError(ERR_ARG, f"unknown precision {precision!r}")
        precision = PRECISIONS[precision]
    o.precision = int(precision)
    o.loss_every = int(loss_every)
    if stream is None:
        stream = torch.cuda.current_stream()
    o.stream = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    o.history = history
    return o


def _dims(Xo, Xv, Z):
    o, Rt = Xo.shape
    v = Xv.shape[0]
    return o, v, Rt


def _ptr4(A, dims, R):
    if len(A) != 4:
        raise ThcCpdError(ERR_ARG, "A must hold four factor matrices")
    return PTR4(*[_dev(a, f"A[{k}]", (dims[k], R)) for k, a in enumerate(A)])


def thc_cpd_exchange(Xo, Xv, Z, A, lam, Lam, Gam, emulated=False, stream=None):
    """CPD+THC LT-MP2 exchange energies (single, double, robust) for the Laplace factors Lam
    (n_alpha x o) and Gam (n_alpha x v); emulated: FP64-accurate tensor-core products."""
    o, v, Rt = _dims(Xo, Xv, Z)
    R = A[0].shape[1]
    na = Lam.shape[0]
    opts = _opts("fp64", stream, ldl="emulated" if emulated else "auto")
    e1, e2, er = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    check(load().thc_cpd_exchange(o, v, Rt, R, na, _dev(Xo, "Xo", (o, Rt)), _dev(Xv, "Xv", (v, Rt)),
                                  _dev(Z, "Z", (Rt, Rt)), _ptr4(A, (o, v, o, v), R),
                                  _dev(lam, "lam", (R,)), _dev(Lam, "Lam", (na, o)),
                                  _dev(Gam, "Gam", (na, v)), ctypes.byref(e1), ctypes.byref(e2),
                                  ctypes.byref(er), ctypes.byref(opts)))
    return e1.value, e2.value, er.value


def thc_cpd_core_fit(Xo, Xv, B, Z=None, loss=False, emulated=False, stream=None):
    """THC core least-squares fit: Z (R_thc x R_thc) from the grid factors Xo (o x R_thc),
    Xv (v x R_thc) and the DF tensor B (naux x o x v). Returns (Z, loss or None, used_pinv);
    emulated: FP64-accurate tensor-core products and the emulated two-level LDL^T."""
    o, Rt = Xo.shape
    v = Xv.shape[0]
    naux = B.shape[0]
    if Z is None:
        Z = torch.empty(Rt, Rt, dtype=torch.float64, device=Xo.device)
    opts = _opts("fp64", stream, ldl="emulated" if emulated else "auto")
    lv, pinv = ctypes.c_double(), ctypes.c_int()
    check(load().thc_cpd_core_fit(o, v, Rt, naux, _dev(Xo, "Xo", (o, Rt)), _dev(Xv, "Xv", (v, Rt)),
                                  _dev(B, "B", (naux, o, v)), _dev(Z, "Z", (Rt, Rt)),
                                  ctypes.byref(lv) if loss else None, ctypes.byref(pinv),
                                  ctypes.byref(opts)))
    return Z, (lv.value if loss else None), bool(pinv.value)


def thc_cpd_emulated_gemm(A, B, C=None, stream=None):
    """C = A @ B.T to FP64 accuracy on the BF16 tensor cores (exact integer slices)."""
    M, K = A.shape
    N = B.shape[0]
    if C is None:
        C = torch.empty(M, N, dtype=torch.float64, device=A.device)
    opts = _opts("fp64", stream)
    check(load().thc_cpd_emulated_gemm(M, N, K, _dev(A, "A"), K, _dev(B, "B", (N, K)), K,
                                       _dev(C, "C", (M, N)), N, ctypes.byref(opts)))
    return C


def thc_cpd_ldl_solve(H, M, A=None, tasks=None, wait_limit_s=0.0, stream=None, ldl="auto"):
    """A with A H = M (H: R x R SPD, M: n x R) by the library's dataflow LDL^T and backward
    solve, pseudo-inverse on a failed pivot. tasks: None (the library's schedule) or an
    int16 array of shape (ntasks, 4) in the format of thc_cpd_ldl_schedule. Returns
    (A, used_pinv)."""
    R = H.shape[0]
    n = M.shape[0]
    if A is None:
        A = torch.empty(n, R, dtype=torch.float64, device=H.device)
    opts = _opts("fp64", stream, wait_limit_s=wait_limit_s, ldl=ldl)
    used = ctypes.c_int(0)
    tp, nt = None, 0
    if tasks is not None:
        import numpy as np
        tasks = np.ascontiguousarray(tasks, dtype=np.int16).reshape(-1, 4)
        tp, nt = tasks.ctypes.data_as(ctypes.POINTER(ctypes.c_short)), int(tasks.shape[0])
    check(load().thc_cpd_ldl_solve(R, n, _dev(H, "H", (R, R)), _dev(M, "M", (n, R)),
                                   _dev(A, "A", (n, R)), tp, nt, ctypes.byref(used),
                                   ctypes.byref(opts)))
    return A, bool(used.value)


def thc_cpd_fp64_fma_rate(stream=None) -> float:
    """Measured FP64 FMA throughput of the current device in TFLOP/s (probe kernel)."""
    out = ctypes.c_double()
    opts = _opts("fp64", stream)
    check(load().thc_cpd_fp64_fma_rate(ctypes.byref(out), ctypes.byref(opts)))
    return out.value


def thc_cpd_version() -> str:
    return load().thc_cpd_version().decode()


def thc_cpd_thc_norm2(Xo, Xv, Z, stream=None) -> float:
    o, v, Rt = _dims(Xo, Xv, Z)
    out = ctypes.c_double()
    opts = _opts("fp64", stream)
    check(load().thc_cpd_thc_norm2(o, v, Rt, _dev(Xo, "Xo", (o, Rt)), _dev(Xv, "Xv", (v, Rt)),
                                   _dev(Z, "Z", (Rt, Rt)), ctypes.byref(out), ctypes.byref(opts)))
    return out.value


def thc_cpd_mttkrp(Xo, Xv, Z, A, mode: int, M=None, precision="fp64", stream=None):
    o, v, Rt = _dims(Xo, Xv, Z)
    R = A[0].shape[1]
    dims = (o, v, o, v)
    if M is None:
        M = torch.empty(dims[mode] if 0 <= mode < 4 else 1, R, dtype=torch.float64, device=Xo.device)
    opts = _opts(precision, stream)
    check(load().thc_cpd_mttkrp(o, v, Rt, R, _dev(Xo, "Xo", (o, Rt)), _dev(Xv, "Xv", (v, Rt)),
                                _dev(Z, "Z", (Rt, Rt)), _ptr4(A, dims, R), int(mode),
                                _dev(M, "M"), ctypes.byref(opts)))
    return M


def thc_cpd_mttkrp_noalloc(Xo, Xv, Z, A, mode: int, M, stream=None):
    """thc_cpd_mttkrp (FP64) with the library's fixed scratch array instead of any device
    allocation; M must be provided by the caller. Only enqueues work on the stream."""
    o, v, Rt = _dims(Xo, Xv, Z)
    R = A[0].shape[1]
    dims = (o, v, o, v)
    opts = _opts("fp64", stream)
    check(load().thc_cpd_mttkrp_noalloc(o, v, Rt, R, _dev(Xo, "Xo", (o, Rt)), _dev(Xv, "Xv", (v, Rt)),
                                        _dev(Z, "Z", (Rt, Rt)), _ptr4(A, dims, R), int(mode),
                                        _dev(M, "M"), ctypes.byref(opts)))
    return M


def thc_cpd_loss(Xo, Xv, Z, A, lam=None, normG2: float = 0.0, stream=None):
    o, v, Rt = _dims(Xo, Xv, Z)
    R = A[0].shape[1]
    loss, fit = ctypes.c_double(), ctypes.c_double()
    opts = _opts("fp64", stream)
    lp = None if lam is None else _dev(lam, "lam", (R,))
    check(load().thc_cpd_loss(o, v, Rt, R, _dev(Xo, "Xo", (o, Rt)), _dev(Xv, "Xv", (v, Rt)),
                              _dev(Z, "Z", (Rt, Rt)), _ptr4(A, (o, v, o, v), R), lp,
                              float(normG2), ctypes.byref(loss), ctypes.byref(fit),
                              ctypes.byref(opts)))
    return loss.value, fit.value


def thc_cpd_als_sweep(Xo, Xv, Z, A, lam, normG2: float = 0.0, precision="fp64", stream=None,
                      ldl="auto"):
    o, v, Rt = _dims(Xo, Xv, Z)
    R = A[0].shape[1]
    loss, fit = ctypes.c_double(), ctypes.c_double()
    opts = _opts(precision, stream, ldl=ldl)
    check(load().thc_cpd_als_sweep(o, v, Rt, R, _dev(Xo, "Xo", (o, Rt)), _dev(Xv, "Xv", (v, Rt)),
                                   _dev(Z, "Z", (Rt, Rt)), _ptr4(A, (o, v, o, v), R),
                                   _dev(lam, "lam", (R,)), float(normG2), ctypes.byref(loss),
                                   ctypes.byref(fit), ctypes.byref(opts)))
    return dict(loss=loss.value, fit=fit.value, flags=opts.flags_out)


def thc_cpd_als(Xo, Xv, Z, A, lam, max_sweeps: int, tol: float = 0.0, precision="fp64",
                stream=None, loss_every: int = 0, history: bool = False, polish_sweeps: int = 0,
                autotune: bool = False, mlp=None, ldl="auto", target_fit: float = 0.0):
    o, v, Rt = _dims(Xo, Xv, Z)
    R = A[0].shape[1]
    loss, fit, done = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    hist = (ctypes.c_double * max(1, 2 * max_sweeps))() if history else None
    opts = _opts(precision, stream, loss_every,
                 ctypes.cast(hist, ctypes.POINTER(ctypes.c_double)) if hist is not None else None,
                 polish_sweeps, autotune, ldl)
    opts.target_fit = float(target_fit)
    if mlp is not None:
        opts.mlp = _fdev(mlp, "mlp", (MLP_NPARAM,))
    check(load().thc_cpd_als(o, v, Rt, R, _dev(Xo, "Xo", (o, Rt)), _dev(Xv, "Xv", (v, Rt)),
                             _dev(Z, "Z", (Rt, Rt)), _ptr4(A, (o, v, o, v), R),
                             _dev(lam, "lam", (R,)), int(max_sweeps), float(tol),
                             ctypes.byref(done), ctypes.byref(loss), ctypes.byref(fit),
                             ctypes.byref(opts)))
    out = dict(sweeps=done.value, loss=loss.value, fit=fit.value, flags=opts.flags_out,
               accepted=opts.accepted_out)
    if hist is not None:
        h = list(hist)[: 2 * done.value]
        out["losses"] = h[0::2]
        out["fits"] = h[1::2]
    return out


def thc_cpd_df_als(B, A, lam, max_sweeps: int, tol: float = 0.0, emulated=False, history=False,
                   stream=None):
    """DF-driven CP-ALS of G_DF = sum_X B[X] (x) B[X] (B: naux x o x v); A (four factors) and lam
    are updated in place. emulated: FP64-accurate tensor-core GEMMs and the emulated LDL^T."""
    naux, o, v = B.shape
    R = A[0].shape[1]
    fit, done = ctypes.c_double(), ctypes.c_int()
    hist = (ctypes.c_double * max(1, 2 * max_sweeps))() if history else None
    opts = _opts("fp64", stream, 0,
                 ctypes.cast(hist, ctypes.POINTER(ctypes.c_double)) if hist is not None else None,
                 ldl="emulated" if emulated else "auto")
    check(load().thc_cpd_df_als(o, v, naux, R, _dev(B, "B", (naux, o, v)), _ptr4(A, (o, v, o, v), R),
                                _dev(lam, "lam", (R,)), int(max_sweeps), float(tol),
                                ctypes.byref(done), ctypes.byref(fit), ctypes.byref(opts)))
    out = dict(sweeps=done.value, fit=fit.value, flags=opts.flags_out)
    if hist is not None:
        h = list(hist)[: 2 * done.value]
        out["losses"] = h[0::2]
        out["fits"] = h[1::2]
    return out


def _nd_args(X, Z, A, dL):
    d = len(X)
    if len(A) != d:
        raise ThcCpdError(ERR_ARG, "X and A must hold the same number of modes")
    Rt = Z.shape[0]
    R = A[0].shape[1]
    dims = (ctypes.c_int * d)(*[int(x.shape[0]) for x in X])
    xs = (ctypes.c_void_p * d)(*[_dev(x, f"X[{k}]", (x.shape[0], Rt)) for k, x in enumerate(X)])
    As = (ctypes.c_void_p * d)(*[_dev(a, f"A[{k}]", (X[k].shape[0], R)) for k, a in enumerate(A)])
    return d, int(dL), dims, Rt, R, xs, _dev(Z, "Z", (Rt, Rt)), As


def thc_cpd_nd_mttkrp(X, Z, A, dL: int, mode: int, M=None, emulated=False, stream=None):
    """Order-d MTTKRP of the THC-like tensor (X: d grid factors, modes < dL on P, the rest on Q)."""
    d, dL, dims, Rt, R, xs, z, As = _nd_args(X, Z, A, dL)
    if M is None:
        M = torch.empty(X[mode].shape[0] if 0 <= mode < d else 1, R, dtype=torch.float64, device=Z.device)
    opts = _opts("fp64", stream, ldl="emulated" if emulated else "auto")
    check(load().thc_cpd_nd_mttkrp(d, dL, dims, Rt, R, xs, z, As, int(mode), _dev(M, "M"),
                                   ctypes.byref(opts)))
    return M


def thc_cpd_nd_als(X, Z, A, lam, dL: int, max_sweeps: int, tol: float = 0.0, emulated=False,
                   history=False, stream=None):
    """Order-d THC-driven CP-ALS; A (d factors) and lam are updated in place."""
    d, dL, dims, Rt, R, xs, z, As = _nd_args(X, Z, A, dL)
    fit, done = ctypes.c_double(), ctypes.c_int()
    hist = (ctypes.c_double * max(1, 2 * max_sweeps))() if history else None
    opts = _opts("fp64", stream, 0,
                 ctypes.cast(hist, ctypes.POINTER(ctypes.c_double)) if hist is not None else None,
                 ldl="emulated" if emulated else "auto")
    check(load().thc_cpd_nd_als(d, dL, dims, Rt, R, xs, z, As, _dev(lam, "lam", (R,)), int(max_sweeps),
                                float(tol), ctypes.byref(done), ctypes.byref(fit), ctypes.byref(opts)))
    out = dict(sweeps=done.value, fit=fit.value, flags=opts.flags_out)
    if hist is not None:
        h = list(hist)[: 2 * done.value]
        out["losses"] = h[0::2]
        out["fits"] = h[1::2]
    return out


def thc_cpd_split_gemm(A, B, precision="bf16x3", C=None, stream=None):
    """C = A @ B.T on the tensor cores with split operands (FP64 in and out)."""
    M, K = A.shape
    N = B.shape[0]
    if C is None:
        C = torch.empty(M, N, dtype=torch.float64, device=A.device)
    opts = _opts(precision, stream)
    check(load().thc_cpd_split_gemm(M, N, K, _dev(A, "A"), _dev(B, "B", (N, K)), _dev(C, "C", (M, N)),
                                    ctypes.byref(opts)))
    return C


def thc_cpd_ldl_schedule(R: int, n: int):
    """Ticket-ordered task list of the dataflow LDL^T for R x R with n appended rows, as a
    list of (type, t, j, k) tuples (type 0: substitution S(t, k); 1: update U(t, j, k)).
    Host only. Raises if the shape is outside the dataflow path or the order fails its
    check."""
    lib = load()
    cnt = lib.thc_cpd_ldl_schedule(int(R), int(n), None, 0)
    if cnt < 0:
        raise ThcCpdError(ERR_ARG, f"no dataflow schedule for R={R} n={n}")
    buf = (ctypes.c_short * (4 * max(cnt, 1)))()
    got = lib.thc_cpd_ldl_schedule(int(R), int(n), buf, cnt)
    if got != cnt:
        raise ThcCpdError(ERR_ARG, "schedule size changed between calls")
    return [tuple(buf[4 * i:4 * i + 4]) for i in range(cnt)]


def thc_cpd_launch_count() -> int:
    return int(load().thc_cpd_launch_count())


def thc_cpd_profile(enable: bool) -> None:
    load().thc_cpd_profile(1 if enable else 0)


def thc_cpd_profile_read() -> dict:
    """Per kernel class: dict(ms, flops, bytes, groups) summed over recorded groups."""
    n = len(KCLASS_NAMES)
    buf = (KStat * n)()
    got = load().thc_cpd_profile_read(buf, n)
    if got < 0:
        raise ThcCpdError(3, "profile read failed")
    return {KCLASS_NAMES[i]: dict(ms=buf[i].ms, flops=buf[i].flops, bytes=buf[i].bytes,
                                  groups=buf[i].groups) for i in range(got)}


def thc_cpd_als_batched(problems, max_sweeps: int, tol: float = 0.0, precision="fp64",
                        stream=None, autotune: bool = False, ldl="auto"):
    """problems: list of dicts with Xo, Xv, Z, A (list of 4), lam (device tensors, updated in
    place). Returns a list of dict(sweeps, loss, fit, flags) per problem."""
    n = len(problems)
    arr = (Problem * max(1, n))()
    for i, pr in enumerate(problems):
        o, v, Rt = _dims(pr["Xo"], pr["Xv"], pr["Z"])
        R = pr["A"][0].shape[1]
        arr[i].o, arr[i].v, arr[i].Rt, arr[i].R = o, v, Rt, R
        arr[i].Xo = _dev(pr["Xo"], "Xo", (o, Rt))
        arr[i].Xv = _dev(pr["Xv"], "Xv", (v, Rt))
        arr[i].Z = _dev(pr["Z"], "Z", (Rt, Rt))
        for k, a in enumerate(pr["A"]):
            arr[i].A[k] = _dev(a, f"A[{k}]", ((o, v, o, v)[k], R))
        arr[i].lam = _dev(pr["lam"], "lam", (R,))
    opts = _opts(precision, stream, autotune=autotune, ldl=ldl)
    check(load().thc_cpd_als_batched(n, ctypes.cast(arr, ctypes.c_void_p), int(max_sweeps),
                                     float(tol), ctypes.byref(opts)))
    return [dict(sweeps=arr[i].sweeps_done, loss=arr[i].loss, fit=arr[i].fit, flags=arr[i].flags_out)
            for i in range(n)]


def thc_cpd_mlp_init(seed: int = 0, params=None, stream=None):
    if params is None:
        params = torch.empty(MLP_NPARAM, dtype=torch.float32, device="cuda")
    opts = _opts("fp64", stream)
    check(load().thc_cpd_mlp_init(_fdev(params, "params", (MLP_NPARAM,)), int(seed), ctypes.byref(opts)))
    return params


def thc_cpd_mlp_forward(params, X, stream=None):
    n = X.shape[0]
    alpha = torch.empty(n, dtype=torch.float32, device=X.device)
    opts = _opts("fp64", stream)
    check(load().thc_cpd_mlp_forward(_fdev(params, "params", (MLP_NPARAM,)), _fdev(X, "X", (n, 40)),
                                     n, _fdev(alpha, "alpha"), ctypes.byref(opts)))
    return alpha


def thc_cpd_mlp_grad(params, X, y, stream=None):
    n = X.shape[0]
    grad = torch.empty(MLP_NPARAM, dtype=torch.float32, device=X.device)
    loss = ctypes.c_float()
    opts = _opts("fp64", stream)
    check(load().thc_cpd_mlp_grad(_fdev(params, "params", (MLP_NPARAM,)), _fdev(X, "X", (n, 40)),
                                  _fdev(y, "y", (n,)), n, _fdev(grad, "grad"), ctypes.byref(loss),
                                  ctypes.byref(opts)))
    return grad, loss.value


def thc_cpd_mlp_adam(params, grad, m, v, t: int, lr: float = 1e-3, stream=None):
    """One Adam update of params (and the moments m, v) in place, as thc_cpd_mlp_train
    applies it after each batch."""
    opts = _opts("fp64", stream)
    check(load().thc_cpd_mlp_adam(_fdev(params, "params", (MLP_NPARAM,)),
                                  _fdev(grad, "grad", (MLP_NPARAM,)), _fdev(m, "m", (MLP_NPARAM,)),
                                  _fdev(v, "v", (MLP_NPARAM,)), int(t), float(lr),
                                  ctypes.byref(opts)))


def thc_cpd_mlp_train(params, X, y, epochs: int, batch: int = 64, lr: float = 1e-3, seed: int = 0,
                      stream=None) -> float:
    n = X.shape[0]
    loss = ctypes.c_float()
    opts = _opts("fp64", stream)
    check(load().thc_cpd_mlp_train(_fdev(params, "params", (MLP_NPARAM,)), _fdev(X, "X", (n, 40)),
                                   _fdev(y, "y", (n,)), n, int(epochs), int(batch), float(lr),
                                   int(seed), ctypes.byref(loss), ctypes.byref(opts)))
    return loss.value


def thc_cpd_als_trajectory(Xo, Xv, Z, A, lam, sweeps: int, alphas, precision="fp64", stream=None,
                           ldl="auto"):
    """Plain ALS for `sweeps` sweeps, recording per sweep the 40 features and the exact losses
    of the trial points at each alpha. Returns (features (sweeps, 40), losses (sweeps, na))."""
    import numpy as np
    o, v, Rt = _dims(Xo, Xv, Z)
    R = A[0].shape[1]
    al = np.ascontiguousarray(np.asarray(alphas, dtype=np.float64))
    feats = np.zeros((sweeps, 40), dtype=np.float32)
    tl = np.zeros((sweeps, len(al)), dtype=np.float64)
    opts = _opts(precision, stream, ldl=ldl)
    check(load().thc_cpd_als_trajectory(
        o, v, Rt, R, _dev(Xo, "Xo", (o, Rt)), _dev(Xv, "Xv", (v, Rt)), _dev(Z, "Z", (Rt, Rt)),
        _ptr4(A, (o, v, o, v), R), _dev(lam, "lam", (R,)), int(sweeps),
        al.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(al),
        feats.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
        tl.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(opts)))
    return feats, tl
