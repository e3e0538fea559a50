"""ctypes loader for the in-tree libthc_cpd.so (the C ABI of include/thc_cpd.h).

There is no fallback: if the library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libthc_cpd.so")

OK, ERR_ARG, ERR_SHAPE, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_ALLOC, ERR_UNSUPPORTED = range(8)
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_SHAPE", 3: "ERR_CUDA", 4: "ERR_NONFINITE",
                5: "ERR_TIMEOUT", 6: "ERR_ALLOC", 7: "ERR_UNSUPPORTED"}
PRECISIONS = {"fp64": 0, "bf16x3": 1, "tf32x3": 2}
LDL_VARIANTS = {"auto": 0, "blocked": 1, "dataflow": 2, "emulated": 3}

# every symbol include/thc_cpd.h declares
EXPORTS = ("thc_cpd_thc_norm2", "thc_cpd_mttkrp", "thc_cpd_loss", "thc_cpd_als_sweep",
           "thc_cpd_als", "thc_cpd_last_error", "thc_cpd_version", "thc_cpd_launch_count",
           "thc_cpd_profile", "thc_cpd_profile_read", "thc_cpd_split_gemm",
           "thc_cpd_mttkrp_noalloc", "thc_cpd_als_batched", "thc_cpd_mlp_init",
           "thc_cpd_mlp_forward", "thc_cpd_mlp_grad", "thc_cpd_mlp_train", "thc_cpd_als_trajectory",
           "thc_cpd_ldl_schedule", "thc_cpd_ldl_solve", "thc_cpd_mlp_adam",
           "thc_cpd_fp64_fma_rate", "thc_cpd_emulated_gemm", "thc_cpd_exchange",
           "thc_cpd_core_fit", "thc_cpd_df_als", "thc_cpd_nd_mttkrp", "thc_cpd_nd_als")
MLP_NPARAM = 6849
KCLASS_NAMES = ("fp64_gemm", "cholesky", "backward_solve", "elementwise", "tc_gemm", "tc_emulated",
                "tc_zgemm")


class ThcCpdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class KStat(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double), ("groups", ctypes.c_long)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int),
                ("loss_every", ctypes.c_int),
                ("stream", ctypes.c_void_p),
                ("history", ctypes.POINTER(ctypes.c_double)),
                ("flags_out", ctypes.c_int),
                ("polish_sweeps", ctypes.c_int),
                ("autotune", ctypes.c_int),
                ("accepted_out", ctypes.c_int),
                ("mlp", ctypes.c_void_p),
                ("ldl", ctypes.c_int),
                ("wait_limit_s", ctypes.c_double),
                ("target_fit", ctypes.c_double)]


class Problem(ctypes.Structure):
    _fields_ = [("o", ctypes.c_int), ("v", ctypes.c_int), ("Rt", ctypes.c_int), ("R", ctypes.c_int),
                ("Xo", ctypes.c_void_p), ("Xv", ctypes.c_void_p), ("Z", ctypes.c_void_p),
                ("A", ctypes.c_void_p * 4), ("lam", ctypes.c_void_p),
                ("sweeps_done", ctypes.c_int), ("flags_out", ctypes.c_int),
                ("loss", ctypes.c_double), ("fit", ctypes.c_double)]


P = ctypes.c_void_p
D = ctypes.c_double
I = ctypes.c_int
DP = ctypes.POINTER(ctypes.c_double)
IP = ctypes.POINTER(ctypes.c_int)
PTR4 = ctypes.c_void_p * 4
OPTS = ctypes.POINTER(Opts)

_SIGS = {
    "thc_cpd_thc_norm2": [I, I, I, P, P, P, DP, OPTS],
    "thc_cpd_mttkrp": [I, I, I, I, P, P, P, PTR4, I, P, OPTS],
    "thc_cpd_loss": [I, I, I, I, P, P, P, PTR4, P, D, DP, DP, OPTS],
    "thc_cpd_als_sweep": [I, I, I, I, P, P, P, PTR4, P, D, DP, DP, OPTS],
    "thc_cpd_als": [I, I, I, I, P, P, P, PTR4, P, I, D, IP, DP, DP, OPTS],
    "thc_cpd_split_gemm": [I, I, I, P, P, P, OPTS],
    "thc_cpd_mttkrp_noalloc": [I, I, I, I, P, P, P, PTR4, I, P, OPTS],
    "thc_cpd_als_batched": [I, ctypes.c_void_p, I, D, OPTS],
    "thc_cpd_mlp_init": [P, ctypes.c_ulonglong, OPTS],
    "thc_cpd_mlp_forward": [P, P, I, P, OPTS],
    "thc_cpd_mlp_grad": [P, P, P, I, P, ctypes.POINTER(ctypes.c_float), OPTS],
    "thc_cpd_fp64_fma_rate": [DP, OPTS],
    "thc_cpd_emulated_gemm": [I, I, I, P, I, P, I, P, I, OPTS],
    "thc_cpd_exchange": [I, I, I, I, I, P, P, P, PTR4, P, P, P, DP, DP, DP, OPTS],
    "thc_cpd_core_fit": [I, I, I, I, P, P, P, P, DP, IP, OPTS],
    "thc_cpd_df_als": [I, I, I, I, P, PTR4, P, I, D, IP, DP, OPTS],
    "thc_cpd_nd_mttkrp": [I, I, IP, I, I, P, P, P, I, P, OPTS],
    "thc_cpd_nd_als": [I, I, IP, I, I, P, P, P, P, I, D, IP, DP, OPTS],
    "thc_cpd_mlp_adam": [P, P, P, P, I, ctypes.c_float, OPTS],
    "thc_cpd_mlp_train": [P, P, P, I, I, I, ctypes.c_float, ctypes.c_ulonglong,
                          ctypes.POINTER(ctypes.c_float), OPTS],
    "thc_cpd_als_trajectory": [I, I, I, I, P, P, P, PTR4, P, I, DP, I,
                               ctypes.POINTER(ctypes.c_float), DP, OPTS],
    "thc_cpd_ldl_schedule": [I, I, ctypes.POINTER(ctypes.c_short), I],
    "thc_cpd_ldl_solve": [I, I, P, P, P, ctypes.POINTER(ctypes.c_short), I, IP, OPTS],
}

_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load (once) and return the library; raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ThcCpdError(ERR_UNSUPPORTED, f"{p} is not built; run __graft_entry__.build() or "
                                           "python -m paper_2502_17683_gb300.build")
    lib = ctypes.CDLL(p)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.thc_cpd_last_error.restype = ctypes.c_char_p
    lib.thc_cpd_last_error.argtypes = []
    lib.thc_cpd_version.restype = ctypes.c_char_p
    lib.thc_cpd_version.argtypes = []
    lib.thc_cpd_launch_count.restype = ctypes.c_long
    lib.thc_cpd_launch_count.argtypes = []
    lib.thc_cpd_profile.restype = None
    lib.thc_cpd_profile.argtypes = [ctypes.c_int]
    lib.thc_cpd_profile_read.restype = ctypes.c_int
    lib.thc_cpd_profile_read.argtypes = [ctypes.POINTER(KStat), ctypes.c_int]
    _lib = lib
    return lib


def check(status: int) -> None:
    if status != OK:
        msg = load().thc_cpd_last_error().decode(errors="replace")
        raise ThcCpdError(status, msg)
