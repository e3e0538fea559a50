"""GB300-native THC-driven matrix-free CP-ALS (arXiv 2502.17683).

The compute path is the CUDA library libthc_cpd.so (C ABI in include/thc_cpd.h);
this package only builds it and marshals torch tensors into it.
"""
from ._lib import PRECISIONS, ThcCpdError, load  # noqa: F401


def __getattr__(name):
    if name.startswith("thc_cpd_"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
