import numpy as np


def to_dev(p, torch, device="cuda"):
    """THCProblem -> dict of contiguous float64 device tensors (A as a list)."""
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(device)
    return dict(Xo=t(p.Xo), Xv=t(p.Xv), Z=t(p.Z), A=[t(a) for a in p.A])


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def sample_cpd_entries(A, lam, idx):
    A1, A2, A3, A4 = A
    i, a, j, b = idx
    return np.einsum("r,nr,nr,nr,nr->n", lam, A1[i], A2[a], A3[j], A4[b])


def sample_idx(dims, n, seed):
    rng = np.random.default_rng(seed)
    return tuple(rng.integers(0, d, n) for d in dims)
