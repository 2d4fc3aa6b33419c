"""Shared helpers of the GPU tests: build the library once, move a problem to
the device, run the oracle on the same seeded inputs."""
import numpy as np
import pytest

from oracle import hsolver as H


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_03189_gb300.build import build

    build()
    return torch


def to_dev(pb):
    import torch

    d = torch.device("cuda:0")
    return (torch.as_tensor(pb.rowptr, dtype=torch.int32, device=d),
            torch.as_tensor(pb.col, dtype=torch.int32, device=d),
            torch.as_tensor(pb.val, dtype=torch.float64, device=d))


def gpu_factor(pb, eps, variant, prec=0, phi=None):
    from paper_1611_03189_gb300 import _lib

    rp, ci, va = to_dev(pb)
    return _lib.Factor(rp, ci, va, pb.perm, pb.leaf_ptr, eps, variant, prec, phi)


def oracle_factor(pb, eps, variant, phi=None):
    return H.factor(pb.n, pb.rowptr, pb.col, pb.val, pb.perm, pb.leaf_ptr, eps, variant, phi=phi)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def elem(a, b):
    """Element-wise error of a against b, per right-hand side: the largest
    max_i |a_ij - b_ij| / max_i |b_ij| over the columns j (a vector is one
    column).  Unlike one global 2-norm ratio, a wrong block of a few entries
    cannot hide under the norm of the whole vector."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.shape != b.shape:
        raise ValueError(f"shapes differ: {a.shape} vs {b.shape}")
    if b.ndim == 1:
        a, b = a[:, None], b[:, None]
    scale = np.maximum(np.max(np.abs(b), axis=0), 1e-300)
    return float(np.max(np.max(np.abs(a - b), axis=0) / scale))
