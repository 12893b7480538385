"""Helpers for the GPU tests: build/load the library and move arrays."""
import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def lib():
    from paper_1902_01458_gb300 import build
    build.build()
    import paper_1902_01458_gb300 as rr
    rr.load()
    return rr


def to_dev(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def phase_align(A, B):
    """Multiply each column of A by the unit phase that best matches B."""
    out = A.copy()
    for j in range(A.shape[1]):
        z = np.vdot(A[:, j], B[:, j])
        if abs(z) > 0:
            out[:, j] *= np.exp(1j * np.angle(z))
    return out
