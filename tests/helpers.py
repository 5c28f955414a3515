"""Shared helpers for the GPU parity tests (tolerances and conversions)."""
import numpy as np
import pytest

# Tolerances: max |x - x_oracle| / max |x_oracle| per curve or vector.
TOL = {"c128": 1e-10, "c64": 1e-5}


def torch_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch


def tdtype(torch, name):
    return torch.complex128 if name == "c128" else torch.complex64


def to_dev(torch, arr, name):
    """(B, D) or (D,) host array -> (D, B) contiguous CUDA tensor of the dtype."""
    a = np.asarray(arr)
    if a.ndim == 2:
        a = a.T
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=tdtype(torch, name)).contiguous()


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
