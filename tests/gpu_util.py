"""Helpers for the GPU parity tests (no arithmetic of the method here)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_02650_gb300 import pecc

    pecc.load()
    return torch, pecc


def split(arr, n):
    """Split a per-circle array into per-instance pieces."""
    off = np.concatenate([[0], np.cumsum(n)])
    return [arr[off[q]:off[q + 1]] for q in range(len(n))]


def ragged_sizes():
    """Ragged instance sizes spanning several blocks and odd tails, including the degenerate ones."""
    return np.array([0, 1, 2, 3, 7, 50, 257, 300, 511, 1000, 1023, 33], dtype=np.int32)
