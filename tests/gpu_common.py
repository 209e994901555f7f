"""Helpers shared by the GPU tests (no oracle code, no method arithmetic)."""
import numpy as np
import pytest


def have_gpu():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.abs(b)


requires_gpu = pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")
