"""Shared helpers for the GPU tests (not a test module)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def ctx_and_lre():
    from paper_1602_08604_gb300 import lre
    return lre, lre.lre_create(0)


def rel_fro(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
