"""Shared helpers for the GPU tests (no method arithmetic here)."""
import numpy as np
import pytest


def spec_norm_sym(M) -> float:
    """Spectral norm of the symmetric part of M (FP64, numpy)."""
    M = np.asarray(M, dtype=np.float64)
    return float(np.abs(np.linalg.eigvalsh(0.5 * (M + M.T))).max())


def cuda_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def lib_or_fail():
    """The CUDA library must be present on a GPU host: a missing build fails the test."""
    import paper_2605_24840_gb300 as rs
    rs.load()
    return rs
