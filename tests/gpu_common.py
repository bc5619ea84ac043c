"""Shared helpers for the GPU parity tests (CUDA path vs the FP64 oracle)."""

import numpy as np
import pytest

import oracle


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def lib():
    torch_cuda()
    import paper_astro_ph_0703100_gb300 as cn

    cn.load()
    return cn


def dev_tensor(a):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_pot_err(pot, ref):
    pot = np.asarray(pot, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(pot - ref) / np.maximum(np.abs(ref), 1e-300))) if ref.size else 0.0


def e_max(a, ref):
    return oracle.e_max(np.asarray(a, dtype=np.float64), ref)
