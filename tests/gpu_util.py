"""Helpers shared by the GPU parity tests (they call the CUDA path through the
C ABI via the ctypes binding and compare with the FP64 oracle)."""
from __future__ import annotations

import numpy as np
import pytest

# FP32 parity bar: per-transform relative L2 error against the FP64 oracle.
TOL_FP32 = 1e-6


def cuda_or_skip():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_4938_b300 import build as B
    B.build()
    return torch


def to_dev(x: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex64)).cuda()


def run(lengths, batch, x: np.ndarray, direction=-1, precision="fp32", inplace=False):
    """Run one plan on x (numpy complex64, [batch, *lengths]) and return numpy."""
    import torch
    from paper_1203_4938_b300 import fft as F
    with F.Plan(lengths, batch, precision) as p:
        d = to_dev(x.reshape(p.shape))
        out = d if inplace else None
        y = p.exec(d, out, direction)
        torch.cuda.synchronize()
        p.check()
        return y.cpu().numpy()


def max_rel_l2(y, ref, axes):
    y = np.asarray(y, np.complex128)
    ref = np.asarray(ref, np.complex128)
    d = np.sqrt(np.sum(np.abs(y - ref) ** 2, axis=axes))
    r = np.sqrt(np.sum(np.abs(ref) ** 2, axis=axes))
    e = np.where(r > 0, d / np.where(r > 0, r, 1), d)
    return float(np.max(e)) if e.size else 0.0
