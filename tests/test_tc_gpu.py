"""Tensor-core radix-16 path (tcgen05, FP16/BF16 operands, FP32 accumulation)
against the FP64 oracle (needs a GPU).

Stated tolerances (per-transform relative L2, max over the batch), from the
operand precision: a hi+lo split keeps ~22 bits (FP16) or ~16 bits (BF16) of
each product, the plain forms 11 and 8 bits, with errors growing slowly with
the number of radix-16 passes:
    fp16 hi+lo 1e-6   bf16 hi+lo 2e-5   fp16 plain 2e-3   bf16 plain 2e-2
"""
import numpy as np
import pytest

import oracle
from paper_1203_4938_b300 import inputs
from tests.gpu_util import cuda_or_skip, max_rel_l2, run

pytestmark = pytest.mark.gpu

TOL = {"tc_fp16": 1e-6, "tc_bf16": 2e-5, "tc_fp16_plain": 2e-3, "tc_bf16_plain": 2e-2}


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.mark.parametrize("mode", list(TOL))
@pytest.mark.parametrize("n,batch", [(256, 37), (4096, 5), (65536, 3)])
def test_tc_parity(torch, mode, n, batch):
    x = inputs.normal_batch(batch, n, seed=n + batch)
    for d in (-1, +1):
        y = run((n,), batch, x, d, precision=mode)
        err = max_rel_l2(y, oracle.fft(x, d), -1)
        assert err <= TOL[mode], (mode, n, d, err)


@pytest.mark.parametrize("n,batch", [(4096, 4096), (65536, 256)])
def test_precision_workload_against_oracle(torch, n, batch):
    """The benchmark's precision workload (normal(0,1) seed 3, both shapes):
    first, middle and last transforms of every mode against the FP64 oracle,
    FP32 at 1e-6 and each tensor-core mode at its stated tolerance."""
    x = inputs.normal_batch(batch, n, seed=3)
    sample = [0, batch // 2, batch - 1]
    ref = oracle.fft(x[sample], -1)
    for mode, tol in [("fp32", 1e-6)] + list(TOL.items()):
        y = run((n,), batch, x, -1, precision=mode)
        err = max_rel_l2(y[sample], ref, -1)
        assert err <= tol, (mode, n, err)


@pytest.mark.parametrize("grid", ["0", "1", "5"])
@pytest.mark.parametrize("n,batch", [(256, 700), (4096, 500), (65536, 40)])
def test_tc_persistent_grids(torch, monkeypatch, grid, n, batch):
    """The persistent tensor-core kernels with one CTA per work unit (0), one
    CTA per SM (1: every CTA runs many units) and more CTAs than fit at once
    (5 per SM: the later ones start as others finish)."""
    monkeypatch.setenv("B300FFT_TC_GRID", grid)
    x = inputs.normal_batch(batch, n, seed=n % 1000 + batch)
    sample = [0, 1, batch // 2, batch - 1]
    y = run((n,), batch, x, -1, precision="tc_fp16")
    err = max_rel_l2(y[sample], oracle.fft(x[sample], -1), -1)
    assert err <= TOL["tc_fp16"], (grid, n, err)


@pytest.mark.parametrize("mode", ["tc_fp16", "tc_bf16"])
def test_tc_dynamic_range(torch, mode):
    """Per-butterfly power-of-two scaling: a large constant offset (DC of
    N * 1e4) and tiny inputs (1e-30) keep the relative error of the split."""
    n = 4096
    base = inputs.normal_batch(2, n, seed=9)
    for x in (base + np.complex64(1e4), base * np.float32(1e-30)):
        y = run((n,), 2, x.astype(np.complex64), -1, precision=mode)
        err = max_rel_l2(y, oracle.fft(x, -1), -1)
        assert err <= TOL[mode], (mode, err)


def test_tc_impulse_and_unsupported(torch):
    from paper_1203_4938_b300 import fft as F
    x = np.zeros((3, 4096), np.complex64)
    x[:, 0] = 1
    y = run((4096,), 3, x, -1, precision="tc_fp16")
    assert np.allclose(y, 1, atol=1e-6)
    for n in (64, 1024, 1 << 20, 3000):
        assert F.fft_plan_create(1, [n], 1, F.FFT_TC_FP16) is None
        assert F.fft_last_error() == F.FFT_ERR_UNSUPPORTED
