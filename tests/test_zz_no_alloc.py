"""The allocation-free entry point fft_exec_pow2_static (GPU).

Some callers cannot allocate device memory once they are running (an engine
that fixed its device budget at start-up, a plugin whose host forbids
cudaMalloc), so they cannot create a plan.  fft_exec_pow2_static runs the same
two-pass four-step kernels with a workspace and tables kept in static device
arrays of the library.  Here its output, called through the C ABI, must match
the plan path (fft_exec) and the FP64 oracle within the FP32 tolerance, on two
calls in a row (the second call reuses the static arrays and the tables the
first one left behind), and calls after the first must leave the device's
free memory unchanged.

This file is named to be collected last."""
import numpy as np
import pytest

import oracle
from paper_1203_4938_b300 import inputs
from tests.gpu_util import TOL_FP32, cuda_or_skip, max_rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.mark.parametrize("logn,batch", [(13, 3), (16, 5), (18, 16), (22, 1)])
def test_static_matches_plan_twice(torch, logn, batch):
    from paper_1203_4938_b300 import fft as F
    n = 1 << logn
    x = to_dev(inputs.normal_batch(batch, n, seed=logn + batch))
    stream = torch.cuda.current_stream().cuda_stream
    for d in (F.FFT_FORWARD, F.FFT_INVERSE):
        with F.Plan((n,), batch) as p:
            ref = p.exec(x, None, d)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy()
        exact = oracle.fft(x.cpu().numpy(), d)
        for call in range(2):
            out = torch.full_like(x, complex(float("nan"), float("nan")))
            rc = F.fft_exec_pow2_static(x.data_ptr(), out.data_ptr(), n, batch, d, stream)
            assert rc == F.FFT_OK, F.fft_status_string(rc)
            torch.cuda.synchronize()
            err = max_rel_l2(out.cpu().numpy(), ref, -1)
            assert err <= TOL_FP32, (logn, batch, d, call, err)
            err = max_rel_l2(out.cpu().numpy(), exact, -1)
            assert err <= TOL_FP32, ("oracle", logn, batch, d, call, err)


def test_static_calls_leave_free_memory_unchanged(torch):
    """After a first call of each length (which may load the module holding
    the static arrays and the kernels it launches), further calls, with the
    same n and alternating with another n, allocate nothing:
    cudaMemGetInfo's free bytes stay the same."""
    from paper_1203_4938_b300 import fft as F
    n, batch = 1 << 14, 6
    x = to_dev(inputs.uniform_batch(batch, n, seed=5))
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream().cuda_stream
    for nn, bb in ((n, batch), (1 << 15, 3)):
        assert F.fft_exec_pow2_static(x.data_ptr(), out.data_ptr(), nn, bb, F.FFT_FORWARD, stream) == F.FFT_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for nn, bb in ((n, batch), (n, batch), (1 << 15, 3), (n, batch)):
        assert F.fft_exec_pow2_static(x.data_ptr(), out.data_ptr(), nn, bb, F.FFT_INVERSE, stream) == F.FFT_OK
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    y = out.cpu().numpy()
    assert max_rel_l2(y, oracle.fft(x.cpu().numpy(), +1), -1) <= TOL_FP32


def test_static_in_place_and_limits(torch):
    from paper_1203_4938_b300 import fft as F
    n, batch = 1 << 15, 4
    xh = inputs.uniform_batch(batch, n, seed=21)
    x = to_dev(xh)
    with F.Plan((n,), batch) as p:
        ref = p.exec(x).cpu().numpy()
    y = x.clone()
    assert F.fft_exec_pow2_static(y.data_ptr(), y.data_ptr(), n, batch, F.FFT_FORWARD, 0) == F.FFT_OK
    torch.cuda.synchronize()
    assert max_rel_l2(y.cpu().numpy(), ref, -1) <= TOL_FP32
    # sizes beyond the static workspace, and shapes it does not cover
    big = x.data_ptr()
    assert F.fft_exec_pow2_static(big, big, 1 << 22, 2, F.FFT_FORWARD, 0) == F.FFT_ERR_INVALID_ARG
    assert F.fft_exec_pow2_static(big, big, 1 << 23, 1, F.FFT_FORWARD, 0) == F.FFT_ERR_INVALID_ARG
    assert F.fft_exec_pow2_static(big, big, 3 << 13, 1, F.FFT_FORWARD, 0) == F.FFT_ERR_INVALID_ARG
    assert F.fft_exec_pow2_static(big, big, 1 << 12, 1, F.FFT_FORWARD, 0) == F.FFT_ERR_INVALID_ARG
    assert F.fft_exec_pow2_static(big + 8, big, 1 << 15, 1, F.FFT_FORWARD, 0) == F.FFT_ERR_MISALIGNED
    assert F.fft_exec_pow2_static(big, big, 1 << 15, 1, 0, 0) == F.FFT_ERR_INVALID_ARG
