"""Parity at the benchmark's full sizes, in the launch configuration it times
(needs a GPU).

For every size of the power-of-two sweep (N = 2^10 .. 2^24, batch 2^26 / N,
the benchmark's own seeded input) the default plan runs forward and then
inverse on the whole batch, as the benchmark does.  The oracle computes
sampled outputs one by one (O(N) per bin, FP64): SAMPLE_T transforms spread
over the batch, SAMPLE_K bins each (0, N/2 and random bins).  The relative
error of a transform is estimated from its sampled bins as
    rms_k |y_k - X_k| / ||x||_2
which is the per-transform relative L2 error when the error is spread evenly
over the bins (Parseval: ||X||_2 = sqrt(N) ||x||_2).  The inverse is checked
the same way against the oracle's inverse DFT of the GPU's forward output."""
import numpy as np
import pytest

import oracle
from paper_1203_4938_b300 import inputs
from tests.gpu_util import TOL_FP32, cuda_or_skip

pytestmark = pytest.mark.gpu

TOTAL_LOG2 = 26
SAMPLE_T = 3
SAMPLE_K = 32


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


def sampled_rel_err(x, y, sign, rng):
    """Estimated relative L2 error of the transforms of x given as y, from
    SAMPLE_K bins of SAMPLE_T transforms; returns the max over them."""
    b, n = x.shape
    rows = sorted({0, b // 2, b - 1})[:SAMPLE_T]
    worst = 0.0
    for r in rows:
        ks = np.unique(np.concatenate([[0, n // 2], rng.integers(0, n, SAMPLE_K - 2)])) % n
        ref = oracle.dft_bins(x[r], ks, sign)
        err = np.sqrt(np.mean(np.abs(y[r, ks].astype(np.complex128) - ref) ** 2))
        norm = np.sqrt(np.sum(np.abs(x[r].astype(np.complex128)) ** 2))
        worst = max(worst, err / norm)
    return worst


@pytest.mark.parametrize("k", list(range(10, 25)))
def test_sweep_size_sampled(torch, k):
    from paper_1203_4938_b300 import fft as F
    n, b = 1 << k, 1 << (TOTAL_LOG2 - k)
    x = inputs.sweep_input(k, TOTAL_LOG2, seed=1)
    rng = np.random.default_rng(1000 + k)
    with F.Plan((n,), b) as p:
        d = torch.from_numpy(x).cuda()
        y = p.forward(d)
        z = p.inverse(y)
        torch.cuda.synchronize()
        p.check()
        yh = y.cpu().numpy()
        zh = z.cpu().numpy()
    del d, y, z
    assert sampled_rel_err(x, yh, -1, rng) <= TOL_FP32, k
    # inverse: oracle inverse DFT of the GPU's forward output
    assert sampled_rel_err(yh, zh, +1, rng) <= TOL_FP32, k
