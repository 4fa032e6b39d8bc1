"""Maximum sizes: batches whose element count passes 2^31 (byte offsets past
2^34), one per kernel family, so that an index kept in 32 bits anywhere on
the path shows up as wrong values in the last transforms.  The inputs are
drawn on the device from a seeded generator; sampled transforms (first,
middle, last) are copied back and compared with the FP64 oracle.
Bar: per-transform relative L2 error <= 1e-6.  Each case holds at most about
52 GB of device memory (input, output, workspace)."""
import numpy as np
import pytest

import oracle
from paper_1203_4938_b300 import fft as F
from tests.gpu_util import TOL_FP32, cuda_or_skip, max_rel_l2

pytestmark = pytest.mark.gpu

TWO31 = 1 << 31


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


def device_input(torch, numel, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    return torch.randn(numel, dtype=torch.complex64, device="cuda", generator=g)


def free(torch):
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


# (length, batch, plan family expected in the description)
CASES_1D = [
    (1024, (TWO31 >> 10) + 3, "rows"),
    (1 << 16, (TWO31 >> 16) + 1, "fourstep-persist"),
    (1 << 21, (TWO31 >> 21) + 1, "fourstep-persist"),  # 16384-point tiles on 1024 threads
    (1 << 24, (TWO31 >> 24) + 1, "threestep"),
    (768, TWO31 // 768 + 1, "rows-mixed"),
    (49152, TWO31 // 49152 + 1, "fourstep-mixed"),
    (1000, TWO31 // 1000 + 1, "generic"),
    (1009, TWO31 // 1009 + 1, "generic"),
]


@pytest.mark.parametrize("n,batch,kind", CASES_1D)
def test_1d_past_2e31_elements(torch, n, batch, kind):
    assert n * batch > TWO31
    x = device_input(torch, n * batch, seed=n)
    try:
        with F.Plan((n,), batch) as p:
            assert p.describe().startswith(kind), p.describe()
            y = p.forward(x.view(batch, n))
            torch.cuda.synchronize()
            p.check()
        rows = sorted({0, batch // 2, batch - 1})
        xs = np.stack([x[r * n:(r + 1) * n].cpu().numpy() for r in rows])
        ys = np.stack([y[r].cpu().numpy() for r in rows])
        del y
        assert max_rel_l2(ys, oracle.fft(xs, -1), -1) <= TOL_FP32, (n, batch)
    finally:
        del x
        free(torch)


@pytest.mark.parametrize("side,batch,kind", [(4096, (TWO31 >> 24) + 1, "2d H="), (2048, (TWO31 >> 22) + 1, "2d-persist")])
def test_2d_past_2e31_elements(torch, side, batch, kind):
    m = side * side
    x = device_input(torch, m * batch, seed=side)
    try:
        with F.Plan((side, side), batch) as p:
            assert p.describe().startswith(kind), p.describe()
            y = p.forward(x.view(batch, side, side))
            torch.cuda.synchronize()
            p.check()
        rows = [0, batch - 1]
        xs = np.stack([x[r * m:(r + 1) * m].cpu().numpy().reshape(side, side) for r in rows])
        ys = np.stack([y[r].cpu().numpy() for r in rows])
        del y
        assert max_rel_l2(ys.reshape(2, -1), oracle.fft2(xs, -1).reshape(2, -1), -1) <= TOL_FP32
    finally:
        del x
        free(torch)


def test_ragged_past_2e31_elements(torch):
    lengths = [1 << 20] * 2048 + [1009, 768, 6000, 65536]
    total = sum(lengths)
    assert total > TWO31
    x = device_input(torch, total, seed=77)
    try:
        with F.Ragged(lengths) as p:
            y = p.forward(x)
            torch.cuda.synchronize()
            p.check()
        offs = np.concatenate([[0], np.cumsum(lengths)])
        for t in [0, 2047, 2048, 2049, 2050, 2051]:
            a, b = int(offs[t]), int(offs[t + 1])
            xs = x[a:b].cpu().numpy()[None]
            ys = y[a:b].cpu().numpy()[None]
            assert max_rel_l2(ys, oracle.fft(xs, -1), -1) <= TOL_FP32, (t, lengths[t])
        del y
    finally:
        del x
        free(torch)


def test_real_past_2e31_complex_elements(torch):
    # R2C of n = 4096: the inner complex plan of 2048 points runs 2^31 + 2048 elements
    n, batch = 4096, (1 << 20) + 1
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    x = torch.randn(batch, n, device="cuda", generator=g)
    try:
        with F.RealPlan(n, batch) as p:
            y = p.forward(x)
            torch.cuda.synchronize()
            p.check()
        rows = [0, batch - 1]
        xs = x[rows].cpu().numpy().astype(np.complex64)
        ys = y[rows].cpu().numpy()
        del y
        ref = oracle.fft(xs, -1)[:, : n // 2 + 1]
        assert max_rel_l2(ys, ref, -1) <= TOL_FP32
    finally:
        del x
        free(torch)
