"""Parity of the six-step plan for 1-D lengths above 2^24 points
(transpose, N1-point plan, twiddle + transpose, N2-point plan, transpose)
with the FP64 oracle: powers of two, 7 * 2^22, 5^11 (sampled bins from the
definition), and 2^30 points by a closed form (an impulse) and the round
trip.  Also in place, kernel by kernel, and the switch.
Bar: per-transform relative L2 error <= 1e-6 (round trips 2e-6)."""
import numpy as np
import pytest

import oracle
from paper_1203_4938_b300 import fft as F
from paper_1203_4938_b300 import inputs
from tests.gpu_util import TOL_FP32, cuda_or_skip, max_rel_l2, run, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


def free(torch):
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("form", ["columns", "transposing"])
@pytest.mark.parametrize("n,batch", [(1 << 25, 2), (7 << 22, 1)])
def test_sixstep_against_oracle(torch, monkeypatch, form, n, batch):
    # columns: 256-point column transforms with the twiddle, N2 plan, one
    # transpose; transposing: transpose, N1 plan, twiddle + transpose, N2
    # plan, transpose (the form for lengths without a factor 2^8)
    if form == "transposing":
        monkeypatch.setenv("B300FFT_SIXSTEP_COLS", "0")
    x = inputs.normal_batch(batch, n, seed=n % 1000)
    with F.Plan((n,), batch) as p:
        assert p.describe().startswith("sixstep"), p.describe()
        assert ("= 256 (columns, C=16, twiddle)" in p.describe()) == (form == "columns"), p.describe()
    for d in (-1, +1):
        y = run((n,), batch, x, d)
        assert max_rel_l2(y, oracle.fft(x, d), -1) <= TOL_FP32, (n, d)
    free(torch)


def test_sixstep_odd_length_sampled_bins(torch):
    # 5^11 = 3125 x 15625: both factors on the stage-graph executor
    n = 5 ** 11
    x = inputs.uniform_batch(1, n, seed=3)
    with F.Plan((n,), 1) as p:
        assert p.describe().startswith("sixstep N=48828125 = 3125 x 15625"), p.describe()
    y = run((n,), 1, x, -1)
    ks = np.array([0, 1, 15625, 4882812, 31250001, n - 1], dtype=np.int64)
    ref = oracle.dft_bins(x[0], ks, -1)
    # the sampled bins' error norm over their norm estimates the relative L2
    err = np.linalg.norm(y[0, ks] - ref) / np.linalg.norm(ref)
    assert err <= TOL_FP32, err
    free(torch)


def test_sixstep_2e30_impulse_and_round_trip(torch):
    n = 1 << 30
    n0 = 123456789
    x = torch.zeros(n, dtype=torch.complex64, device="cuda")
    x[n0] = 1
    try:
        with F.Plan((n,), 1) as p:
            assert p.describe().startswith("sixstep"), p.describe()
            y = p.forward(x.view(1, n))
            torch.cuda.synchronize()
            p.check()
            ks = np.random.default_rng(7).integers(0, n, 4096, dtype=np.int64)
            ks[:3] = [0, 1, n - 1]
            got = y[0, torch.from_numpy(ks).cuda()].cpu().numpy().astype(np.complex128)
            ref = np.exp(-2j * np.pi * ((n0 * ks) % n).astype(np.float64) / n)  # X[k] = W_N^{n0 k}
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL_FP32
            del y
            g = torch.Generator(device="cuda")
            g.manual_seed(11)
            x.copy_(torch.randn(n, dtype=torch.complex64, device="cuda", generator=g))
            y = p.forward(x.view(1, n))
            z = p.inverse(y)
            torch.cuda.synchronize()
            p.check()
            del y
            z.div_(n).sub_(x.view(1, n))
            num = torch.linalg.vector_norm(z).item()
            den = torch.linalg.vector_norm(x).item()
            assert num / den <= 2 * TOL_FP32, num / den
            del z
    finally:
        del x
        free(torch)


@pytest.mark.parametrize("cols", ["1", "0"])
def test_sixstep_in_place_and_kernel_sequence(torch, monkeypatch, cols):
    monkeypatch.setenv("B300FFT_SIXSTEP_COLS", cols)
    n, batch = 1 << 25, 1
    x = to_dev(inputs.uniform_batch(batch, n, seed=4))
    with F.Plan((n,), batch) as p:
        ref = p.forward(x).clone()
        inplace = x.clone()
        p.exec(inplace, inplace, F.FFT_FORWARD)
        out = torch.empty_like(x)
        for k in range(p.kernel_count):
            p.exec_kernel(k, x, out, F.FFT_FORWARD)
        seq_in = x.clone()
        for k in range(p.kernel_count):
            p.exec_kernel(k, seq_in, seq_in, F.FFT_FORWARD)
        torch.cuda.synchronize()
        p.check()
        assert torch.equal(inplace, ref)
        assert torch.equal(out, ref)
        assert torch.equal(seq_in, ref)
    del x, ref, inplace, out, seq_in
    free(torch)


def test_sixstep_switched_off(torch, monkeypatch):
    monkeypatch.setenv("B300FFT_SIXSTEP", "0")
    assert F.fft_plan_create(1, [1 << 25], 1, 0) is None
    assert F.fft_last_error() == F.FFT_ERR_UNSUPPORTED
