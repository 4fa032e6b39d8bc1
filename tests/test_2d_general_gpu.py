"""Parity of the general 2-D plan (1-D plan over the rows, transpose, 1-D
plan over the transposed columns, transpose back) with the FP64 oracle's 2-D
DFT: sides the in-place column kernels do not cover (any length the 1-D path
supports, including primes and powers of two above 4096), in place, the
kernel-by-kernel sequence, and the status words of the inner plans.
Bar: per-image relative L2 error <= 1e-6."""
import numpy as np
import pytest

import oracle
from paper_1203_4938_b300 import fft as F
from tests.gpu_util import TOL_FP32, cuda_or_skip, max_rel_l2, run, to_dev

pytestmark = pytest.mark.gpu

SHAPES = [(7, 5, 3), (9, 64, 2), (64, 11, 2), (97, 1009, 1), (1080, 1920, 1), (1000, 1000, 1), (8192, 512, 1),
          (16384, 64, 2), (3, 6000, 2), (6000, 3, 2), (1, 77, 4), (77, 1, 4)]


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


def image(h, w, batch, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((batch, h, w)) + 1j * rng.standard_normal((batch, h, w))).astype(np.complex64)


@pytest.mark.parametrize("h,w,batch", SHAPES)
def test_general_2d(torch, h, w, batch):
    x = image(h, w, batch, h * 31 + w)
    with F.Plan((h, w), batch) as p:
        assert p.describe().startswith("2d-transpose"), p.describe()
    for d in (-1, +1):
        y = run((h, w), batch, x, d)
        ref = oracle.fft2(x, d)
        assert max_rel_l2(y.reshape(batch, -1), ref.reshape(batch, -1), -1) <= TOL_FP32, (h, w, d)


@pytest.mark.parametrize("h,w", [(1000, 1000), (8192, 512)])
def test_general_2d_in_place_round_trip(torch, h, w):
    x = image(h, w, 1, 5)
    y = run((h, w), 1, x, -1, inplace=True)
    assert max_rel_l2(y.reshape(1, -1), oracle.fft2(x, -1).reshape(1, -1), -1) <= TOL_FP32
    z = run((h, w), 1, y.astype(np.complex64), +1, inplace=True) / (h * w)
    assert max_rel_l2(z.reshape(1, -1), x.reshape(1, -1), -1) <= 2 * TOL_FP32


@pytest.mark.parametrize("h,w,batch", [(96, 1009, 2), (8192, 512, 1), (1024, 1000, 1), (1000, 1024, 1)])
def test_general_2d_kernel_sequence(torch, h, w, batch):
    # fft_exec_kernel k = 0 .. count-1 in order equals one fft_exec (rows plan
    # + two transposes, and the transposed-store rows form)
    x = to_dev(image(h, w, batch, 8))
    with F.Plan((h, w), batch) as p:
        n = F.fft_plan_kernel_count(p.handle)
        assert n >= 3, n
        full = p.forward(x).clone()
        out = torch.empty_like(x)
        for k in range(n):
            p.exec_kernel(k, x, out, F.FFT_FORWARD)
        torch.cuda.synchronize()
        p.check()
        assert torch.equal(out, full)


@pytest.mark.parametrize("h,w,batch,force", [(8192, 512, 1, False), (1000, 64, 3, False), (36, 32, 5, False),
                                             (1024, 1000, 1, False), (64, 36, 3, False), (64, 128, 2, True),
                                             (4096, 32, 1, True)])
def test_general_2d_transposed_store_forms(torch, monkeypatch, h, w, batch, force):
    """A pass over rows of 2^5..2^12 points stores transposed (the
    four-step's transposed-row kernel, no transpose after it): the rows pass
    for such widths, the columns pass for such heights, both when the plan is
    forced on two power-of-two sides; the plan + transpose form when that is
    switched off."""
    if force:
        monkeypatch.setenv("B300FFT_2D_TRANSPOSE", "2")
    x = image(h, w, batch, h + w)
    ref = oracle.fft2(x, -1)
    for rowst in ("1", "0"):
        monkeypatch.setenv("B300FFT_2D_ROWST", rowst)
        with F.Plan((h, w), batch) as p:
            assert ("transposed store" in p.describe()) == (rowst == "1"), p.describe()
        y = run((h, w), batch, x, -1)
        assert max_rel_l2(y.reshape(batch, -1), ref.reshape(batch, -1), -1) <= TOL_FP32, (h, w, rowst)
        z = run((h, w), batch, x, +1, inplace=True)
        assert max_rel_l2(z.reshape(batch, -1), oracle.fft2(x, +1).reshape(batch, -1), -1) <= TOL_FP32


def test_general_2d_switched_off(torch, monkeypatch):
    monkeypatch.setenv("B300FFT_2D_TRANSPOSE", "0")
    assert F.fft_plan_create(2, [7, 5], 1, 0) is None
    assert F.fft_last_error() == F.FFT_ERR_UNSUPPORTED


def test_inner_plan_timeout_reaches_outer_check(torch, monkeypatch):
    """A bounded wait that expires inside the column plan (a persistent
    four-step over H = 2^16, one chunk withheld) is reported by
    fft_plan_check on the 2-D plan, and the words are cleared."""
    h, w, batch = 1 << 16, 3, 1
    x = to_dev(image(h, w, batch, 2))
    monkeypatch.setenv("B300FFT_DEBUG_WITHHOLD_CHUNK", "0")
    monkeypatch.setenv("B300FFT_SPIN_LIMIT", "20000")
    monkeypatch.setenv("B300FFT_CHUNK_MB", "1")
    with F.Plan((h, w), batch) as p:
        assert "persist" in p.describe(), p.describe()
        p.forward(x)
        torch.cuda.synchronize()
        assert F.fft_plan_check(p.handle) == F.FFT_ERR_TIMEOUT
        assert F.fft_plan_check(p.handle) == F.FFT_OK


def test_real_plan_reports_inner_timeout(torch, monkeypatch):
    # the same for a real plan whose complex plan of N/2 = 2^16 times out
    n, batch = 1 << 17, 2
    x = torch.randn(batch, n, device="cuda")
    monkeypatch.setenv("B300FFT_DEBUG_WITHHOLD_CHUNK", "0")
    monkeypatch.setenv("B300FFT_SPIN_LIMIT", "20000")
    monkeypatch.setenv("B300FFT_CHUNK_MB", "1")
    h = F.fft_plan_create_real(n, batch)
    assert h is not None
    try:
        out = torch.empty(batch, n // 2 + 1, dtype=torch.complex64, device="cuda")
        assert F.fft_exec(h, x.data_ptr(), out.data_ptr(), F.FFT_FORWARD) == F.FFT_OK
        torch.cuda.synchronize()
        assert F.fft_plan_check(h) == F.FFT_ERR_TIMEOUT
        assert F.fft_plan_check(h) == F.FFT_OK
    finally:
        F.fft_plan_destroy(h)


@pytest.mark.parametrize("shape,batch", [((96, 1009), 2), ((1 << 25,), 1), ((5 ** 11,), 1)])
def test_per_size_form_matches(torch, shape, batch):
    """fft_exec_per_size runs the inner stage-graph plans as one launch per
    (stage, length) group; through the transposing 2-D plan and both six-step
    forms it gives bitwise the values of fft_exec (the same tiles run, only
    the launch split differs)."""
    numel = batch
    for s in shape:
        numel *= s
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    x = torch.randn((batch,) + shape, dtype=torch.complex64, device="cuda", generator=g)
    with F.Plan(shape, batch) as p:
        a = p.forward(x).clone()
        b = p.exec_per_size(x)
        torch.cuda.synchronize()
        p.check()
        assert torch.equal(a, b), p.describe()
    del x, a, b
    torch.cuda.empty_cache()
