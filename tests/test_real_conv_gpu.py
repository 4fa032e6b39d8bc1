"""Real-to-complex / complex-to-real transforms and FFT convolution on the
GPU against the FP64 oracle (needs a GPU).  Bar: relative L2 <= 1e-6."""
import numpy as np
import pytest

import oracle
from paper_1203_4938_b300 import inputs
from tests.gpu_util import TOL_FP32, cuda_or_skip, max_rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.mark.parametrize("n,batch", [(2, 3), (6, 5), (64, 7), (1000, 3), (4096, 9), (1 << 16, 3),
                                     (2 * 1009, 2), (3 * 2 ** 13, 2), (1 << 20, 1)])
def test_r2c_c2r(torch, n, batch):
    from paper_1203_4938_b300 import fft as F
    rng = np.random.default_rng(n + batch)
    xr = rng.standard_normal((batch, n)).astype(np.float32)
    ref = oracle.fft(xr.astype(np.complex128), -1)[:, : n // 2 + 1]
    with F.RealPlan(n, batch) as p:
        X = p.forward(torch.from_numpy(xr).cuda())
        torch.cuda.synchronize()
        assert max_rel_l2(X.cpu().numpy(), ref, -1) <= TOL_FP32
        y = p.inverse(X)
        torch.cuda.synchronize()
        p.check()
    assert max_rel_l2((y.cpu().numpy() / n).astype(np.complex128), xr.astype(np.complex128), -1) <= 2 * TOL_FP32


@pytest.mark.parametrize("logh", [5, 6, 7, 8, 9, 10, 11, 12])
@pytest.mark.parametrize("fused", ["1", "0"])
def test_r2c_c2r_fused_range(torch, monkeypatch, logh, fused):
    """n = 2h with h = 2^5..2^12: one fused pass per direction (split /
    merge inside the tile), or the two-pass form when switched off; the batch
    leaves the last CTA partly empty."""
    from paper_1203_4938_b300 import fft as F
    monkeypatch.setenv("B300FFT_REAL_FUSED", fused)
    h = 1 << logh
    n = 2 * h
    tpc = max(1, 256 // (h // 16))
    batch = 2 * tpc + 1
    rng = np.random.default_rng(logh)
    xr = rng.standard_normal((batch, n)).astype(np.float32)
    ref = oracle.fft(xr.astype(np.complex128), -1)[:, : n // 2 + 1]
    with F.RealPlan(n, batch) as p:
        assert ("fused" in p.describe()) == (fused == "1"), p.describe()
        X = p.forward(torch.from_numpy(xr).cuda())
        torch.cuda.synchronize()
        assert max_rel_l2(X.cpu().numpy(), ref, -1) <= TOL_FP32
        y = p.inverse(X)
        torch.cuda.synchronize()
        p.check()
    assert max_rel_l2((y.cpu().numpy() / n).astype(np.complex128), xr.astype(np.complex128), -1) <= 2 * TOL_FP32


@pytest.mark.parametrize("n", [256, 4096])
def test_r2c_c2r_in_place(torch, n):
    """in == out (the buffer holds batch * (n/2+1) complex values): the fused
    plan falls back to the two-pass form, which reads its input first."""
    from paper_1203_4938_b300 import fft as F
    batch, h = 5, n // 2
    rng = np.random.default_rng(n)
    xr = rng.standard_normal((batch, n)).astype(np.float32)
    ref = oracle.fft(xr.astype(np.complex128), -1)[:, : h + 1]
    buf = torch.zeros(batch * (h + 1), dtype=torch.complex64, device="cuda")
    buf.view(torch.float32)[: batch * n].copy_(torch.from_numpy(xr.reshape(-1)).cuda())
    with F.RealPlan(n, batch) as p:
        assert "fused" in p.describe()
        assert F.fft_exec(p.handle, buf.data_ptr(), buf.data_ptr(), F.FFT_FORWARD) == F.FFT_OK
        torch.cuda.synchronize()
        assert max_rel_l2(buf.view(batch, h + 1).cpu().numpy(), ref, -1) <= TOL_FP32
        assert F.fft_exec(p.handle, buf.data_ptr(), buf.data_ptr(), F.FFT_INVERSE) == F.FFT_OK
        torch.cuda.synchronize()
        p.check()
    y = buf.view(torch.float32)[: batch * n].cpu().numpy().reshape(batch, n) / n
    assert max_rel_l2(y.astype(np.complex128), xr.astype(np.complex128), -1) <= 2 * TOL_FP32


def test_c2r_of_oracle_half_spectrum(torch):
    """C2R alone, fed the oracle's half spectrum of a real signal."""
    from paper_1203_4938_b300 import fft as F
    n, batch = 4096, 4
    xr = np.random.default_rng(3).uniform(-1, 1, (batch, n))
    half = oracle.fft(xr.astype(np.complex128), -1)[:, : n // 2 + 1].astype(np.complex64)
    with F.RealPlan(n, batch) as p:
        y = p.inverse(to_dev(half))
        torch.cuda.synchronize()
    assert max_rel_l2(y.cpu().numpy().astype(np.complex128) / n, xr.astype(np.complex128), -1) <= 2 * TOL_FP32


def test_real_plan_rejects_odd(torch):
    from paper_1203_4938_b300 import fft as F
    assert F.fft_plan_create_real(1001, 1) is None
    assert F.fft_last_error() == F.FFT_ERR_UNSUPPORTED


@pytest.mark.parametrize("n,batch", [(8, 3), (1024, 4), (1000, 2), (1 << 16, 2), (97, 3)])
@pytest.mark.parametrize("corr", [False, True])
def test_convolution_1d(torch, n, batch, corr):
    from paper_1203_4938_b300 import fft as F
    x = inputs.uniform_batch(batch, n, seed=n)
    h = inputs.uniform_batch(1, n, seed=n + 1)[0]
    y = F.convolve(to_dev(x), to_dev(h), corr).cpu().numpy()
    ref = oracle.circ_conv(x, h, corr) if n <= 4096 else None
    if ref is None:  # long signal: convolution theorem with the oracle's FFT
        ref = oracle.fft(oracle.fft(x, -1) * (np.conj(oracle.fft(h, -1)) if corr else oracle.fft(h, -1)), +1) / n
    assert max_rel_l2(y, ref, -1) <= 2 * TOL_FP32


@pytest.mark.parametrize("hgt,wid", [(64, 128), (60, 90), (96, 1009)])
def test_convolution_2d_image_blur(torch, hgt, wid):
    """2-D circular filtering of image-shaped data (a 3x3 box kernel) in one
    fft_convolve call on a 2-D plan (in-place column kernels for 64 x 128,
    the transposing plan for 60 x 90 and 96 x 1009), against the sum of
    shifted images that defines it."""
    from paper_1203_4938_b300 import fft as F
    img = inputs.image_batch(np.random.default_rng(1), 2, hgt, wid)
    k = np.zeros((hgt, wid), np.complex64)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            k[dy % hgt, dx % wid] = 1.0 / 9
    y = F.convolve(to_dev(img), to_dev(k)).cpu().numpy()
    ref = np.zeros_like(img, dtype=np.complex128)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            ref += np.roll(img.astype(np.complex128), (dy, dx), axis=(1, 2)) / 9
    assert max_rel_l2(y.reshape(2, -1), ref.reshape(2, -1), -1) <= 2 * TOL_FP32


@pytest.mark.parametrize("n,batch", [(8, 3), (1024, 5), (4096, 7), (8192, 3), (16384, 2), (1000, 3), (1 << 16, 2),
                                     (3 * 1024, 4)])
@pytest.mark.parametrize("corr", [False, True])
def test_fft_convolve_one_call(torch, n, batch, corr):
    """fft_convolve against the oracle's circular convolution / correlation:
    one fused pass for powers of two <= 2^14, the three-step form otherwise;
    out == x in place on the second call."""
    from paper_1203_4938_b300 import fft as F
    rng = np.random.default_rng(n * 3 + batch)
    x = (rng.standard_normal((batch, n)) + 1j * rng.standard_normal((batch, n))).astype(np.complex64)
    h = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    ref = oracle.circ_conv(x, h, corr) if n <= 8192 else None
    with F.Plan((n,), batch) as p, F.Plan((n,), 1) as ph:
        H = ph.forward(to_dev(h.reshape(1, n)))
        xd = to_dev(x)
        out = torch.empty_like(xd)
        s = torch.cuda.current_stream().cuda_stream
        assert F.fft_convolve(p.handle, xd.data_ptr(), H.data_ptr(), out.data_ptr(), 1.0 / n, corr, s) == F.FFT_OK
        assert F.fft_convolve(p.handle, xd.data_ptr(), H.data_ptr(), xd.data_ptr(), 1.0 / n, corr, s) == F.FFT_OK
        torch.cuda.synchronize()
        y, y2 = out.cpu().numpy(), xd.cpu().numpy()
    if ref is None:  # long rows: the convolution theorem against the oracle's transforms
        X = oracle.fft(x, -1)
        Hh = oracle.fft(h[None], -1)[0]
        ref = oracle.fft(X * (np.conj(Hh) if corr else Hh), +1) / n
    assert max_rel_l2(y, ref, -1) <= 4 * TOL_FP32, (n, corr)
    assert np.array_equal(y, y2)


def test_fft_convolve_rejects_ragged_and_real(torch):
    from paper_1203_4938_b300 import fft as F
    buf = torch.zeros(4096, dtype=torch.complex64, device="cuda")
    with F.Ragged([64, 128]) as r, F.RealPlan(64, 1) as q:
        for p in (r, q):
            assert F.fft_convolve(p.handle, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), 1.0, False) == \
                F.FFT_ERR_INVALID_ARG
