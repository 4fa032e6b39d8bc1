"""Parity of the fused image-example kernel (Sec. III-B steps 1-3: colour
transform, chroma 2x2 downscale, directional derivative of luminance) with the
FP64 oracle (needs a GPU).

Tolerance (absolute, on values up to 255): 2e-4.  The kernel evaluates the
same formulas in FP32 with FMA: each luminance/chroma value is three products
of constants (rounded to FP32, relative 2^-24) with integers <= 255 plus an
offset, about 5e-5 worst case; a 2x2 mean or a derivative combines up to
four such values (<= 1e-4)."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import cuda_or_skip

pytestmark = pytest.mark.gpu
TOL = 2e-4


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


def check(torch, rgb, ux, uy):
    from paper_1203_4938_b300 import fft as F
    y, cb, cr, d = F.image_steps(torch.from_numpy(rgb).cuda(), ux, uy)
    torch.cuda.synchronize()
    ry, rcb, rcr, rd = oracle.image_steps(rgb, ux, uy)
    for name, got, ref in (("y", y, ry), ("cb", cb, rcb), ("cr", cr, rcr), ("d", d, rd)):
        err = float(np.max(np.abs(got.cpu().numpy().astype(np.float64) - ref))) if ref.size else 0.0
        assert err <= TOL, (name, rgb.shape, ux, uy, err)


@pytest.mark.parametrize("b,h,w", [(1, 2, 2), (1, 32, 128), (2, 34, 130), (3, 66, 258), (1, 512, 512),
                                   (2, 100, 70), (1, 2, 200), (1, 300, 2), (4, 64, 1024), (1, 30, 126), (2, 40, 132), (1, 4, 4)])
@pytest.mark.parametrize("ux,uy", [(1.0, 0.0), (0.0, 1.0), (0.6, -0.8)])
def test_image_steps(torch, b, h, w, ux, uy):
    rgb = np.random.default_rng(h * 1000 + w + b).integers(0, 256, (b, h, w, 3)).astype(np.uint8)
    check(torch, rgb, ux, uy)


def test_image_workload_shape(torch):
    """An image-shaped input (smooth field plus noise) of the benchmark's kind."""
    from paper_1203_4938_b300 import inputs
    rgb = inputs.rgb_images(np.random.default_rng(7), 2, 256, 384)
    check(torch, rgb, 0.70710678, 0.70710678)


def test_bad_arguments(torch):
    from paper_1203_4938_b300 import fft as F
    t = torch.zeros((1, 4, 4, 3), dtype=torch.uint8, device="cuda")
    y = torch.empty((1, 4, 4), device="cuda")
    c = torch.empty((1, 2, 2), device="cuda")
    assert F.fft_image_steps(t.data_ptr(), 1, 3, 4, 1.0, 0.0, y.data_ptr(), c.data_ptr(), c.data_ptr(),
                             y.data_ptr()) == F.FFT_ERR_INVALID_ARG  # odd height
    assert F.fft_image_steps(t.data_ptr(), 1, 4, 4, 1.0, 0.0, y.data_ptr() + 2, c.data_ptr(), c.data_ptr(),
                             y.data_ptr()) == F.FFT_ERR_MISALIGNED
    assert F.fft_image_steps(t.data_ptr() + 1, 1, 4, 4, 1.0, 0.0, y.data_ptr(), c.data_ptr(), c.data_ptr(),
                             y.data_ptr()) == F.FFT_ERR_MISALIGNED
    assert F.fft_image_steps(0, 1, 4, 4, 1.0, 0.0, y.data_ptr(), c.data_ptr(), c.data_ptr(),
                             y.data_ptr()) == F.FFT_ERR_INVALID_ARG
