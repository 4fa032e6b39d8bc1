"""Parity of the compile-time mixed-radix kernel (L = M * 2^K <= 4096,
M = 3, 5, 7) with the FP64 oracle: every supported length, a batch whose
last CTA holds fewer lines than the others, both directions, in place, and
the stage-graph path the same lengths take when the kernel is switched off.
Bar: per-transform relative L2 error <= 1e-6."""
import numpy as np
import pytest

import oracle
from paper_1203_4938_b300 import fft as F
from paper_1203_4938_b300 import inputs
from tests.gpu_util import TOL_FP32, cuda_or_skip, max_rel_l2, run

pytestmark = pytest.mark.gpu

LENGTHS = [m << k for m, kmax in ((3, 10), (5, 9), (7, 9)) for k in range(kmax + 1)]


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


def lines_per_cta(n):
    return 4096 // n


@pytest.mark.parametrize("n", LENGTHS)
def test_every_length_ragged_last_cta(torch, n):
    # two full CTAs of lines plus a partial third (one line when a CTA holds one)
    nl = lines_per_cta(n)
    batch = 2 * nl + max(1, nl // 3)
    x = inputs.normal_batch(batch, n, seed=n)
    with F.Plan((n,), batch) as p:
        assert p.describe().startswith("rows-mixed"), p.describe()
    for d in (-1, +1):
        y = run((n,), batch, x, d)
        assert max_rel_l2(y, oracle.fft(x, d), -1) <= TOL_FP32, (n, batch, d)


@pytest.mark.parametrize("n", [3, 96, 768, 2560, 3584])
def test_in_place_and_single_line(torch, n):
    for batch in (1, 5):
        x = inputs.uniform_batch(batch, n, seed=7 * n + batch)
        for d in (-1, +1):
            y = run((n,), batch, x, d, inplace=True)
            assert max_rel_l2(y, oracle.fft(x, d), -1) <= TOL_FP32, (n, batch, d)


@pytest.mark.parametrize("n", [6, 1536, 3072])
def test_round_trip(torch, n):
    batch = 9
    x = inputs.normal_batch(batch, n, seed=n + 1)
    y = run((n,), batch, x, -1)
    z = run((n,), batch, y.astype(np.complex64), +1) / n
    assert max_rel_l2(z, x, -1) <= 2 * TOL_FP32


@pytest.mark.parametrize("n", [3, 48, 320, 768, 3584])
def test_stage_graph_path_when_switched_off(torch, monkeypatch, n):
    monkeypatch.setenv("B300FFT_MIXED", "0")
    batch = 7
    x = inputs.uniform_batch(batch, n, seed=n + 3)
    with F.Plan((n,), batch) as p:
        assert p.describe().startswith("generic"), p.describe()
    for d in (-1, +1):
        y = run((n,), batch, x, d)
        assert max_rel_l2(y, oracle.fft(x, d), -1) <= TOL_FP32, (n, d)


def test_large_batch_sampled(torch):
    # 2^24 elements of 768-point lines (the timed size), 16 sampled transforms
    n, batch = 768, (1 << 24) // 768
    x = inputs.normal_batch(batch, n, seed=11)
    rows = np.random.default_rng(5).choice(batch, 16, replace=False)
    for d in (-1, +1):
        y = run((n,), batch, x, d)
        assert max_rel_l2(y[rows], oracle.fft(x[rows], d), -1) <= TOL_FP32, d


FOURSTEP = [m << k for m, k0, k1 in ((3, 11, 19), (5, 10, 18), (7, 10, 18)) for k in range(k0, k1 + 1)]


@pytest.mark.parametrize("n", FOURSTEP)
def test_mixed_fourstep_every_length(torch, n):
    # N = (M * 2^a) * 2^b: compile-time column kernel, then power-of-two transposed rows
    batch = 3 if n <= (1 << 16) else 1
    x = inputs.normal_batch(batch, n, seed=n % 9973)
    with F.Plan((n,), batch) as p:
        assert p.describe().startswith("fourstep-mixed"), p.describe()
    for d in (-1, +1):
        y = run((n,), batch, x, d)
        assert max_rel_l2(y, oracle.fft(x, d), -1) <= TOL_FP32, (n, d)


@pytest.mark.parametrize("n", [6144, 7 * 2 ** 14])
def test_mixed_fourstep_in_place(torch, n):
    batch = 2
    x = inputs.uniform_batch(batch, n, seed=n % 991)
    for d in (-1, +1):
        y = run((n,), batch, x, d, inplace=True)
        assert max_rel_l2(y, oracle.fft(x, d), -1) <= TOL_FP32, (n, d)


@pytest.mark.parametrize("n", [3 * 2 ** 20, 5 * 2 ** 19])
def test_beyond_column_kernels_falls_back(torch, n):
    # N1 would exceed 512 points: the stage-graph executor takes the length
    with F.Plan((n,), 1) as p:
        assert p.describe().startswith("generic"), p.describe()
    x = inputs.normal_batch(1, n, seed=3)
    y = run((n,), 1, x, -1)
    assert max_rel_l2(y, oracle.fft(x, -1), -1) <= TOL_FP32


@pytest.mark.parametrize("h,w,batch", [(768, 1024, 2), (1024, 768, 2), (96, 160, 5), (3, 64, 7), (5, 7 * 32, 3),
                                       (3072, 512, 1), (448, 3584, 1), (2048, 5 * 128, 1), (4096, 3072, 1)])
def test_2d_with_mixed_sides(torch, h, w, batch):
    rng = np.random.default_rng(h * 7 + w)
    x = (rng.standard_normal((batch, h, w)) + 1j * rng.standard_normal((batch, h, w))).astype(np.complex64)
    with F.Plan((h, w), batch) as p:
        assert p.describe().startswith("2d-mixed"), p.describe()
    for d in (-1, +1):
        y = run((h, w), batch, x, d)
        assert max_rel_l2(y.reshape(batch, -1), oracle.fft2(x, d).reshape(batch, -1), -1) <= TOL_FP32, (h, w, d)


def test_2d_mixed_in_place(torch):
    h, w, batch = 320, 96, 3
    x = inputs.uniform_batch(batch * h, w, seed=9).reshape(batch, h, w)
    for d in (-1, +1):
        y = run((h, w), batch, x, d, inplace=True)
        assert max_rel_l2(y.reshape(batch, -1), oracle.fft2(x, d).reshape(batch, -1), -1) <= TOL_FP32, d


@pytest.mark.parametrize("h,w", [(7, 5), (9, 64), (64, 11)])
def test_2d_sides_outside_the_column_kernels(torch, monkeypatch, h, w):
    # 7 x 5: a 7-point column tile holds 32 columns and 5 is not a multiple;
    # 9 and 11 are not M * 2^K: no in-place 2-D plan, so the general
    # (transposing) plan takes them, and without it FFT_ERR_UNSUPPORTED
    with F.Plan((h, w), 1) as p:
        assert p.describe().startswith("2d-transpose"), p.describe()
    monkeypatch.setenv("B300FFT_2D_TRANSPOSE", "0")
    assert F.fft_plan_create(2, [h, w], 1, 0) is None
    assert F.fft_last_error() == F.FFT_ERR_UNSUPPORTED
