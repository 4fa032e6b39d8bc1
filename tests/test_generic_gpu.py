"""Parity of the mixed-radix, Bluestein and ragged paths with the FP64 oracle
(needs a GPU).  Bar: per-transform relative L2 error <= 1e-6."""
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


def ref_bins(x, sign, nbins=48, seed=0):
    """Oracle for one long transform: selected bins only (O(N) each)."""
    n = x.shape[-1]
    ks = np.unique(np.concatenate([[0, 1, n - 1, n // 2],
                                   np.random.default_rng(seed).integers(0, n, nbins)]))
    return ks, oracle.dft_bins(x, ks, sign)


def bins_rel_err(y, ks, vals):
    return float(np.linalg.norm(y[ks] - vals) / np.linalg.norm(vals))


@pytest.mark.parametrize("n", [1, 3, 5, 6, 7, 9, 12, 15, 21, 25, 35, 48, 49, 80, 96, 112, 320, 448, 768,
                               1000, 1536, 2560, 3072, 3584, 4000, 4032])
@pytest.mark.parametrize("batch", [1, 7])
def test_mixed_radix_single_tile(torch, n, batch):
    x = inputs.uniform_batch(batch, n, seed=n + batch)
    for d in (-1, +1):
        y = run((n,), batch, x, d)
        assert max_rel_l2(y, oracle.fft(x, d), -1) <= TOL_FP32, (n, batch, d)


@pytest.mark.parametrize("n", [3 * 2 ** 12, 5 * 2 ** 12, 7 * 2 ** 13, 3 * 2 ** 14, 3 ** 9, 5 ** 6, 6000, 7 * 2 ** 16])
def test_mixed_radix_four_step(torch, n):
    batch = 2
    x = inputs.normal_batch(batch, n, seed=n % 1000)
    for d in (-1, +1):
        y = run((n,), batch, x, d)
        assert max_rel_l2(y, oracle.fft(x, d), -1) <= TOL_FP32, (n, d)


@pytest.mark.parametrize("n", [11, 13, 22, 97, 101, 143, 1009, 2003, 2053, 4099])
def test_bluestein(torch, n):
    batch = 3
    x = inputs.uniform_batch(batch, n, seed=n)
    for d in (-1, +1):
        y = run((n,), batch, x, d)
        ref = oracle.dft_naive(x, d)
        assert max_rel_l2(y, ref, -1) <= TOL_FP32, (n, d)


@pytest.mark.parametrize("n", [30011, 65521])
def test_bluestein_large_sampled(torch, n):
    x = inputs.uniform_batch(1, n, seed=n)
    for d in (-1, +1):
        y = run((n,), 1, x, d)[0]
        ks, vals = ref_bins(x[0], d)
        assert bins_rel_err(y, ks, vals) <= TOL_FP32, (n, d)
        # whole-transform property check: Parseval
        e_in = np.sum(np.abs(x[0].astype(np.complex128)) ** 2)
        e_out = np.sum(np.abs(y.astype(np.complex128)) ** 2)
        assert abs(e_out - n * e_in) <= 4 * TOL_FP32 * n * e_in


def _ragged_check(torch, lengths, data, per_size, d, full_limit=20000):
    from paper_1203_4938_b300 import fft as F
    offs = np.zeros(len(lengths) + 1, np.int64)
    np.cumsum(lengths, out=offs[1:])
    with F.Ragged(lengths) as p:
        xd = to_dev(data)
        y = (p.exec_per_size(xd, None, d) if per_size else p.exec(xd, None, d))
        torch.cuda.synchronize()
        p.check()
        yh = y.cpu().numpy()
    worst = 0.0
    for t, n in enumerate(lengths):
        xs, ys = data[offs[t]:offs[t + 1]], yh[offs[t]:offs[t + 1]]
        if n <= full_limit:
            e = max_rel_l2(ys[None], oracle.fft(xs[None], d), -1)
        else:
            ks, vals = ref_bins(xs, d, nbins=16, seed=t)
            e = bins_rel_err(ys, ks, vals)
        worst = max(worst, e)
    return worst


@pytest.mark.parametrize("per_size", [False, True])
def test_ragged_small_mix(torch, per_size):
    lengths, _ = inputs.ragged_lengths(count=160, seed=11)
    lengths = [int(v) for v in lengths]
    data = np.random.default_rng(3).uniform(-1, 1, 2 * sum(lengths)).astype(np.float32).view(np.complex64)
    for d in (-1, +1):
        assert _ragged_check(torch, lengths, data, per_size, d) <= TOL_FP32


@pytest.mark.parametrize("env", [{}, {"B300FFT_G_POW2T": "0"}, {"B300FFT_G_LAG": "1"}, {"B300FFT_G_LAG": "100000"},
                                 {"B300FFT_G_SPLIT": "0"}, {"B300FFT_G_LEAN": "0"}, {"B300FFT_GRAPH": "0"},
                                 {"B300FFT_G_MIXT": "0"}])
def test_ragged_pow2_templated_stages(torch, monkeypatch, env):
    """Power-of-two lengths 2^13..2^16 inside a ragged batch run as templated
    four-step stages (or, with B300FFT_G_POW2T=0, as runtime-radix stages) in
    a launch of the lean executor after the other transforms, with the other
    compile-time tiles (B300FFT_G_SPLIT=0 or B300FFT_G_LEAN=0: one launch of
    the full executor); the persistent
    queue lags each transform's second stage (B300FFT_G_LAG items, 1 = right
    behind).  Every transform is compared in full."""
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    lengths = [8192, 16384, 32768, 65536, 3 * 2 ** 13, 8192, 65536, 100, 4096, 16384, 2 ** 13, 7 * 2 ** 12, 1009]
    data = np.random.default_rng(21).standard_normal(2 * sum(lengths)).astype(np.float32).view(np.complex64)
    with F.Ragged(lengths) as p:
        # the 4096-point line and the 3 * 2^13 four-step stay compile-time tiles
        # whichever of the templated-tile switches is off, so the plan splits
        # unless the lean launch itself is switched off
        split = env.get("B300FFT_G_SPLIT", "1") != "0" and env.get("B300FFT_G_LEAN", "1") != "0"
        assert ("+lean launch" in p.describe()) == split, p.describe()
    for per_size in (False, True):
        for d in (-1, +1):
            assert _ragged_check(torch, lengths, data, per_size, d, full_limit=70000) <= TOL_FP32, (env, per_size, d)


@pytest.mark.parametrize("env", [{}, {"B300FFT_G_MIXSPLIT": "0"}, {"B300FFT_G_MIXT": "0"}])
def test_ragged_mixed_fourstep_transposed_rows(torch, monkeypatch, env):
    """M * 2^k four-steps in the stage graph.  Default: the batched mixed
    four-step's split (6144 = 12 x 512, 20480 = 80 x 256, ...: short mixed
    columns, long power-of-two rows).  With the balanced split
    (B300FFT_G_MIXSPLIT=0) the second stage has 64 or 128 points and a row
    count the fixed 256-thread tile does not divide (5120 = 80 x 64, 6144 =
    96 x 64, 7168 = 112 x 64, 10240 = 80 x 128, ...): the compile-time
    transposed-row tile with a partial last tile; with the compile-time tiles
    off, runtime tiles.  Every transform compared in full."""
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    lengths = [5120, 6144, 7168, 10240, 14336, 6144, 100, 4099, 20480, 3 * 2 ** 15]
    data = np.random.default_rng(23).standard_normal(2 * sum(lengths)).astype(np.float32).view(np.complex64)
    for per_size in (False, True):
        for d in (-1, +1):
            assert _ragged_check(torch, lengths, data, per_size, d, full_limit=100000) <= TOL_FP32, (env, per_size, d)


def test_ragged_all_lean(torch, monkeypatch):
    """A ragged batch of power-of-two lengths 2^13..2^16 only runs in the lean
    executor alone (one launch)."""
    lengths = [8192, 65536, 16384, 32768, 8192, 65536, 16384]
    data = np.random.default_rng(22).standard_normal(2 * sum(lengths)).astype(np.float32).view(np.complex64)
    with F.Ragged(lengths) as p:
        assert " lean " in p.describe(), p.describe()
    for per_size in (False, True):
        for d in (-1, +1):
            assert _ragged_check(torch, lengths, data, per_size, d, full_limit=70000) <= TOL_FP32, (per_size, d)


def test_ragged_edge_lengths(torch):
    lengths = [1, 2, 3, 4096, 4097, 17, 65536, 64, 5, 7 * 2 ** 13, 1, 2053]
    data = np.random.default_rng(5).standard_normal(2 * sum(lengths)).astype(np.float32).view(np.complex64)
    for per_size in (False, True):
        assert _ragged_check(torch, lengths, data, per_size, -1) <= TOL_FP32


def test_ragged_graph_capture_by_caller(torch):
    """fft_exec inside the caller's stream capture launches the persistent
    kernel directly (not the plan's own graph) and replays correctly."""
    from paper_1203_4938_b300 import fft as F
    lengths = [64, 96, 1000, 4096, 12288, 131]
    data = np.random.default_rng(6).uniform(-1, 1, 2 * sum(lengths)).astype(np.float32).view(np.complex64)
    ref = np.concatenate([oracle.fft(data[a:a + n], -1) for a, n in
                          zip(np.concatenate([[0], np.cumsum(lengths)[:-1]]), lengths)])
    with F.Ragged(lengths) as p:
        xd = to_dev(data)
        out = torch.empty_like(xd)
        p.exec(xd, out)  # first exec outside capture builds the plan's graph
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        out2 = torch.empty_like(xd)
        with torch.cuda.graph(g):
            p.exec(xd, out2)
        g.replay()
        g.replay()
        torch.cuda.synchronize()
        assert max_rel_l2(out2.cpu().numpy()[None], ref[None], -1) <= TOL_FP32


def test_ragged_autotuned_tiles_and_cache(torch, monkeypatch, tmp_path):
    """FFT_AUTOTUNE=1 times candidate tile shapes per length; the choice is
    written to FFT_TUNE_CACHE and the plan is still exact to 1e-6."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("FFT_AUTOTUNE", "1")
    monkeypatch.setenv("FFT_TUNE_CACHE", str(cache))
    lengths = [96, 640, 4096, 7 * 2 ** 11, 3 * 2 ** 13, 65536, 1024, 96, 101]
    data = np.random.default_rng(8).uniform(-1, 1, 2 * sum(lengths)).astype(np.float32).view(np.complex64)
    for per_size in (False, True):
        assert _ragged_check(torch, lengths, data, per_size, -1) <= TOL_FP32
    text = cache.read_text().split()
    assert len(text) >= 6 and any(t.endswith(":65536") for t in text)
