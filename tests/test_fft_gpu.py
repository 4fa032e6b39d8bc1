"""Parity of the FP32 CUDA path with the FP64 oracle (needs a GPU).

Each case runs the kernels through the C ABI on seeded synthetic input and
compares every transform with the oracle: the bar is a per-transform
relative L2 error <= 1e-6 (max over the batch), in FP64."""
import numpy as np
import pytest

import oracle
from paper_1203_4938_b300 import inputs
from tests.gpu_util import TOL_FP32, cuda_or_skip, max_rel_l2, run, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


# ---------------------------------------------------------------- 1-D pow2
@pytest.mark.parametrize("logn", list(range(0, 15)))
@pytest.mark.parametrize("batch", [1, 7, 37])
def test_rows_single_pass(torch, logn, batch):
    n = 1 << logn
    x = inputs.uniform_batch(batch, n, seed=logn * 100 + batch)
    for d in (-1, +1):
        y = run((n,), batch, x, d)
        ref = oracle.fft(x, d)
        assert max_rel_l2(y, ref, -1) <= TOL_FP32, (n, batch, d)


@pytest.mark.parametrize("logn", [13, 14, 15, 16, 17, 18, 19, 20])
def test_fourstep(torch, logn):
    n = 1 << logn
    batch = 3 if logn <= 18 else 2
    x = inputs.normal_batch(batch, n, seed=logn)
    for d in (-1, +1):
        y = run((n,), batch, x, d)
        ref = oracle.fft(x, d)
        assert max_rel_l2(y, ref, -1) <= TOL_FP32, (n, d)


@pytest.mark.parametrize("logn", [21, 22, 23, 24])
def test_fourstep_large(torch, logn):
    n = 1 << logn
    x = inputs.normal_batch(1, n, seed=logn)
    y = run((n,), 1, x, -1)
    ref = oracle.fft(x, -1)
    assert max_rel_l2(y, ref, -1) <= TOL_FP32


@pytest.mark.parametrize("staged", ["0", "1"])
@pytest.mark.parametrize("logn", [13, 14])
@pytest.mark.parametrize("batch", [1, 7, 300])
def test_rows_staged_and_plain(torch, monkeypatch, staged, logn, batch):
    """2^13 / 2^14 rows, both the plain one-CTA-per-transform kernel and the
    persistent form that bulk-copies the next row into shared memory (batch
    300 > grid: every CTA runs several staged rows, some one more than
    others)."""
    monkeypatch.setenv("B300FFT_ROWS_STAGED", staged)
    n = 1 << logn
    x = inputs.normal_batch(batch, n, seed=logn * 7 + batch)
    for d in (-1, +1):
        y = run((n,), batch, x, d)
        assert max_rel_l2(y, oracle.fft(x, d), -1) <= TOL_FP32, (logn, batch, staged, d)
    y = run((n,), batch, x, -1, inplace=True)
    assert max_rel_l2(y, oracle.fft(x, -1), -1) <= TOL_FP32, (logn, batch, staged, "in place")


def test_config_small_uniform_1024x64(torch):
    """N=1024, batch 64, uniform[-1,1] from seed 0, forward."""
    x = inputs.uniform_batch(64, 1024, seed=0)
    y = run((1024,), 64, x, -1)
    err = max_rel_l2(y, oracle.fft(x, -1), -1)
    assert err <= TOL_FP32, err


@pytest.mark.parametrize("logn", [4, 10, 12, 16, 20])
def test_round_trip(torch, logn):
    n = 1 << logn
    x = inputs.normal_batch(2, n, seed=7)
    y = run((n,), 2, run((n,), 2, x, -1), +1) / n
    assert max_rel_l2(y, x, -1) <= 2 * TOL_FP32


@pytest.mark.parametrize("logn", [6, 12, 18])
def test_in_place(torch, logn):
    n = 1 << logn
    x = inputs.uniform_batch(5, n, seed=11)
    y = run((n,), 5, x, -1, inplace=True)
    assert max_rel_l2(y, oracle.fft(x, -1), -1) <= TOL_FP32


def test_impulse_exact_ones(torch):
    """delta -> all ones: every butterfly only adds zeros, so FP32 is exact."""
    for logn in (3, 8, 12, 16):
        n = 1 << logn
        x = np.zeros((2, n), np.complex64)
        x[:, 0] = 1
        y = run((n,), 2, x, -1)
        assert np.array_equal(y, np.ones_like(y)), n


def test_large_batch_tiny_n(torch):
    x = inputs.uniform_batch(1 << 18, 2, seed=5)
    y = run((2,), 1 << 18, x, -1)
    assert max_rel_l2(y, oracle.fft(x, -1), -1) <= TOL_FP32


# ---------------------------------------------------------------- 2-D
@pytest.mark.parametrize("h,w,b", [(2, 2, 1), (16, 64, 3), (64, 16, 2), (256, 512, 2), (1024, 1024, 1),
                                   (4096, 64, 1), (32, 8192, 1), (512, 512, 5), (2048, 2048, 2)])
def test_2d(torch, h, w, b):
    rng = np.random.default_rng(h * 7 + w)
    x = inputs.image_batch(rng, b, h, w)
    for d in (-1, +1):
        y = run((h, w), b, x, d)
        ref = oracle.fft2(x, d)
        assert max_rel_l2(y.reshape(b, -1), ref.reshape(b, -1), -1) <= TOL_FP32, (h, w, d)


# ---------------------------------------------------------------- ABI on GPU
def test_misaligned_pointer(torch):
    from paper_1203_4938_b300 import fft as F
    with F.Plan((64,), 4) as p:
        buf = torch.zeros(64 * 4 + 2, dtype=torch.complex64, device="cuda")
        base = buf.data_ptr()
        assert F.fft_exec(p.handle, base + 8, base, F.FFT_FORWARD) == F.FFT_ERR_MISALIGNED
        assert F.fft_exec(p.handle, base, base + 8, F.FFT_FORWARD) == F.FFT_ERR_MISALIGNED
        assert F.fft_exec(p.handle, base, base, 0) == F.FFT_ERR_INVALID_ARG
        assert F.fft_exec(p.handle, 0, base, F.FFT_FORWARD) == F.FFT_ERR_INVALID_ARG


def test_exec_after_destroy(torch):
    from paper_1203_4938_b300 import fft as F
    h = F.fft_plan_create(1, [256], 2, 0)
    assert h
    assert F.fft_plan_destroy(h) == F.FFT_OK
    buf = torch.zeros(512, dtype=torch.complex64, device="cuda")
    assert F.fft_exec(h, buf.data_ptr(), buf.data_ptr(), -1) == F.FFT_ERR_BAD_HANDLE
    assert F.fft_plan_destroy(h) == F.FFT_ERR_BAD_HANDLE


def test_workspace_and_description(torch):
    from paper_1203_4938_b300 import fft as F
    with F.Plan((4096,), 3) as p:
        assert p.workspace_bytes == 0 and p.kernel_count == 1
        assert "rows" in p.describe()
    with F.Plan((1 << 16,), 3) as p:
        assert p.workspace_bytes == (1 << 16) * 3 * 8 and p.kernel_count in (1, 2)
        assert "fourstep" in p.describe()


def test_side_stream_and_graph_capture(torch):
    from paper_1203_4938_b300 import fft as F
    n, b = 1 << 14, 4
    x = inputs.uniform_batch(b, n, seed=3)
    ref = oracle.fft(x, -1)
    for shape in [(n,), (1 << 16,)]:
        nn = shape[0]
        xx = inputs.uniform_batch(b, nn, seed=4)
        rr = oracle.fft(xx, -1)
        with F.Plan(shape, b) as p:
            d = to_dev(xx)
            out = torch.empty_like(d)
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                p.exec(d, out)
            torch.cuda.current_stream().wait_stream(s)
            torch.cuda.synchronize()
            assert max_rel_l2(out.cpu().numpy(), rr, -1) <= TOL_FP32
            g = torch.cuda.CUDAGraph()
            out2 = torch.empty_like(d)
            with torch.cuda.graph(g):
                p.exec(d, out2)
            for _ in range(3):
                g.replay()
            torch.cuda.synchronize()
            assert max_rel_l2(out2.cpu().numpy(), rr, -1) <= TOL_FP32
    del ref


# ---------------------------------------------------------------- plan variants
@pytest.mark.parametrize("logn,env", [
    (13, {"B300FFT_SINGLE_MAX_LOG": "12"}),                       # two-launch four-step
    (14, {"B300FFT_SINGLE_MAX_LOG": "12"}),
    (16, {"B300FFT_PERSIST": "0"}),                              # two-launch instead of persistent
    (16, {"B300FFT_PIPE": "0"}),                                 # persistent kernel with plain loads
    # two-pass persistent tiles of 16384 points on 1024 threads (one CTA per SM)
    (16, {"B300FFT_PERSIST_CFG": "8,64,8,64"}),
    (17, {"B300FFT_PERSIST_CFG": "8,64,9,32"}),
    (18, {"B300FFT_PERSIST_CFG": "8,64,10,16", "B300FFT_CHUNK_MB": "2"}),
    (18, {"B300FFT_PERSIST_CFG": "9,32,9,32"}),
    (19, {"B300FFT_PERSIST_CFG": "9,32,10,16"}),
    (20, {"B300FFT_PERSIST_CFG": "10,16,10,16", "B300FFT_CHUNK_MB": "64"}),
    (21, {}),                                                    # 2^10 x 2^11 with 16384-point tiles (default)
    (21, {"B300FFT_PERSIST_CFG": "11,8,10,16", "B300FFT_CHUNK_MB": "4"}),
    (21, {"B300FFT_PERSIST_CFG": "10,8,11,4"}),
    (22, {"B300FFT_THREE": "0", "B300FFT_PERSIST_CFG": "11,8,11,8"}),
    # persistent four-step fed by tensor-memory-accelerator copies (ring of 2 or 3 slots)
    (15, {"B300FFT_PIPE": "2"}),
    (15, {"B300FFT_PIPE": "3", "B300FFT_PERSIST_CFG": "8,16,7,32"}),
    (16, {"B300FFT_PIPE": "3", "B300FFT_CHUNK_MB": "1"}),        # many chunks, ragged last chunk
    (16, {"B300FFT_PIPE": "2", "B300FFT_CHUNK_MB": "64"}),       # one chunk: B tiles wait on A tiles
    (17, {"B300FFT_PIPE": "2"}),
    (18, {"B300FFT_PIPE": "3", "B300FFT_PERSIST_CFG": "9,8,9,8"}),
    (19, {"B300FFT_PIPE": "3", "B300FFT_PERSIST_CFG": "9,8,10,4"}),
    (19, {"B300FFT_PIPE": "2"}),
    (20, {"B300FFT_PIPE": "3", "B300FFT_PERSIST_CFG": "10,4,10,4"}),
    (20, {"B300FFT_PIPE": "2", "B300FFT_PERSIST_CFG": "10,4,10,4", "B300FFT_CHUNK_MB": "4"}),
    (20, {"B300FFT_PIPE": "0"}),
    (20, {"B300FFT_PERSIST": "0"}),
    (17, {"B300FFT_CHUNK_MB": "1"}),                             # many chunks, ragged last chunk
    (18, {"B300FFT_PERSIST_CFG": "9,8,9,8", "B300FFT_CHUNK_MB": "3"}),
    (18, {"B300FFT_PERSIST_CFG": "9,8,9,8", "B300FFT_CHUNK_MB": "64"}),  # one chunk: B tiles wait on A tiles
    (22, {"B300FFT_PERSIST_CFG": "11,4,11,4", "B300FFT_CHUNK_MB": "16"}),
    # thread-block-cluster single pass (N = K * M on K CTAs, DSMEM exchanges)
    (15, {"B300FFT_CLUSTER": "1", "B300FFT_CLUSTER_CFG": "12,8"}),
    (16, {"B300FFT_CLUSTER": "1", "B300FFT_CLUSTER_CFG": "13,8"}),
    (16, {"B300FFT_CLUSTER": "1", "B300FFT_CLUSTER_CFG": "12,16"}),
    (17, {"B300FFT_CLUSTER": "1", "B300FFT_CLUSTER_CFG": "14,8"}),
    (17, {"B300FFT_CLUSTER": "1", "B300FFT_CLUSTER_CFG": "13,16"}),
    # three-stage persistent kernel (N = N1 * M1 * M2)
    (19, {"B300FFT_THREE": "1", "B300FFT_THREE_CFG": "6,6,7", "B300FFT_CHUNK_MB": "4"}),   # many chunks
    (19, {"B300FFT_THREE": "1", "B300FFT_THREE_CFG": "6,6,7", "B300FFT_CHUNK_MB": "64"}),  # one chunk
    (20, {"B300FFT_THREE": "1", "B300FFT_THREE_CFG": "7,7,6"}),
    (20, {"B300FFT_THREE": "1", "B300FFT_THREE_CFG": "6,7,7", "B300FFT_THREE_LOOKAHEAD": "1"}),
    (21, {"B300FFT_THREE": "1", "B300FFT_THREE_CFG": "7,7,7", "B300FFT_CHUNK_MB": "40"}),
    (22, {"B300FFT_THREE": "1", "B300FFT_THREE_CFG": "7,7,8"}),
    (22, {"B300FFT_THREE": "0"}),                                # two-pass persistent instead
    (23, {"B300FFT_THREE": "1", "B300FFT_THREE_CFG": "8,7,8"}),
    (23, {"B300FFT_THREE": "1", "B300FFT_THREE_CFG": "7,8,8", "B300FFT_THREE_LOOKAHEAD": "64"}),
    (22, {"B300FFT_THREE": "0", "B300FFT_PERSIST_CFG": "10,16,12,4"}),   # 128-byte first-pass segments
    (23, {"B300FFT_THREE": "0", "B300FFT_PERSIST_CFG": "11,8,12,4"}),
    (24, {"B300FFT_THREE": "1", "B300FFT_THREE_CFG": "8,8,8"}),
    (24, {"B300FFT_THREE": "0"}),
])
def test_fourstep_variants(torch, monkeypatch, logn, env):
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    n = 1 << logn
    batch = 5 if logn <= 21 else 2
    x = inputs.normal_batch(batch, n, seed=logn + 50)
    for d in (-1, +1):
        y = run((n,), batch, x, d)
        assert max_rel_l2(y, oracle.fft(x, d), -1) <= TOL_FP32, (logn, env, d)


@pytest.mark.parametrize("cfg", [None, "8,8,8,8", "three", "pipe2"])
def test_persistent_wait_timeout_is_reported(torch, monkeypatch, cfg):
    """A chunk counter that nothing ever completes makes the bounded waits of
    the second-pass tiles expire: the kernel returns, the plan reports
    FFT_ERR_TIMEOUT, and the device stays usable for the next plan (default
    four-step tiles, 128-thread tiles and the three-stage kernel)."""
    from paper_1203_4938_b300 import fft as F
    n, b = 1 << 16, 8
    x = to_dev(inputs.uniform_batch(b, n, seed=9))
    if cfg == "three":
        n = 1 << 19
        x = to_dev(inputs.uniform_batch(b, n, seed=9))
        monkeypatch.setenv("B300FFT_THREE", "1")
        monkeypatch.setenv("B300FFT_THREE_CFG", "6,6,7")
    elif cfg == "pipe2":
        monkeypatch.setenv("B300FFT_PIPE", "2")
    elif cfg:
        monkeypatch.setenv("B300FFT_PERSIST_CFG", cfg)
    monkeypatch.setenv("B300FFT_DEBUG_WITHHOLD_CHUNK", "0")
    monkeypatch.setenv("B300FFT_SPIN_LIMIT", "20000")
    monkeypatch.setenv("B300FFT_CHUNK_MB", "1")
    with F.Plan((n,), b) as p:
        assert ("threestep" if cfg == "three" else "persist") in p.describe()
        p.forward(x)
        torch.cuda.synchronize()
        assert F.fft_plan_check(p.handle) == F.FFT_ERR_TIMEOUT
        assert F.fft_plan_check(p.handle) == F.FFT_OK  # the word is cleared
    monkeypatch.delenv("B300FFT_DEBUG_WITHHOLD_CHUNK")
    monkeypatch.delenv("B300FFT_SPIN_LIMIT")
    with F.Plan((n,), b) as p:
        y = p.forward(x)
        torch.cuda.synchronize()
        p.check()
        ref = oracle.fft(x.cpu().numpy(), -1)
        assert max_rel_l2(y.cpu().numpy(), ref, -1) <= TOL_FP32


@pytest.mark.parametrize("cfg", ["12,8", "13,16"])
def test_cluster_in_place_and_round_trip(torch, monkeypatch, cfg):
    """Cluster kernel writing over its own input (every CTA of a cluster loads
    its chunk before any CTA stores), then the inverse back."""
    from paper_1203_4938_b300 import fft as F
    lm, k = (int(v) for v in cfg.split(","))
    n = k << lm
    monkeypatch.setenv("B300FFT_CLUSTER", "1")
    monkeypatch.setenv("B300FFT_CLUSTER_CFG", cfg)
    x = inputs.uniform_batch(3, n, seed=77)
    with F.Plan((n,), 3) as p:
        assert "cluster" in p.describe()
        d = to_dev(x)
        p.forward(d, d)
        torch.cuda.synchronize()
        assert max_rel_l2(d.cpu().numpy(), oracle.fft(x, -1), -1) <= TOL_FP32
        p.inverse(d, d)
        torch.cuda.synchronize()
        assert max_rel_l2(d.cpu().numpy() / n, x, -1) <= 2 * TOL_FP32


@pytest.mark.parametrize("side,b,env", [
    (512, 7, {"B300FFT_CHUNK_MB": "1"}),                    # one image per chunk, ragged tail
    (1024, 3, {"B300FFT_2D_CFG": "16,16"}),
    (2048, 3, {"B300FFT_2D_CFG": "4,4", "B300FFT_CHUNK_MB": "64"}),  # one chunk
    (2048, 2, {"B300FFT_PERSIST": "0"}),                    # two-launch form
])
def test_2d_persistent_variants(torch, monkeypatch, side, b, env):
    from paper_1203_4938_b300 import fft as F
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    x = inputs.image_batch(np.random.default_rng(side + b), b, side, side)
    with F.Plan((side, side), b) as p:
        want = "2d H=" if env.get("B300FFT_PERSIST") == "0" else "2d-persist"
        assert want in p.describe(), p.describe()
    for d in (-1, +1):
        y = run((side, side), b, x, d)
        ref = oracle.fft2(x, d)
        assert max_rel_l2(y.reshape(b, -1), ref.reshape(b, -1), -1) <= TOL_FP32, (side, env, d)


def test_2d_in_place(torch):
    x = inputs.image_batch(np.random.default_rng(11), 2, 1024, 1024)
    y = run((1024, 1024), 2, x, -1, inplace=True)
    assert max_rel_l2(y.reshape(2, -1), oracle.fft2(x, -1).reshape(2, -1), -1) <= TOL_FP32
