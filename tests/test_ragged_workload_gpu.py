"""The ragged workload at its stated size, against the FP64 oracle (GPU).

10,000 one-dimensional transforms with lengths drawn by
``inputs.ragged_lengths(10000, seed=4)`` (powers of two 2^6..2^16, 3/5/7 * 2^k,
about 1 % primes through Bluestein), packed back to back (about 9.47e7
complex64 elements), uniform[-1, 1] data from the same generator: the "flow of
many DFTs" of Sec. III-A with uneven lengths.  The plan runs as one persistent
launch replayed from its CUDA graph, in both directions, and once as one
launch per (stage, length) group.  Every transform is checked: the full
oracle FFT for every composite length, the O(N^2) definition for primes up to
4096 points, and 24 bins from the definition for longer primes.  Bar: the FP32
tolerance, 1e-6 relative L2 per transform (max over all 10,000)."""
import numpy as np
import pytest

import oracle
from paper_1203_4938_b300 import fft as F
from paper_1203_4938_b300 import inputs
from tests.gpu_util import TOL_FP32, cuda_or_skip, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


def _is_prime(n: int) -> bool:
    if n < 2:
        return False
    i = 2
    while i * i <= n:
        if n % i == 0:
            return False
        i += 1
    return True


def worst_error(lengths, offsets, data, y, sign):
    """Max per-transform relative L2 error of y against the oracle."""
    groups = {}
    for t, n in enumerate(lengths):
        groups.setdefault(int(n), []).append(t)
    worst, where = 0.0, None
    for n, ts in groups.items():
        xs = np.stack([data[offsets[t]:offsets[t + 1]] for t in ts])
        ys = np.stack([y[offsets[t]:offsets[t + 1]] for t in ts]).astype(np.complex128)
        if _is_prime(n) and n > 4096:
            ks = np.unique(np.concatenate([[0, 1, n - 1, n // 2], np.random.default_rng(n).integers(0, n, 20)]))
            for j in range(len(ts)):
                vals = oracle.dft_bins(xs[j], ks, sign)
                e = float(np.linalg.norm(ys[j][ks] - vals) / np.linalg.norm(vals))
                if e > worst:
                    worst, where = e, (ts[j], n)
            continue
        ref = oracle.dft_naive(xs, sign) if _is_prime(n) else oracle.fft(xs, sign)
        e = np.sqrt(np.sum(np.abs(ys - ref) ** 2, -1)) / np.sqrt(np.sum(np.abs(ref) ** 2, -1))
        j = int(np.argmax(e))
        if e[j] > worst:
            worst, where = float(e[j]), (ts[j], n)
    return worst, where


def test_ragged_workload_full_size(torch):
    lengths, offsets, data = inputs.ragged_workload(10000, seed=4)
    lens = [int(v) for v in lengths]
    assert len(lens) == 10000 and int(offsets[-1]) > 9e7
    with F.Ragged(lens) as p:
        xd = to_dev(data)
        out = torch.empty_like(xd)
        for sign in (-1, +1):
            p.exec(xd, out, sign)
            torch.cuda.synchronize()
            p.check()
            e, where = worst_error(lens, offsets, data, out.cpu().numpy(), sign)
            assert e <= TOL_FP32, ("persistent", sign, e, where)
        out.fill_(float("nan"))
        p.exec_per_size(xd, out, -1)
        torch.cuda.synchronize()
        p.check()
        e, where = worst_error(lens, offsets, data, out.cpu().numpy(), -1)
        assert e <= TOL_FP32, ("per-size", e, where)


def test_ragged_executor_wait_timeout_is_reported(torch, monkeypatch):
    """A transform whose first stage never signals its counter (test-only
    B300FFT_DEBUG_WITHHOLD_XF) makes the bounded waits of its later stages
    expire: the persistent executor returns, the plan reports FFT_ERR_TIMEOUT
    (then clears the word), and a plan built afterwards is exact.  Both a
    four-step length (2^16: two stages) and a Bluestein length (1009: a chain
    of three stages) are withheld in turn."""
    lengths = [65536, 1009, 4096, 96, 3 * 2 ** 13, 100]
    data = np.random.default_rng(31).uniform(-1, 1, 2 * sum(lengths)).astype(np.float32).view(np.complex64)
    offs = np.concatenate([[0], np.cumsum(lengths)])
    xd = to_dev(data)
    monkeypatch.setenv("B300FFT_SPIN_LIMIT", "20000")
    for victim in (0, 1):
        monkeypatch.setenv("B300FFT_DEBUG_WITHHOLD_XF", str(victim))
        with F.Ragged(lengths) as p:
            p.exec(xd, None, -1)
            torch.cuda.synchronize()
            assert F.fft_plan_check(p.handle) == F.FFT_ERR_TIMEOUT, victim
            assert F.fft_plan_check(p.handle) == F.FFT_OK
    monkeypatch.delenv("B300FFT_DEBUG_WITHHOLD_XF")
    monkeypatch.delenv("B300FFT_SPIN_LIMIT")
    with F.Ragged(lengths) as p:
        y = p.exec(xd, None, -1)
        torch.cuda.synchronize()
        p.check()
        yh = y.cpu().numpy()
    for t, n in enumerate(lengths):
        xs = data[offs[t]:offs[t + 1]][None]
        ref = oracle.dft_naive(xs, -1) if n == 1009 else oracle.fft(xs, -1)
        e = np.linalg.norm(yh[offs[t]:offs[t + 1]] - ref[0]) / np.linalg.norm(ref[0])
        assert e <= TOL_FP32, (n, e)
