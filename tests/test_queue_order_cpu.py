"""Queue order of the persistent kernels, checked on the host (no GPU).

tests/queue_order_check.cu includes the kernels' own queue decoders
(decode_item for the two-pass four-step, three_decode for the three-stage
form) and checks, for every queue position of a parameter set, that the
decoder is a bijection onto the tiles and that every tile that waits comes
after all the tiles it waits for.  With one item per CTA at a time and
signals published before any wait, that is what makes every bounded wait of
those kernels end (Sec. III-A's split N = N1 * N2 run as one launch).

The parameter sets are the ones the planner derives for the benchmark sweep
(2^26 elements per length, the measured shape tables) plus edge cases:
one chunk, one group, lookahead 1 and lookahead = groups."""
import math
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GRID = 148 * 4  # persistent CTAs of the 256-thread kernels on a B300

# (l1, columns, l2, rows per tile, chunk MiB) and (la, lb1, lb2, chunk MiB, tile)
TWO_PASS = {15: (7, 32, 8, 16, 32), 16: (8, 16, 8, 16, 16), 17: (8, 16, 9, 8, 32), 18: (8, 16, 10, 4, 32),
            19: (9, 16, 10, 8, 16), 20: (10, 8, 10, 8, 16), 21: (10, 16, 11, 8, 16), 22: (11, 4, 11, 4, 32),
            23: (12, 4, 11, 8, 48), 24: (12, 4, 12, 4, 8)}
THREE = {19: (6, 6, 7, 128, 4096), 20: (6, 7, 7, 128, 4096), 21: (7, 7, 7, 32, 4096), 22: (7, 7, 8, 32, 4096),
         23: (8, 7, 8, 32, 4096), 24: (8, 8, 8, 32, 4096)}


def two_params(logn, batch):
    l1, c, l2, tpc, mb = TWO_PASS[logn]
    n = 1 << logn
    cb = min(max((mb << 20) // (n * 8), 1), batch)
    return ["two", cb * ((1 << l2) // c), cb * ((1 << l1) // tpc), math.ceil(batch / cb)]


def three_params(logn, batch, grid=GRID):
    la, lb1, lb2, mb, tile = THREE[logn]
    n = 1 << logn
    cb = min(max((mb << 20) // (n * 8), 1), batch)
    ca, cbc, tpc = tile >> la, tile >> lb1, tile >> lb2
    na = cb * ((1 << (lb1 + lb2)) // ca)
    groups = cb * ((1 << la) // tpc)
    nb1g, nb2g = tpc * ((1 << lb2) // cbc), 1 << lb1
    d = min(max(-(-2 * grid // nb1g), 1), groups)
    return ["three", na, math.ceil(batch / cb), groups, nb1g, nb2g, d]


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("qoc") / "queue_order_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe,
                    os.path.join(ROOT, "tests", "queue_order_check.cu")], check=True, capture_output=True)
    return exe


def run(exe, *sets):
    args = [str(v) for s in sets for v in s]
    r = subprocess.run([exe] + args, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = r.stdout.strip().splitlines()
    assert len(lines) == len(sets) and all(ln.startswith("OK ") for ln in lines), r.stdout
    return lines


def lag(line, key):
    return int(line.split(key + "=")[1].split()[0])


def test_two_pass_sweep_shapes(checker):
    sets = [two_params(k, (1 << 26) >> k) for k in sorted(TWO_PASS)]
    for s, line in zip(sets, run(checker, *sets)):
        # the second pass of a chunk starts a whole chunk of first-pass tiles
        # after that chunk's last first-pass tile (unless it is the last chunk)
        na, nb, nch = s[1:]
        assert lag(line, "min_lag") == (na + 1 if nch > 1 else 1), line


def test_three_stage_sweep_shapes(checker):
    sets = [three_params(k, (1 << 26) >> k) for k in sorted(THREE)]
    for s, line in zip(sets, run(checker, *sets)):
        na, nch, groups, nb1g, nb2g, d = s[1:]
        assert lag(line, "min_lag_b1") >= 1 and lag(line, "min_lag_b2") >= 1, line
        if d >= 2:  # B2 of a group trails its B1 tiles by the D - 1 groups in between
            assert lag(line, "min_lag_b2") > (d - 1) * nb1g, line


@pytest.mark.parametrize("batch", [1, 3, 1000])
def test_ragged_batches(checker, batch):
    run(checker, two_params(16, batch), two_params(21, batch), three_params(22, batch), three_params(24, batch))


def test_edge_cases(checker):
    run(checker,
        ["two", 1, 1, 1], ["two", 3, 5, 1], ["two", 7, 2, 3], ["two", 2, 9, 5],
        ["three", 1, 1, 1, 1, 1, 1], ["three", 5, 2, 3, 2, 4, 3], ["three", 7, 3, 4, 2, 3, 1],
        ["three", 4, 4, 6, 3, 2, 6], ["three", 9, 2, 1, 5, 7, 1])


@pytest.mark.parametrize("case", [["two", 16, 16, 4], ["three", 8, 3, 4, 2, 8, 2]])
def test_checker_catches_a_planted_early_second_pass(checker, case):
    """The checker itself: with --plant every decoded second-pass (B1) tile
    is attributed to the chunk two ahead, so it precedes the first-pass
    tiles it needs; the check must report it."""
    r = subprocess.run([checker, "--plant"] + [str(v) for v in case], capture_output=True, text=True)
    assert r.returncode != 0 and "FAIL" in r.stdout and "before" in r.stdout, r.stdout
