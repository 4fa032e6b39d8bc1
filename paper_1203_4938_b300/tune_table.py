"""Re-derive the batched power-of-two planner's default table on this GPU.

For every length 2^k of the benchmark sweep (k = 13..24, batch 2^26 / 2^k,
the sizes the table in csrc/fft_api.cu was measured at) a plan is created with
FFT_AUTOTUNE=1: the library times every compiled kernel family and shape for
that length (tune_pow2.cu) and keeps the fastest.  The picks are printed one
line per length (family, shape, chunk MiB, ring slots, lookahead, time per
forward exec) and appended to the cache file given by --cache, which a later
process can reuse through FFT_TUNE_CACHE.

Usage: python -m paper_1203_4938_b300.tune_table [--cache FILE] [--lo 13] [--hi 24]
"""
from __future__ import annotations

import argparse
import os
import sys

FAMILIES = {1: "rows", 2: "fourstep-persist", 3: "threestep"}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--cache", default="fft_tune_cache.txt")
    ap.add_argument("--lo", type=int, default=13)
    ap.add_argument("--hi", type=int, default=24)
    ap.add_argument("--total-log2", type=int, default=26)
    a = ap.parse_args(argv)
    os.environ["FFT_AUTOTUNE"] = "1"
    os.environ["FFT_TUNE_CACHE"] = os.path.abspath(a.cache)
    import torch  # noqa: F401  (device memory for the library's own allocations)
    from . import fft as F
    F.load()
    for k in range(a.lo, a.hi + 1):
        n, b = 1 << k, 1 << (a.total_log2 - k)
        with F.Plan((n,), b) as p:
            desc = p.describe()
        line = ""
        with open(a.cache) as fh:
            for ln in fh:
                if ln.startswith("pow2:") and ln.split()[0].endswith(f":{k}:{b}"):
                    line = ln.split()
        if line:
            fam, x1, x2, x3, x4, mb, ring, ahead, us = line[1:10]
            print(f"2^{k} x {b}: {FAMILIES.get(int(fam), fam)} ({x1},{x2},{x3},{x4}) chunk={mb}MiB ring={ring} "
                  f"ahead={ahead} {float(us):.1f} us | {desc}", flush=True)
        else:
            print(f"2^{k} x {b}: (no candidates) | {desc}", flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
