"""Seeded synthetic inputs for the batched FFT workloads.

This module holds input generation only -- none of the transform's arithmetic
-- and is the one piece shared by the CUDA-path tests, the oracle tests and
the benchmark.  All generators use ``numpy.random.default_rng(seed)`` and
return interleaved complex64 data (``numpy.complex64``), the paper's
``float2`` element type.

Workloads (sizes and distributions of the batched-FFT study):
  * ``uniform_batch``   i.i.d. uniform[-1, 1] real and imaginary parts.
  * ``normal_batch``    i.i.d. standard normal real and imaginary parts.
  * ``sweep_sizes``     N = 2^10 .. 2^24 with batch 2^26 / N (512 MiB per buffer).
  * ``image_batch``     image-shaped 2-D data: uint8-range integers plus a
                        smooth integer-period sinusoid in the real part, zero
                        imaginary part.
  * ``ragged_lengths``  log-uniform mix of 2^k, 3*2^k, 5*2^k, 7*2^k and ~1 %
                        prime lengths in [64, 65536].
"""
from __future__ import annotations

import math

import numpy as np

# Largest prime below 2^16, the cap for prime lengths in the ragged mix.
PRIME_CAP = 65521
RAGGED_MIN, RAGGED_MAX = 64, 65536


def _interleaved_to_c64(a: np.ndarray) -> np.ndarray:
    """(..., 2) float32 -> (...) complex64, re = a[..., 0], im = a[..., 1]."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a.view(np.complex64).reshape(a.shape[:-1])


def uniform_batch(batch: int, n: int, seed: int = 0) -> np.ndarray:
    """[batch][n] complex64, re and im i.i.d. uniform[-1, 1] (seed 0 by default)."""
    rng = np.random.default_rng(seed)
    return _interleaved_to_c64(rng.uniform(-1.0, 1.0, (batch, n, 2)).astype(np.float32))


def normal_batch(batch: int, n: int, seed: int = 1) -> np.ndarray:
    """[batch][n] complex64, re and im i.i.d. standard normal."""
    rng = np.random.default_rng(seed)
    return _interleaved_to_c64(rng.standard_normal((batch, n, 2), dtype=np.float32))


def sweep_sizes(total_log2: int = 26, lo: int = 10, hi: int = 24):
    """(n, N, batch) for the power-of-two sweep holding 2^total_log2 elements."""
    return [(k, 1 << k, 1 << (total_log2 - k)) for k in range(lo, hi + 1)]


def sweep_input(k: int, total_log2: int = 26, seed: int = 1) -> np.ndarray:
    """Sweep input for N = 2^k: normal(0,1), re-seeded for every k."""
    return normal_batch(1 << (total_log2 - k), 1 << k, seed)


def image_batch(rng: np.random.Generator, batch: int, h: int, w: int,
                amp: float = 32.0, fx: int = 3, fy: int = 2) -> np.ndarray:
    """[batch][h][w] complex64 image-shaped data.

    real = uint8-range integers (uniform over 0..255, cast to float32) plus
    ``amp*sin(2*pi*(fx*x/w + fy*y/h))`` (integer periods, so it sums to zero);
    imag = 0.  ``rng`` is shared so that consecutive images differ.
    """
    ints = rng.integers(0, 256, (batch, h, w)).astype(np.float32)
    y = np.arange(h, dtype=np.float64)[:, None]
    x = np.arange(w, dtype=np.float64)[None, :]
    field = (amp * np.sin(2.0 * np.pi * (fx * x / w + fy * y / h))).astype(np.float32)
    out = np.zeros((batch, h, w), dtype=np.complex64)
    out.real = ints + field[None]
    return out


def image_workload(seed: int = 2, big: int = 4096, small: int = 2048, nsmall: int = 16):
    """The image-shaped pair: one big x big image, then nsmall small x small ones."""
    rng = np.random.default_rng(seed)
    a = image_batch(rng, 1, big, big)
    b = image_batch(rng, nsmall, small, small)
    return a, b


def _next_prime(v: int) -> int:
    def is_prime(p: int) -> bool:
        if p < 2:
            return False
        if p % 2 == 0:
            return p == 2
        r = int(math.isqrt(p))
        for d in range(3, r + 1, 2):
            if p % d == 0:
                return False
        return True

    while not is_prime(v):
        v += 1
    return v


def ragged_lengths(count: int = 10000, seed: int = 4):
    """Length mix of the ragged batch; returns (lengths int64 array, rng).

    Per transform: u = rng.random(), e = rng.uniform(6, 16), t = 2^e.
      u < 0.01  -> smallest prime >= round(t), capped at 65521;
      u < 0.55  -> 2^round(e);
      otherwise -> m in {3, 5, 7} by thirds of [0.55, 1), length m * 2^j with
                   j = round(log2(t/m)) clamped so that 64 <= m*2^j <= 65536.
    The returned generator continues the same stream for the data draw.
    """
    rng = np.random.default_rng(seed)
    out = np.empty(count, dtype=np.int64)
    for i in range(count):
        u = rng.random()
        e = rng.uniform(6.0, 16.0)
        t = 2.0 ** e
        if u < 0.01:
            v = min(_next_prime(int(round(t))), PRIME_CAP)
            if v > PRIME_CAP or not v:
                v = PRIME_CAP
            out[i] = v
        elif u < 0.55:
            out[i] = 1 << int(round(e))
        else:
            m = 3 if u < 0.55 + 0.45 / 3 else (5 if u < 0.55 + 2 * 0.45 / 3 else 7)
            j = int(round(math.log2(t / m)))
            jlo = math.ceil(math.log2(RAGGED_MIN / m))
            jhi = math.floor(math.log2(RAGGED_MAX / m))
            j = min(max(j, jlo), jhi)
            out[i] = m << j
    return out, rng


def rgb_images(rng: np.random.Generator, batch: int, h: int, w: int) -> np.ndarray:
    """[batch][h][w][3] uint8 RGB images: per channel a smooth field
    (128 + 100 sin/cos with integer periods, different per channel) plus
    uniform noise in [-24, 24], clipped to 0..255."""
    y = np.arange(h, dtype=np.float32)[:, None] / h
    x = np.arange(w, dtype=np.float32)[None, :] / w
    fields = (np.sin(2 * np.pi * (3 * x + 2 * y)), np.cos(2 * np.pi * (2 * x - y)), np.sin(2 * np.pi * (x + 4 * y)))
    out = np.empty((batch, h, w, 3), dtype=np.uint8)
    for c in range(3):
        base = 128.0 + 100.0 * fields[c]
        for b in range(batch):
            v = base + rng.integers(-24, 25, (h, w)).astype(np.float32)
            out[b, :, :, c] = np.clip(v, 0, 255).astype(np.uint8)
    return out


def rgb_workload(seed: int = 2, big: int = 4096, small: int = 2048, nsmall: int = 16):
    """The image-example workload in RGB: one big x big and nsmall small x
    small images (the shapes of the 2-D FFT workload), seeded."""
    rng = np.random.default_rng(seed)
    return rgb_images(rng, 1, big, big), rgb_images(rng, nsmall, small, small)


def ragged_workload(count: int = 10000, seed: int = 4):
    """(lengths, offsets, packed complex64 data) for the ragged batch.

    Data: one draw of uniform[-1, 1] over 2*sum(lengths) floats, packed back to
    back; offsets are the exclusive prefix sum of the lengths.
    """
    lengths, rng = ragged_lengths(count, seed)
    offsets = np.zeros(count + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    total = int(offsets[-1])
    flat = rng.uniform(-1.0, 1.0, 2 * total).astype(np.float32)
    return lengths, offsets, flat.view(np.complex64)
