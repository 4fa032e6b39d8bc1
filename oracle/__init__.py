"""FP64 CPU oracle for the discrete Fourier transform (test infrastructure).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
and never imports it.  The arithmetic lives in ``oracle.c`` (plain C, FP64);
this module compiles it with gcc on first use and marshals numpy arrays.

Definition followed (paper Sec. III-A, the DFT example): for a length-N complex
sequence, ``X[k] = sum_n x[n] exp(sign*2*pi*i*n*k/N)`` with sign -1 for the
forward and +1 for the inverse transform, both unnormalised; the paper
computes it with radix-2 Cooley-Tukey, which ``fft`` follows for powers of two.

``image_steps`` follows the image example of Sec. III-B (its GPU steps 1-3:
colour transform, chroma downscale, directional derivative of luminance).

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, textbook values in ``tests/golden/``, Parseval, linearity,
shift, symmetry, brute force and an independent library witness); planted
mistakes in copies of ``oracle.c`` are shown to fail those pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_default = None

FORWARD = -1
INVERSE = +1


def compile_source(src: str, out: str) -> str:
    """Compile an oracle C source into a shared library (no -ffast-math)."""
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-o", tmp, src,
           "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it when missing or stale."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(SOURCE)):
        return _LIB_PATH
    return compile_source(SOURCE, _LIB_PATH)


def _c128(x) -> np.ndarray:
    """Widen to contiguous complex128 (float32 values are represented exactly)."""
    return np.ascontiguousarray(np.asarray(x), dtype=np.complex128)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


class OracleLib:
    """numpy front end over one compiled copy of oracle.c."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        lib.oracle_dft_naive.argtypes = [dp, dp, i64, ctypes.c_int]
        lib.oracle_dft_bins.argtypes = [dp, i64, ctypes.c_int,
                                        ctypes.POINTER(i64), i64, dp]
        lib.oracle_fft_radix2.argtypes = [dp, dp, i64, ctypes.c_int]
        lib.oracle_fft_split_m.argtypes = [dp, dp, i64, i64, ctypes.c_int]
        lib.oracle_fft.argtypes = [dp, dp, i64, ctypes.c_int]
        lib.oracle_fft_batch.argtypes = [dp, dp, i64, i64, ctypes.c_int,
                                         ctypes.c_int]
        lib.oracle_fft2d.argtypes = [dp, dp, i64, i64, i64, ctypes.c_int,
                                     ctypes.c_int]
        lib.oracle_circ_conv.argtypes = [dp, dp, dp, i64, ctypes.c_int]
        lib.oracle_circ_conv.restype = ctypes.c_int
        lib.oracle_image_steps.argtypes = [ctypes.c_void_p, i64, i64, i64, ctypes.c_double, ctypes.c_double,
                                           dp, dp, dp, dp]
        lib.oracle_image_steps.restype = ctypes.c_int
        lib.oracle_num_cpus.argtypes = []
        for f in ("oracle_dft_naive", "oracle_dft_bins", "oracle_fft_radix2",
                  "oracle_fft_split_m", "oracle_fft", "oracle_fft_batch",
                  "oracle_fft2d", "oracle_num_cpus"):
            getattr(lib, f).restype = ctypes.c_int
        self.lib = lib
        self.path = path

    def num_cpus(self) -> int:
        return int(self.lib.oracle_num_cpus())

    def _per_row(self, fn, x, *args):
        x = _c128(x)
        n = x.shape[-1]
        flat = x.reshape(-1, n)
        y = np.empty_like(flat)
        for b in range(flat.shape[0]):
            _check(fn(_ptr(flat[b]), _ptr(y[b]), n, *args), fn.__name__)
        return y.reshape(x.shape)

    def dft_naive(self, x, sign: int = FORWARD) -> np.ndarray:
        """O(N^2) DFT straight from the definition, along the last axis."""
        return self._per_row(self.lib.oracle_dft_naive, x, sign)

    def fft_radix2(self, x, sign: int = FORWARD) -> np.ndarray:
        """Radix-2 Cooley-Tukey along the last axis (length a power of two)."""
        return self._per_row(self.lib.oracle_fft_radix2, x, sign)

    def fft_split_m(self, x, m: int, sign: int = FORWARD) -> np.ndarray:
        """One Cooley-Tukey step N = m * 2^j over radix-2 sub-transforms."""
        return self._per_row(self.lib.oracle_fft_split_m, x, m, sign)

    def dft_bins(self, x, ks, sign: int = FORWARD) -> np.ndarray:
        """Selected bins X[k] of one length-N sequence, O(N) each."""
        x = _c128(x).reshape(-1)
        ks = np.ascontiguousarray(np.asarray(ks, dtype=np.int64).reshape(-1))
        out = np.empty(ks.shape[0], dtype=np.complex128)
        _check(self.lib.oracle_dft_bins(
            _ptr(x), x.shape[0], sign,
            ks.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ks.shape[0],
            _ptr(out)), "dft_bins")
        return out

    def fft(self, x, sign: int = FORWARD, threads: int = 0) -> np.ndarray:
        """Batched DFT along the last axis (radix-2, m*2^j split, or naive)."""
        x = _c128(x)
        if x.size == 0:
            return x.copy()
        n = x.shape[-1]
        y = np.empty_like(x)
        _check(self.lib.oracle_fft_batch(_ptr(x), _ptr(y), n, x.size // n, sign,
                                         threads), "fft_batch")
        return y

    def circ_conv(self, x, h, corr: bool = False) -> np.ndarray:
        """Circular convolution (or correlation) of each row of x with h, by
        the definition, O(N^2) per row."""
        x = _c128(x)
        h = _c128(h).reshape(-1)
        n = x.shape[-1]
        assert h.shape[0] == n
        flat = x.reshape(-1, n)
        y = np.empty_like(flat)
        for b in range(flat.shape[0]):
            _check(self.lib.oracle_circ_conv(_ptr(flat[b]), _ptr(h), _ptr(y[b]), n, int(bool(corr))),
                   "circ_conv")
        return y.reshape(x.shape)

    def image_steps(self, rgb, ux: float = 1.0, uy: float = 0.0):
        """Steps 1-3 of the image example (Sec. III-B): YCbCr, chroma 2x2 mean,
        directional derivative of Y.  rgb: uint8 [batch, h, w, 3].  Returns
        (y, cb, cr, d) in FP64: y, d [batch, h, w]; cb, cr [batch, h/2, w/2]."""
        rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
        b, h, w, c = rgb.shape
        assert c == 3
        y = np.empty((b, h, w))
        d = np.empty((b, h, w))
        cb = np.empty((b, h // 2, w // 2))
        cr = np.empty((b, h // 2, w // 2))
        _check(self.lib.oracle_image_steps(rgb.ctypes.data_as(ctypes.c_void_p), b, h, w, float(ux), float(uy),
                                           _ptr(y), _ptr(cb), _ptr(cr), _ptr(d)), "image_steps")
        return y, cb, cr, d

    def fft2(self, x, sign: int = FORWARD, threads: int = 0) -> np.ndarray:
        """2-D DFT over the last two axes: rows first, then columns."""
        x = _c128(x)
        if x.size == 0:
            return x.copy()
        h, w = x.shape[-2], x.shape[-1]
        y = np.empty_like(x)
        _check(self.lib.oracle_fft2d(_ptr(x), _ptr(y), h, w, x.size // (h * w),
                                     sign, threads), "fft2d")
        return y


def default() -> OracleLib:
    """The oracle built from oracle.c (compiled on first use)."""
    global _default
    with _lock:
        if _default is None:
            _default = OracleLib(build())
        return _default


def num_cpus() -> int:
    return default().num_cpus()


def dft_naive(x, sign: int = FORWARD) -> np.ndarray:
    return default().dft_naive(x, sign)


def dft_bins(x, ks, sign: int = FORWARD) -> np.ndarray:
    return default().dft_bins(x, ks, sign)


def fft_radix2(x, sign: int = FORWARD) -> np.ndarray:
    return default().fft_radix2(x, sign)


def fft_split_m(x, m: int, sign: int = FORWARD) -> np.ndarray:
    return default().fft_split_m(x, m, sign)


def fft(x, sign: int = FORWARD, threads: int = 0) -> np.ndarray:
    return default().fft(x, sign, threads)


def fft2(x, sign: int = FORWARD, threads: int = 0) -> np.ndarray:
    return default().fft2(x, sign, threads)


def circ_conv(x, h, corr: bool = False) -> np.ndarray:
    return default().circ_conv(x, h, corr)


def image_steps(rgb, ux: float = 1.0, uy: float = 0.0):
    return default().image_steps(rgb, ux, uy)


def rel_l2(y, ref) -> np.ndarray:
    """Per-transform relative L2 error along the last axis, in FP64.

    Where the reference transform is all zeros the absolute L2 is returned.
    """
    y = _c128(y)
    ref = _c128(ref)
    d = np.sqrt(np.sum(np.abs(y - ref) ** 2, axis=-1))
    r = np.sqrt(np.sum(np.abs(ref) ** 2, axis=-1))
    return np.where(r > 0, d / np.where(r > 0, r, 1.0), d)
