"""Python binding of the C ABI in include/fft.h (ctypes; marshalling only).

Every transform runs in the CUDA kernels of ``libb300fft.so``; this module
only converts arguments.  There is no CPU fallback: if the library is missing
or no CUDA device is present, the calls raise.

The functions keep the C names (``fft_plan_create``, ``fft_exec``, ...).
``Plan`` and ``Ragged`` wrap a handle for torch tensors: device memory and the
stream come from PyTorch, the arithmetic from the library.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libb300fft.so")

FFT_OK = 0
FFT_ERR_INVALID_ARG = 1
FFT_ERR_UNSUPPORTED = 2
FFT_ERR_ALLOC = 3
FFT_ERR_MISALIGNED = 4
FFT_ERR_CUDA = 5
FFT_ERR_TIMEOUT = 6
FFT_ERR_BAD_HANDLE = 7

FFT_FP32 = 0
FFT_TC_FP16 = 1
FFT_TC_BF16 = 2
FFT_TC_FP16_PLAIN = 3
FFT_TC_BF16_PLAIN = 4

FFT_FORWARD = -1
FFT_INVERSE = +1

PRECISIONS = {"fp32": FFT_FP32, "tc_fp16": FFT_TC_FP16, "tc_bf16": FFT_TC_BF16,
              "tc_fp16_plain": FFT_TC_FP16_PLAIN, "tc_bf16_plain": FFT_TC_BF16_PLAIN}

# Symbols declared in include/fft.h (checked by the CPU test-suite).
EXPORTS = ("fft_plan_create", "fft_plan_create_ragged", "fft_last_error", "fft_exec",
           "fft_plan_check", "fft_plan_destroy", "fft_plan_workspace_bytes", "fft_status_string",
           "fft_plan_kernel_count", "fft_plan_describe", "fft_exec_kernel", "fft_exec_per_size",
           "fft_exec_pow2_static", "fft_plan_create_real", "fft_spectrum_product", "fft_image_steps",
           "fft_probe_fma", "fft_convolve")

_lock = threading.Lock()
_lib = None


class FFTError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = fft_status_string(status) if _lib is not None else str(status)
        super().__init__(f"{what}: {msg} (status {status})" if what else f"{msg} (status {status})")


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libb300fft.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing; run `python -m paper_1203_4938_b300.build` "
                               "(no CPU fallback exists)")
        lib = ctypes.CDLL(path)
        vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
        lib.fft_plan_create.argtypes = [ctypes.c_int, i64p, ctypes.c_int64, ctypes.c_int]
        lib.fft_plan_create.restype = vp
        lib.fft_plan_create_ragged.argtypes = [i64p, ctypes.c_int64, ctypes.c_int]
        lib.fft_plan_create_ragged.restype = vp
        lib.fft_spectrum_product.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_float,
                                             ctypes.c_int, vp]
        lib.fft_spectrum_product.restype = ctypes.c_int
        lib.fft_image_steps.argtypes = [vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_float,
                                        ctypes.c_float, vp, vp, vp, vp, vp]
        lib.fft_image_steps.restype = ctypes.c_int
        lib.fft_convolve.argtypes = [vp, vp, vp, vp, ctypes.c_float, ctypes.c_int, vp]
        lib.fft_convolve.restype = ctypes.c_int
        lib.fft_probe_fma.argtypes = [vp, ctypes.c_int64, ctypes.c_int64, vp]
        lib.fft_probe_fma.restype = ctypes.c_int
        lib.fft_plan_create_real.argtypes = [ctypes.c_int64, ctypes.c_int64]
        lib.fft_plan_create_real.restype = vp
        lib.fft_last_error.argtypes = []
        lib.fft_last_error.restype = ctypes.c_int
        lib.fft_exec.argtypes = [vp, vp, vp, ctypes.c_int, vp]
        lib.fft_exec.restype = ctypes.c_int
        lib.fft_plan_check.argtypes = [vp]
        lib.fft_plan_check.restype = ctypes.c_int
        lib.fft_plan_destroy.argtypes = [vp]
        lib.fft_plan_destroy.restype = ctypes.c_int
        lib.fft_plan_workspace_bytes.argtypes = [vp]
        lib.fft_plan_workspace_bytes.restype = ctypes.c_size_t
        lib.fft_status_string.argtypes = [ctypes.c_int]
        lib.fft_status_string.restype = ctypes.c_char_p
        lib.fft_plan_kernel_count.argtypes = [vp]
        lib.fft_plan_kernel_count.restype = ctypes.c_int
        lib.fft_exec_pow2_static.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, vp]
        lib.fft_exec_pow2_static.restype = ctypes.c_int
        lib.fft_exec_per_size.argtypes = [vp, vp, vp, ctypes.c_int, vp]
        lib.fft_exec_per_size.restype = ctypes.c_int
        lib.fft_exec_kernel.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int, vp]
        lib.fft_exec_kernel.restype = ctypes.c_int
        lib.fft_plan_describe.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
        lib.fft_plan_describe.restype = ctypes.c_int
        _lib = lib
        return lib


# --------------------------------------------------------------------------
# thin wrappers with the C names
# --------------------------------------------------------------------------
def _i64_array(vals):
    vals = [int(v) for v in vals]
    return (ctypes.c_int64 * max(1, len(vals)))(*vals)


def fft_plan_create(dims: int, lengths, batch: int, precision: int = FFT_FP32):
    """Returns the plan handle (int) or None; see fft_last_error()."""
    h = load().fft_plan_create(int(dims), _i64_array(lengths), int(batch), int(precision))
    return h or None


def fft_plan_create_ragged(lengths, count: int, precision: int = FFT_FP32):
    h = load().fft_plan_create_ragged(_i64_array(lengths), int(count), int(precision))
    return h or None


def fft_plan_create_real(n: int, batch: int):
    h = load().fft_plan_create_real(int(n), int(batch))
    return h or None


def fft_spectrum_product(a_ptr: int, b_ptr: int, out_ptr: int, n: int, batch: int, scale: float,
                         conj_b: bool = False, stream: int = 0) -> int:
    return int(load().fft_spectrum_product(a_ptr, b_ptr, out_ptr, int(n), int(batch), float(scale),
                                           int(bool(conj_b)), stream or None))


def fft_image_steps(rgb_ptr: int, batch: int, h: int, w: int, ux: float, uy: float, y_ptr: int, cb_ptr: int,
                    cr_ptr: int, d_ptr: int, stream: int = 0) -> int:
    return int(load().fft_image_steps(rgb_ptr, int(batch), int(h), int(w), float(ux), float(uy), y_ptr, cb_ptr,
                                      cr_ptr, d_ptr, stream or None))


def fft_convolve(plan, x_ptr: int, h_ptr: int, out_ptr: int, scale: float, conj_h: bool, stream: int = 0) -> int:
    return int(load().fft_convolve(plan, x_ptr, h_ptr, out_ptr, float(scale), int(bool(conj_h)), stream or None))


def fft_probe_fma(out_ptr: int, blocks: int, iters: int, stream: int = 0) -> int:
    return int(load().fft_probe_fma(out_ptr, int(blocks), int(iters), stream or None))


def fma_probe(blocks: int, iters: int, out=None):
    """Run the FP32 FMA probe on the current stream; returns (out, flops).
    out: float32 CUDA tensor of blocks * 256 elements (allocated if None)."""
    import torch
    if out is None:
        out = torch.empty(blocks * 256, dtype=torch.float32, device="cuda")
    if out.dtype != torch.float32 or not out.is_cuda or out.numel() < blocks * 256:
        raise ValueError("out must be a CUDA float32 tensor of blocks * 256 elements")
    st = fft_probe_fma(out.data_ptr(), blocks, iters, torch.cuda.current_stream().cuda_stream)
    if st != 0:
        raise FFTError(st, "fft_probe_fma")
    return out, 2.0 * 16 * 256 * blocks * iters


def fft_last_error() -> int:
    return int(load().fft_last_error())


def fft_exec(plan, in_ptr: int, out_ptr: int, direction: int, stream: int = 0) -> int:
    return int(load().fft_exec(plan, in_ptr, out_ptr, int(direction), stream or None))


def fft_exec_pow2_static(in_ptr: int, out_ptr: int, n: int, batch: int, direction: int, stream: int = 0) -> int:
    """Allocation-free transform of batch x n (power of two, 2^13..2^22,
    n*batch <= 2^22) using the library's static workspace; see include/fft.h."""
    return int(load().fft_exec_pow2_static(in_ptr, out_ptr, int(n), int(batch), int(direction), stream or None))


def fft_exec_per_size(plan, in_ptr: int, out_ptr: int, direction: int, stream: int = 0) -> int:
    return int(load().fft_exec_per_size(plan, in_ptr, out_ptr, int(direction), stream or None))


def fft_exec_kernel(plan, k: int, in_ptr: int, out_ptr: int, direction: int, stream: int = 0) -> int:
    return int(load().fft_exec_kernel(plan, int(k), in_ptr, out_ptr, int(direction), stream or None))


def fft_plan_check(plan) -> int:
    return int(load().fft_plan_check(plan))


def fft_plan_destroy(plan) -> int:
    return int(load().fft_plan_destroy(plan))


def fft_plan_workspace_bytes(plan) -> int:
    return int(load().fft_plan_workspace_bytes(plan))


def fft_status_string(status: int) -> str:
    return load().fft_status_string(int(status)).decode()


def fft_plan_kernel_count(plan) -> int:
    return int(load().fft_plan_kernel_count(plan))


def fft_plan_describe(plan) -> str:
    buf = ctypes.create_string_buffer(512)
    n = load().fft_plan_describe(plan, buf, 512)
    if n < 0:
        raise FFTError(FFT_ERR_BAD_HANDLE, "fft_plan_describe")
    return buf.value.decode()


# --------------------------------------------------------------------------
# torch-facing helpers
# --------------------------------------------------------------------------
def _check_tensor(t, numel: int, what: str):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.complex64 or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA complex64 tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{what} has {t.numel()} elements, the plan needs {numel}")


class Plan:
    """Batched 1-D or 2-D C2C plan; exec() enqueues on torch's current stream."""

    def __init__(self, lengths, batch: int = 1, precision="fp32"):
        if isinstance(lengths, int):
            lengths = (lengths,)
        self.lengths = tuple(int(v) for v in lengths)
        self.batch = int(batch)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.handle = fft_plan_create(len(self.lengths), self.lengths, self.batch, self.precision)
        if self.handle is None:
            raise FFTError(fft_last_error(), "fft_plan_create")
        n = self.batch
        for v in self.lengths:
            n *= v
        self.numel = n

    @property
    def shape(self):
        return (self.batch,) + self.lengths

    def exec(self, x, out=None, direction: int = FFT_FORWARD, stream=None):
        import torch
        _check_tensor(x, self.numel, "input")
        if out is None:
            out = torch.empty(self.shape, dtype=torch.complex64, device=x.device)
        _check_tensor(out, self.numel, "output")
        s = stream if stream is not None else torch.cuda.current_stream(x.device)
        rc = fft_exec(self.handle, x.data_ptr(), out.data_ptr(), direction, s.cuda_stream)
        if rc != FFT_OK:
            raise FFTError(rc, "fft_exec")
        return out

    def exec_per_size(self, x, out=None, direction: int = FFT_FORWARD, stream=None):
        """fft_exec_per_size: one launch per (stage, length) group (baseline form)."""
        import torch
        _check_tensor(x, self.numel, "input")
        if out is None:
            out = torch.empty(self.shape, dtype=torch.complex64, device=x.device)
        _check_tensor(out, self.numel, "output")
        s = stream if stream is not None else torch.cuda.current_stream(x.device)
        rc = fft_exec_per_size(self.handle, x.data_ptr(), out.data_ptr(), direction, s.cuda_stream)
        if rc != FFT_OK:
            raise FFTError(rc, "fft_exec_per_size")
        return out

    def exec_kernel(self, k: int, x, out, direction: int = FFT_FORWARD, stream=None):
        """Enqueue only kernel k of this plan's sequence (for per-kernel timing)."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(x.device)
        rc = fft_exec_kernel(self.handle, k, x.data_ptr(), out.data_ptr(), direction, s.cuda_stream)
        if rc != FFT_OK:
            raise FFTError(rc, "fft_exec_kernel")
        return out

    def forward(self, x, out=None):
        return self.exec(x, out, FFT_FORWARD)

    def inverse(self, x, out=None):
        return self.exec(x, out, FFT_INVERSE)

    def check(self):
        rc = fft_plan_check(self.handle)
        if rc != FFT_OK:
            raise FFTError(rc, "fft_plan_check")

    @property
    def workspace_bytes(self) -> int:
        return fft_plan_workspace_bytes(self.handle)

    @property
    def kernel_count(self) -> int:
        return fft_plan_kernel_count(self.handle)

    def describe(self) -> str:
        return fft_plan_describe(self.handle)

    def close(self):
        if self.handle is not None:
            fft_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Ragged(Plan):
    """Uneven-length 1-D batch packed back to back (one persistent launch)."""

    def __init__(self, lengths, precision="fp32"):
        self.lengths = tuple(int(v) for v in lengths)
        self.batch = len(self.lengths)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.handle = fft_plan_create_ragged(self.lengths, len(self.lengths), self.precision)
        if self.handle is None:
            raise FFTError(fft_last_error(), "fft_plan_create_ragged")
        self.numel = sum(self.lengths)

    @property
    def shape(self):
        return (self.numel,)


class RealPlan(Plan):
    """Real <-> half-spectrum plan: forward() takes float32 [batch, n] and
    returns complex64 [batch, n/2+1]; inverse() the reverse (unnormalised)."""

    def __init__(self, n: int, batch: int = 1):
        self.lengths = (int(n),)
        self.batch = int(batch)
        self.precision = FFT_FP32
        self.handle = fft_plan_create_real(n, batch)
        if self.handle is None:
            raise FFTError(fft_last_error(), "fft_plan_create_real")
        self.numel = self.batch * int(n)

    def forward(self, x, out=None):
        import torch
        n = self.lengths[0]
        if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous() or x.numel() != self.numel:
            raise TypeError("forward input must be a contiguous CUDA float32 tensor of batch*n values")
        if out is None:
            out = torch.empty((self.batch, n // 2 + 1), dtype=torch.complex64, device=x.device)
        s = torch.cuda.current_stream(x.device)
        rc = fft_exec(self.handle, x.data_ptr(), out.data_ptr(), FFT_FORWARD, s.cuda_stream)
        if rc != FFT_OK:
            raise FFTError(rc, "fft_exec")
        return out

    def inverse(self, x, out=None):
        import torch
        n = self.lengths[0]
        if x.dtype != torch.complex64 or not x.is_cuda or not x.is_contiguous() or \
                x.numel() != self.batch * (n // 2 + 1):
            raise TypeError("inverse input must be a contiguous CUDA complex64 tensor [batch, n/2+1]")
        if out is None:
            out = torch.empty((self.batch, n), dtype=torch.float32, device=x.device)
        s = torch.cuda.current_stream(x.device)
        rc = fft_exec(self.handle, x.data_ptr(), out.data_ptr(), FFT_INVERSE, s.cuda_stream)
        if rc != FFT_OK:
            raise FFTError(rc, "fft_exec")
        return out


def convolve(x, h, corr: bool = False):
    """Circular convolution (or correlation) of every row of x ([batch, n] or
    [batch, H, W] complex64 on CUDA) with h ([n] or [H, W]): forward
    transforms, the spectrum product with 1/N folded in, inverse transform --
    all on the GPU through the C ABI."""
    import torch
    shape = tuple(x.shape[1:])
    batch = x.shape[0]
    n = 1
    for v in shape:
        n *= v
    with Plan(shape, batch) as px, Plan(shape, 1) as ph:
        H = ph.forward(h.reshape((1,) + shape).contiguous())
        s = torch.cuda.current_stream(x.device)
        # one call (fused for 1-D power-of-two lengths up to 2^14)
        _check_tensor(x, px.numel, "input")
        out = torch.empty_like(x)
        rc = fft_convolve(px.handle, x.data_ptr(), H.data_ptr(), out.data_ptr(), 1.0 / n, corr, s.cuda_stream)
        if rc != FFT_OK:
            raise FFTError(rc, "fft_convolve")
        return out


def image_steps(rgb, ux: float = 1.0, uy: float = 0.0, out=None):
    """Steps 1-3 of the image example on the GPU: rgb is a [batch, h, w, 3]
    uint8 CUDA tensor (h, w even).  Returns (y, cb, cr, d) float32 tensors:
    luminance and its directional derivative along (ux, uy) at full size,
    chroma at half width and half height.  ``out`` may supply the four
    output tensors."""
    import torch
    if rgb.dtype != torch.uint8 or not rgb.is_cuda or not rgb.is_contiguous() or rgb.dim() != 4 or rgb.shape[3] != 3:
        raise TypeError("rgb must be a contiguous CUDA uint8 tensor of shape [batch, h, w, 3]")
    b, h, w, _ = rgb.shape
    if out is None:
        out = (torch.empty((b, h, w), dtype=torch.float32, device=rgb.device),
               torch.empty((b, h // 2, w // 2), dtype=torch.float32, device=rgb.device),
               torch.empty((b, h // 2, w // 2), dtype=torch.float32, device=rgb.device),
               torch.empty((b, h, w), dtype=torch.float32, device=rgb.device))
    y, cb, cr, d = out
    s = torch.cuda.current_stream(rgb.device)
    rc = fft_image_steps(rgb.data_ptr(), b, h, w, ux, uy, y.data_ptr(), cb.data_ptr(), cr.data_ptr(), d.data_ptr(),
                         s.cuda_stream)
    if rc != FFT_OK:
        raise FFTError(rc, "fft_image_steps")
    return y, cb, cr, d
