"""Host-side checks of the C ABI that need no GPU: the library loads, every
symbol include/fft.h declares is exported, and argument errors come back as
status codes before any device work (nothing is computed here)."""
import ctypes
import os
import re

import pytest

from paper_1203_4938_b300 import build as B
from paper_1203_4938_b300 import fft as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return F.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "fft.h")).read()
    return sorted(set(re.findall(r"FFT_API\s+[\w\s\*]*?\b(fft_\w+)\s*\(", text)))


def test_header_declares_the_binding_names():
    assert declared_symbols() == sorted(F.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_status_strings(lib):
    for s in range(8):
        assert F.fft_status_string(s)
    assert F.fft_status_string(99) == "unknown status"


@pytest.mark.parametrize("dims,lengths,batch,prec", [
    (0, [8], 1, 0), (3, [8, 8, 8], 1, 0), (1, [0], 1, 0), (1, [-4], 1, 0),
    (1, [8], 0, 0), (1, [8], -1, 0), (1, [8], 1, 7), (1, [8], 1, -1),
    (2, [8, 0], 1, 0), (1, [1 << 31], 1, 0), (1, [1 << 30], 1 << 20, 0),
])
def test_invalid_arguments_rejected_on_host(lib, dims, lengths, batch, prec):
    assert F.fft_plan_create(dims, lengths, batch, prec) is None
    assert F.fft_last_error() == F.FFT_ERR_INVALID_ARG


def test_null_lengths(lib):
    assert lib.fft_plan_create(1, None, 4, 0) is None
    assert F.fft_last_error() == F.FFT_ERR_INVALID_ARG


def test_bad_handles(lib):
    assert F.fft_exec(None, 16, 16, F.FFT_FORWARD) == F.FFT_ERR_BAD_HANDLE
    bogus = ctypes.c_void_p(0x1000).value
    assert F.fft_exec(bogus, 16, 16, F.FFT_FORWARD) == F.FFT_ERR_BAD_HANDLE
    assert F.fft_plan_destroy(None) == F.FFT_ERR_BAD_HANDLE
    assert F.fft_plan_destroy(bogus) == F.FFT_ERR_BAD_HANDLE
    assert F.fft_plan_check(bogus) == F.FFT_ERR_BAD_HANDLE
    assert F.fft_plan_workspace_bytes(bogus) == 0
    assert F.fft_plan_kernel_count(bogus) == 0
    with pytest.raises(F.FFTError):
        F.fft_plan_describe(bogus)


def test_ragged_invalid_arguments(lib):
    assert F.fft_plan_create_ragged([64, 0], 2, 0) is None
    assert F.fft_last_error() == F.FFT_ERR_INVALID_ARG
    assert F.fft_plan_create_ragged([64], 0, 0) is None
    assert F.fft_last_error() == F.FFT_ERR_INVALID_ARG
    assert lib.fft_plan_create_ragged(None, 3, 0) is None
    assert F.fft_last_error() == F.FFT_ERR_INVALID_ARG


@pytest.mark.parametrize("out,blocks,iters,status", [
    (0, 1, 1, F.FFT_ERR_INVALID_ARG), (256, 0, 1, F.FFT_ERR_INVALID_ARG), (256, 1, 0, F.FFT_ERR_INVALID_ARG),
    (256, 1, (1 << 20) + 1, F.FFT_ERR_INVALID_ARG), (256, (1 << 24) + 1, 1, F.FFT_ERR_INVALID_ARG),
    (258, 1, 1, F.FFT_ERR_MISALIGNED),
])
def test_fma_probe_argument_errors(lib, out, blocks, iters, status):
    # rejected before any launch: the pointer is never dereferenced
    assert F.fft_probe_fma(out, blocks, iters) == status
