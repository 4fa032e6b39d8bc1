"""The C ABI used from plain C: tests/c_abi_demo.c includes only
include/fft.h and the CUDA runtime, links libb300fft.so and checks closed
forms (tone spectra, round trip, a 2-D impulse) and argument errors.  It is
compiled here on the CPU and run on the GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1203_4938_b300")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def compile_demo(tmp_path) -> str:
    from paper_1203_4938_b300 import build as B
    B.build()
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "c_abi_demo")
    cmd = [cc, "-std=c99", "-O2", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(CUDA, "include"), os.path.join(ROOT, "tests", "c_abi_demo.c"), "-o", exe,
           "-L", PKG, "-lb300fft", "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-lm", f"-Wl,-rpath,{PKG}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_demo_compiles_and_links(tmp_path):
    assert os.path.exists(compile_demo(tmp_path))


@pytest.mark.gpu
def test_c_demo_runs(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = compile_demo(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "c_abi_demo: ok" in r.stdout
