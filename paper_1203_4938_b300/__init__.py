"""B300-native batched complex-to-complex FFT (sm_103a).

The DFT of the paper's Sec. III-A example, run on one GPU by hand-written CUDA
kernels behind the C ABI of include/fft.h.  ``fft`` is the Python binding;
``inputs`` the seeded synthetic workloads.  Importing the package loads no
native code; the first call into ``fft`` does.
"""
__all__ = ["fft", "inputs", "build"]
