// probe.cu -- FP32 FMA throughput probe: the non-tensor arithmetic ceiling of
// the GPU, against which the butterfly work of the transforms is compared
// (the measured peaks available otherwise are HBM copy and tensor-core GEMM).
//
// Each thread runs kChains independent chains a <- fma(a, m, c) for `iters`
// rounds (m = c = 1 at run time, so nothing folds): chain i ends at i + iters,
// exactly while iters <= 2^20.  out[j] = sum of its chains
// = kChains (kChains - 1) / 2 + kChains * iters, also exact.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fft.h"

namespace b300fft {

constexpr int kProbeThreads = 256, kChains = 16;

__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(float* __restrict__ out, int iters, float m, float c) {
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = (float)i;
#pragma unroll 8
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    out[(int64_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace b300fft

using namespace b300fft;

extern "C" fft_status fft_probe_fma(void* out, int64_t blocks, int64_t iters, void* stream) {
    if (!out || blocks < 1 || blocks > (int64_t(1) << 24) || iters < 1 || iters > (int64_t(1) << 20))
        return FFT_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(out) & 3) return FFT_ERR_MISALIGNED;
    k_fma_probe<<<(unsigned)blocks, kProbeThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<float*>(out), (int)iters, 1.0f, 1.0f);
    return cudaGetLastError() == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
}
