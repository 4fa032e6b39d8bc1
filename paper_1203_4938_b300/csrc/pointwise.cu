// pointwise.cu -- the spectrum product of FFT convolution and correlation
// (the paper's Sec. III-A lists convolutions among the DFT's applications):
// circular convolution y = x (*) h is IDFT(DFT(x) . DFT(h)) / N, and
// correlation uses conj(DFT(h)).  The product runs between the forward and
// the inverse transform, one filter spectrum broadcast over the batch, with
// the 1/N folded in.
#include <cuda_runtime.h>

#include "../../include/fft.h"
#include "butterfly.cuh"

namespace b300fft {

// out[t][k] = scale * a[t][k] * (conj ? conj(b[k]) : b[k]), two elements per
// thread and step with 16-byte accesses (n even) or one (n odd).
template <bool CONJ, bool VEC>
__global__ void k_pointwise(const float2* __restrict__ a, const float2* __restrict__ b, float2* __restrict__ out,
                            int64_t n, int64_t total, float scale) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if constexpr (VEC) {
        const float4* a4 = reinterpret_cast<const float4*>(a);
        float4* o4 = reinterpret_cast<float4*>(out);
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total / 2; i += stride) {
            const float4 v = __ldcs(a4 + i);
            const int64_t k = (2 * i) % n;  // n even: both elements share the row
            const float2 f0 = __ldg(b + k), f1 = __ldg(b + k + 1);
            const float2 p0 = CONJ ? cmulc(make_float2(v.x, v.y), f0) : cmul(make_float2(v.x, v.y), f0);
            const float2 p1 = CONJ ? cmulc(make_float2(v.z, v.w), f1) : cmul(make_float2(v.z, v.w), f1);
            __stcs(o4 + i, make_float4(p0.x * scale, p0.y * scale, p1.x * scale, p1.y * scale));
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
            const float2 f = __ldg(b + i % n);
            const float2 p = CONJ ? cmulc(__ldcs(a + i), f) : cmul(__ldcs(a + i), f);
            __stcs(out + i, make_float2(p.x * scale, p.y * scale));
        }
    }
}

}  // namespace b300fft

using namespace b300fft;

extern "C" fft_status fft_spectrum_product(const void* a, const void* b, void* out, int64_t n, int64_t batch,
                                           float scale, int conj_b, void* stream) {
    if (!a || !b || !out || n < 1 || batch < 1 || batch > (int64_t(1) << 40) / n) return FFT_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(a) & 15) || (reinterpret_cast<uintptr_t>(b) & 15) ||
        (reinterpret_cast<uintptr_t>(out) & 15))
        return FFT_ERR_MISALIGNED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t total = n * batch;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool vec = (n % 2) == 0;
    const int64_t work = vec ? total / 2 : total;
    int64_t blocks = (work + 255) / 256;
    if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
    if (blocks < 1) blocks = 1;
    const float2* A = static_cast<const float2*>(a);
    const float2* B = static_cast<const float2*>(b);
    float2* O = static_cast<float2*>(out);
    if (conj_b) {
        if (vec) k_pointwise<true, true><<<(unsigned)blocks, 256, 0, st>>>(A, B, O, n, total, scale);
        else k_pointwise<true, false><<<(unsigned)blocks, 256, 0, st>>>(A, B, O, n, total, scale);
    } else {
        if (vec) k_pointwise<false, true><<<(unsigned)blocks, 256, 0, st>>>(A, B, O, n, total, scale);
        else k_pointwise<false, false><<<(unsigned)blocks, 256, 0, st>>>(A, B, O, n, total, scale);
    }
    return cudaGetLastError() == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
}
