// conv.cu -- FFT convolution / correlation of rows in one pass (the DFT use
// the paper's Sec. III-A names): for a power-of-two length N <= 2^14 each
// row is loaded once, transformed forward in its tile, multiplied by the
// filter spectrum H (or conj(H)) and the scale, transformed back in the same
// tile and stored -- one HBM round trip instead of three (forward transform,
// spectrum product, inverse transform).
#include "kernels_launch.cuh"

namespace b300fft {

template <int LOGN, int TPC, int RT, bool CORR>
__global__ void __launch_bounds__(RowsCfg<LOGN, TPC, RT>::THREADS,
                                  (RT == 16 ? 1024 : 512) / RowsCfg<LOGN, TPC, RT>::THREADS)
    k_conv_rows(const float2* __restrict__ in, float2* __restrict__ out, int64_t nrows, const float2* __restrict__ tw,
                const float2* __restrict__ hs, float scale) {
    using PL = P2Plan<LOGN, RT>;
    extern __shared__ float2 smem[];
    const int t = threadIdx.x & (PL::T - 1), sub = threadIdx.x / PL::T;
    const int64_t row = (int64_t)blockIdx.x * TPC + sub;
    const bool ok = row < nrows;
    float2* s = smem + sub * PL::PADDED;
    float2 v[PL::R];
    const float2* src = in + row * PL::N;
#pragma unroll
    for (int i = 0; i < PL::R; ++i) v[i] = ok ? __ldcs(src + t + i * PL::T) : make_float2(0.f, 0.f);
    run_passes<PL, 0, false, false, 1>(v, t, s, 0, tw);  // X[t + i T], natural order
#pragma unroll
    for (int i = 0; i < PL::R; ++i) {
        const float2 h = __ldg(hs + t + i * PL::T);
        const float2 p = CORR ? cmulc(v[i], h) : cmul(v[i], h);
        v[i] = make_float2(scale * p.x, scale * p.y);
    }
    run_passes<PL, 0, true, false, 1>(v, t, s, 0, tw);  // the inverse, from natural order
    if (ok) {
        float2* dst = out + row * PL::N;
#pragma unroll
        for (int i = 0; i < PL::R; ++i) __stcs(dst + t + i * PL::T, v[i]);
    }
}

namespace {
template <int LOGN>
cudaError_t conv_one(bool corr, const float2* in, float2* out, int64_t nrows, const float2* tw, const float2* hs,
                     float scale, cudaStream_t st) {
    constexpr int RT = rows_rt(LOGN), TPC = rows_tpc_rt(LOGN);
    using CF = RowsCfg<LOGN, TPC, RT>;
    auto kf = k_conv_rows<LOGN, TPC, RT, false>;
    auto kc = k_conv_rows<LOGN, TPC, RT, true>;
    static bool prepared[2] = {false, false};  // the attribute is set once per instantiation
    if (!prepared[corr]) {
        cudaError_t e = cudaFuncSetAttribute(corr ? kc : kf, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM);
        if (e != cudaSuccess) return e;
        prepared[corr] = true;
    }
    if (nrows <= 0) return cudaSuccess;
    const int64_t g = (nrows + TPC - 1) / TPC;
    if (g > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (corr) kc<<<(unsigned)g, CF::THREADS, CF::SMEM, st>>>(in, out, nrows, tw, hs, scale);
    else kf<<<(unsigned)g, CF::THREADS, CF::SMEM, st>>>(in, out, nrows, tw, hs, scale);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_conv_rows(int logn, bool corr, const float2* in, float2* out, int64_t nrows, const float2* tw,
                             const float2* hs, float scale, cudaStream_t st) {
    switch (logn) {
#define B300_C(L) \
    case L:       \
        return conv_one<L>(corr, in, out, nrows, tw, hs, scale, st);
        B300_C(0) B300_C(1) B300_C(2) B300_C(3) B300_C(4) B300_C(5) B300_C(6) B300_C(7) B300_C(8) B300_C(9)
            B300_C(10) B300_C(11) B300_C(12) B300_C(13) B300_C(14)
#undef B300_C
    }
    return cudaErrorInvalidValue;
}

}  // namespace b300fft
