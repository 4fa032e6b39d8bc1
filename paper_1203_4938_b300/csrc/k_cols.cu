// k_cols.cu -- instantiations and launcher of the power-of-two columns kernel
// (2-D column pass; four-step first pass with the inter-pass twiddle).
#include "launch.h"
#include "stockham_pow2.cuh"

namespace b300fft {

namespace {
constexpr int width_of(int logn) {
    const int c = 16384 >> logn;
    return c < 4 ? 4 : (c > 64 ? 64 : c);
}

template <int LOGN, int C>
cudaError_t prepare_one() {
    const int smem = ColsCfg<LOGN, C>::SMEM;
    cudaError_t e;
    e = cudaFuncSetAttribute(k_cols_pow2<LOGN, C, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_cols_pow2<LOGN, C, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if constexpr (C == width_of(LOGN)) {
        e = cudaFuncSetAttribute(k_cols_pow2<LOGN, C, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_cols_pow2<LOGN, C, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
    }
    return e;
}

template <int LOGN, int C>
cudaError_t launch_one(bool inv, bool tw_out, const float2* in, float2* out, int64_t S, int64_t ncols,
                       int64_t item_stride, int64_t nitems, const float2* tw, const float2* lo, const float2* hi,
                       int sh, cudaStream_t st) {
    using CF = ColsCfg<LOGN, C>;
    if (ncols % C != 0) return cudaErrorInvalidValue;
    const int64_t groups = ncols / C;
    const int64_t grid = groups * nitems;
    if (grid <= 0) return cudaSuccess;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const unsigned g = (unsigned)grid;
    if constexpr (C == width_of(LOGN)) {
        if (tw_out) {
            if (inv)
                k_cols_pow2<LOGN, C, true, true><<<g, CF::THREADS, CF::SMEM, st>>>(in, out, S, groups, item_stride,
                                                                                     nitems, tw, lo, hi, sh);
            else
                k_cols_pow2<LOGN, C, false, true><<<g, CF::THREADS, CF::SMEM, st>>>(in, out, S, groups, item_stride,
                                                                                      nitems, tw, lo, hi, sh);
            return cudaGetLastError();
        }
    } else {
        if (tw_out) return cudaErrorInvalidValue;
    }
    if (inv)
        k_cols_pow2<LOGN, C, true, false><<<g, CF::THREADS, CF::SMEM, st>>>(in, out, S, groups, item_stride, nitems,
                                                                              tw, lo, hi, sh);
    else
        k_cols_pow2<LOGN, C, false, false><<<g, CF::THREADS, CF::SMEM, st>>>(in, out, S, groups, item_stride,
                                                                               nitems, tw, lo, hi, sh);
    return cudaGetLastError();
}

// Widths instantiated per length: the default, 4 and 1 (for narrow arrays).
template <int LOGN>
cudaError_t prepare_w(int c) {
    constexpr int D = width_of(LOGN);
    if (c == D) return prepare_one<LOGN, D>();
    if constexpr (D > 4) {
        if (c == 4) return prepare_one<LOGN, 4>();
    }
    if (c == 1) return prepare_one<LOGN, 1>();
    return cudaErrorInvalidValue;
}

template <int LOGN>
cudaError_t launch_w(int c, bool inv, bool tw_out, const float2* in, float2* out, int64_t S, int64_t ncols,
                     int64_t item_stride, int64_t nitems, const float2* tw, const float2* lo, const float2* hi, int sh,
                     cudaStream_t st) {
    constexpr int D = width_of(LOGN);
    if (c == D) return launch_one<LOGN, D>(inv, tw_out, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
    if constexpr (D > 4) {
        if (c == 4)
            return launch_one<LOGN, 4>(inv, tw_out, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
    }
    if (c == 1) return launch_one<LOGN, 1>(inv, tw_out, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
    return cudaErrorInvalidValue;
}
}  // namespace

#define B300_COLS_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)

int cols_width(int logn) { return width_of(logn); }

int cols_width_for(int logn, int64_t ncols) {
    const int d = width_of(logn);
    if (ncols % d == 0) return d;
    if (ncols % 4 == 0) return 4;
    return 1;
}

int cols_threads(int logn, int c) { return (logn >= 4 ? (1 << logn) / 16 : 1) * c; }

int cols_smem(int logn, int c) {
    const int n = 1 << logn;
    const int npass = logn >= 4 ? logn / 4 + (logn % 4 ? 1 : 0) : 1;
    return npass > 1 ? padi(n * c) * 8 : 0;
}

cudaError_t cols_prepare(int logn, int c) {
    switch (logn) {
#define B300_C(L) \
    case L:       \
        return prepare_w<L>(c);
        B300_COLS_CASES(B300_C)
#undef B300_C
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_cols(int logn, int c, bool inv, bool twiddle_out, const float2* in, float2* out, int64_t S,
                        int64_t ncols, int64_t item_stride, int64_t nitems, const float2* tw, const float2* lo,
                        const float2* hi, int sh, cudaStream_t st) {
    switch (logn) {
#define B300_C(L) \
    case L:       \
        return launch_w<L>(c, inv, twiddle_out, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
        B300_COLS_CASES(B300_C)
#undef B300_C
    }
    return cudaErrorInvalidValue;
}

}  // namespace b300fft
