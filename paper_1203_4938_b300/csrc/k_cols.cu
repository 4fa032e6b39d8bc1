// k_cols.cu -- columns kernel: width selection and dispatch over lengths.
#include "kernels_launch.cuh"

namespace b300fft {

cudaError_t cols_dispatch_a(int, int, bool, bool, bool, const float2*, float2*, int64_t, int64_t, int64_t, int64_t,
                            const float2*, const float2*, const float2*, int, cudaStream_t);
cudaError_t cols_dispatch_b(int, int, bool, bool, bool, const float2*, float2*, int64_t, int64_t, int64_t, int64_t,
                            const float2*, const float2*, const float2*, int, cudaStream_t);

namespace {
cudaError_t dispatch(int logn, int c, bool prep, bool inv, bool twd, const float2* in, float2* out, int64_t S,
                     int64_t ncols, int64_t item_stride, int64_t nitems, const float2* tw, const float2* lo,
                     const float2* hi, int sh, cudaStream_t st) {
    if (logn >= 1 && logn <= 8)
        return cols_dispatch_a(logn, c, prep, inv, twd, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
    if (logn >= 9 && logn <= 12)
        return cols_dispatch_b(logn, c, prep, inv, twd, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
    return cudaErrorInvalidValue;
}
}  // namespace

bool cols_width_valid(int logn, int c) {
    const int t = logn >= 4 ? (1 << logn) / 16 : 1;
    return logn >= 1 && logn <= kColsMaxLog && (c & (c - 1)) == 0 && c >= 1 && c <= 64 && c * t <= kThreadsMax;
}

int cols_width(int logn) {
    const int c = 16384 >> logn;
    int w = c < 4 ? 4 : (c > 64 ? 64 : c);
    while (w > 1 && !cols_width_valid(logn, w)) w /= 2;
    while (w < 64 && !cols_width_valid(logn, w)) w *= 2;
    return w;
}

int cols_width_for(int logn, int64_t ncols) {
    for (int w = cols_width(logn); w >= 1; w /= 2)
        if (ncols % w == 0 && cols_width_valid(logn, w)) return w;
    return 0;
}

int cols_threads(int logn, int c) { return (logn >= 4 ? (1 << logn) / 16 : 1) * c; }

cudaError_t cols_prepare(int logn, int c) {
    return dispatch(logn, c, true, false, false, nullptr, nullptr, 0, 0, 0, 0, nullptr, nullptr, nullptr, 0, 0);
}

cudaError_t launch_cols(int logn, int c, bool inv, bool twiddle_out, const float2* in, float2* out, int64_t S,
                        int64_t ncols, int64_t item_stride, int64_t nitems, const float2* tw, const float2* lo,
                        const float2* hi, int sh, cudaStream_t st) {
    return dispatch(logn, c, false, inv, twiddle_out, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
}

}  // namespace b300fft
