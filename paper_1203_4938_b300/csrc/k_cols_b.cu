// k_cols_b.cu -- columns kernel instantiations, log2 N in {9 10 11 12}.
#include "kernels_launch.cuh"

namespace b300fft {

cudaError_t cols_dispatch_b(int logn, int c, bool prep, bool inv, bool twd, const float2* in, float2* out, int64_t S,
                           int64_t ncols, int64_t item_stride, int64_t nitems, const float2* tw, const float2* lo,
                           const float2* hi, int sh, cudaStream_t st) {
    switch (logn) {
        case 9: return cols_l<9>(c, prep, inv, twd, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
        case 10: return cols_l<10>(c, prep, inv, twd, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
        case 11: return cols_l<11>(c, prep, inv, twd, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
        case 12: return cols_l<12>(c, prep, inv, twd, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace b300fft
