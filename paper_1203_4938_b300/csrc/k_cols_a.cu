// k_cols_a.cu -- columns kernel instantiations, log2 N in {1 2 3 4 5 6 7 8}.
#include "kernels_launch.cuh"

namespace b300fft {

cudaError_t cols_dispatch_a(int logn, int c, bool prep, bool inv, bool twd, const float2* in, float2* out, int64_t S,
                           int64_t ncols, int64_t item_stride, int64_t nitems, const float2* tw, const float2* lo,
                           const float2* hi, int sh, cudaStream_t st) {
    switch (logn) {
        case 1: return cols_l<1>(c, prep, inv, twd, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
        case 2: return cols_l<2>(c, prep, inv, twd, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
        case 3: return cols_l<3>(c, prep, inv, twd, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
        case 4: return cols_l<4>(c, prep, inv, twd, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
        case 5: return cols_l<5>(c, prep, inv, twd, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
        case 6: return cols_l<6>(c, prep, inv, twd, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
        case 7: return cols_l<7>(c, prep, inv, twd, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
        case 8: return cols_l<8>(c, prep, inv, twd, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace b300fft
