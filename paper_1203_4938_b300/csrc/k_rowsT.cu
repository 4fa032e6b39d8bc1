// k_rowsT.cu -- transposed rows kernel (four-step second pass), log2 N in [5, 12].
#include "kernels_launch.cuh"

namespace b300fft {

cudaError_t rowsT_dispatch(int logn, int tpc, bool prep, bool inv, const float2* in, float2* out, int64_t nrows,
                           const float2* tw, int64_t n1, cudaStream_t st) {
    switch (logn) {
#define B300_C(L) \
    case L:       \
        return rowsT_l<L>(tpc, prep, inv, in, out, nrows, tw, n1, st);
        B300_C(5) B300_C(6) B300_C(7) B300_C(8) B300_C(9) B300_C(10) B300_C(11) B300_C(12)
#undef B300_C
    }
    return cudaErrorInvalidValue;
}

int rowsT_threads(int logn, int tpc) { return (1 << logn) / 16 * tpc; }

cudaError_t rowsT_prepare(int logn, int tpc) {
    return rowsT_dispatch(logn, tpc, true, false, nullptr, nullptr, 0, nullptr, 0, 0);
}

cudaError_t launch_rowsT(int logn, int tpc, bool inv, const float2* in, float2* out, int64_t nrows, const float2* tw,
                         int64_t n1, cudaStream_t st) {
    return rowsT_dispatch(logn, tpc, false, inv, in, out, nrows, tw, n1, st);
}

}  // namespace b300fft
