// k_rows.cu -- plain rows kernel, log2 N in [0, 14].
#include "kernels_launch.cuh"

namespace b300fft {

#define B300_PLAIN_CASES(X) X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14)

int rows_tpc(int logn) { return rows_tpc_rt(logn); }
int rows_threads(int logn) { return (logn >= 4 ? (1 << logn) / rows_rt(logn) : 1) * rows_tpc_rt(logn); }

cudaError_t rows_prepare(int logn) {
    switch (logn) {
#define B300_C(L) \
    case L:       \
        return rows_prepare_l<L>();
        B300_PLAIN_CASES(B300_C)
#undef B300_C
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_rows(int logn, bool inv, const float2* in, float2* out, int64_t nrows, const float2* tw,
                        cudaStream_t st) {
    switch (logn) {
#define B300_C(L) \
    case L:       \
        return rows_launch_l<L>(inv, in, out, nrows, tw, st);
        B300_PLAIN_CASES(B300_C)
#undef B300_C
    }
    return cudaErrorInvalidValue;
}

}  // namespace b300fft
