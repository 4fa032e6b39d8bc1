// k_rows.cu -- instantiations and launcher of the power-of-two rows kernel
// (contiguous batched transforms, and the four-step second pass with its
// transposed store).
#include "launch.h"
#include "stockham_pow2.cuh"

namespace b300fft {

namespace {
constexpr int plain_tpc(int logn) {
    const int t = logn >= 4 ? (1 << logn) / 16 : 1;
    return t >= 256 ? 1 : 256 / t;
}
constexpr int trans_tpc(int logn) {
    const int c = 16384 >> logn;
    return c < 4 ? 4 : (c > 64 ? 64 : c);
}

template <int LOGN, bool TR>
constexpr int tpc_of() {
    return TR ? trans_tpc(LOGN) : plain_tpc(LOGN);
}

template <int LOGN, bool TR>
int smem_of() {
    using CF = RowsCfg<LOGN, tpc_of<LOGN, TR>()>;
    return TR ? CF::SMEM_T : CF::SMEM_PLAIN;
}

template <int LOGN, bool TR>
cudaError_t prepare_one() {
    constexpr int TPC = tpc_of<LOGN, TR>();
    const int smem = smem_of<LOGN, TR>();
    cudaError_t e = cudaFuncSetAttribute(k_rows_pow2<LOGN, TPC, false, TR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_rows_pow2<LOGN, TPC, true, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem);
}

template <int LOGN, bool TR>
cudaError_t launch_one(bool inv, const float2* in, float2* out, int64_t nrows, const float2* tw, int64_t n1,
                       cudaStream_t st) {
    constexpr int TPC = tpc_of<LOGN, TR>();
    using CF = RowsCfg<LOGN, TPC>;
    const int smem = smem_of<LOGN, TR>();
    const int64_t grid = (nrows + TPC - 1) / TPC;
    if (grid <= 0) return cudaSuccess;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (inv)
        k_rows_pow2<LOGN, TPC, true, TR><<<(unsigned)grid, CF::THREADS, smem, st>>>(in, out, nrows, tw, n1);
    else
        k_rows_pow2<LOGN, TPC, false, TR><<<(unsigned)grid, CF::THREADS, smem, st>>>(in, out, nrows, tw, n1);
    return cudaGetLastError();
}
}  // namespace

// Plain rows: log2 N in [0, 14]; transposed (four-step pass 2): [5, 12].
#define B300_PLAIN_CASES(X) X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14)
#define B300_TRANS_CASES(X) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)

int rows_tpc(int logn, bool transposed) { return transposed ? trans_tpc(logn) : plain_tpc(logn); }

int rows_threads(int logn, bool transposed) {
    const int t = logn >= 4 ? (1 << logn) / 16 : 1;
    return t * rows_tpc(logn, transposed);
}

int rows_smem(int logn, bool transposed) {
    if (transposed) {
        switch (logn) {
#define B300_C(L) \
    case L:       \
        return smem_of<L, true>();
            B300_TRANS_CASES(B300_C)
#undef B300_C
        }
    } else {
        switch (logn) {
#define B300_C(L) \
    case L:       \
        return smem_of<L, false>();
            B300_PLAIN_CASES(B300_C)
#undef B300_C
        }
    }
    return -1;
}

cudaError_t rows_prepare(int logn, bool transposed) {
    if (transposed) {
        switch (logn) {
#define B300_C(L) \
    case L:       \
        return prepare_one<L, true>();
            B300_TRANS_CASES(B300_C)
#undef B300_C
        }
    } else {
        switch (logn) {
#define B300_C(L) \
    case L:       \
        return prepare_one<L, false>();
            B300_PLAIN_CASES(B300_C)
#undef B300_C
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_rows(int logn, bool inv, bool transposed, const float2* in, float2* out, int64_t nrows,
                        const float2* tw, int64_t n1, cudaStream_t st) {
    if (transposed) {
        switch (logn) {
#define B300_C(L) \
    case L:       \
        return launch_one<L, true>(inv, in, out, nrows, tw, n1, st);
            B300_TRANS_CASES(B300_C)
#undef B300_C
        }
    } else {
        switch (logn) {
#define B300_C(L) \
    case L:       \
        return launch_one<L, false>(inv, in, out, nrows, tw, n1, st);
            B300_PLAIN_CASES(B300_C)
#undef B300_C
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace b300fft
