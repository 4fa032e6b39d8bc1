// k_mixed.cu -- instantiations, tables and launcher of the single-pass
// mixed-radix kernel (mixed.cuh) for L = M * 2^K <= 4096, M = 3, 5, 7.
#include "launch.h"
#include "mixed.cuh"

namespace b300fft {

#define B300_MIXED_CASES(X)                                                                                     \
    X(3, 0) X(3, 1) X(3, 2) X(3, 3) X(3, 4) X(3, 5) X(3, 6) X(3, 7) X(3, 8) X(3, 9) X(3, 10) X(5, 0) X(5, 1)    \
    X(5, 2) X(5, 3) X(5, 4) X(5, 5) X(5, 6) X(5, 7) X(5, 8) X(5, 9) X(7, 0) X(7, 1) X(7, 2) X(7, 3) X(7, 4)     \
    X(7, 5) X(7, 6) X(7, 7) X(7, 8) X(7, 9)

bool mixed_supported(int64_t n, int* m, int* k) {
    for (int mm : {3, 5, 7}) {
        if (n % mm) continue;
        const int64_t q = n / mm;
        if (q < 1 || (q & (q - 1)) || n > 4096) continue;
        int kk = 0;
        while ((int64_t(1) << kk) < q) ++kk;
        *m = mm;
        *k = kk;
        return true;
    }
    return false;
}

// Column tiles of the mixed four-step: N1 = M * 2^A with NL = the largest power
// of two <= 4096 / N1 adjacent columns per CTA (at least 8: 64-byte rows).
#define B300_MIXED_COLS(X)                                                                             \
    X(3, 2, 256) X(3, 3, 128) X(3, 4, 64) X(3, 5, 32) X(3, 6, 16) X(3, 7, 8) X(5, 2, 128) X(5, 3, 64)      \
    X(5, 4, 32) X(5, 5, 16) X(5, 6, 8) X(7, 2, 128) X(7, 3, 64) X(7, 4, 32) X(7, 5, 16) X(7, 6, 8)

int mixed_cols_width(int m, int a) {
#define B300_X(M, A, NL) \
    if (m == M && a == A) return NL;
    B300_MIXED_COLS(B300_X)
#undef B300_X
    return 0;
}

cudaError_t launch_cols_mixed(int m, int a, bool inv, const float2* in, float2* out, int64_t S2, int64_t items,
                              const float2* tw, const float2* lo, const float2* hi, int sh, cudaStream_t st) {
#define B300_X(M, A, NL)                                                                                         \
    if (m == M && a == A) {                                                                                      \
        if (S2 % NL != 0 || items <= 0) return cudaErrorInvalidValue;                                          \
        const int64_t g = items * (S2 / NL);                                                                     \
        if (g > 0x7fffffffLL) return cudaErrorInvalidConfiguration;                                             \
        if (inv) k_cols_mixed<M, A, NL, true><<<(unsigned)g, 256, 0, st>>>(in, out, S2, items, tw, lo, hi, sh); \
        else k_cols_mixed<M, A, NL, false><<<(unsigned)g, 256, 0, st>>>(in, out, S2, items, tw, lo, hi, sh);    \
        return cudaGetLastError();                                                                               \
    }
    B300_MIXED_COLS(B300_X)
#undef B300_X
    return cudaErrorInvalidValue;
}

// Column pass of a 2-D transform with a side of M * 2^K: NL = min(32, the
// largest power of two <= 4096 / L) adjacent columns per CTA.
#define B300_MIXED_COLS2D(X)                                                                                  \
    X(3, 0, 32) X(3, 1, 32) X(3, 2, 32) X(3, 3, 32) X(3, 4, 32) X(3, 5, 32) X(3, 6, 16) X(3, 7, 8) X(3, 8, 4)   \
    X(3, 9, 2) X(3, 10, 1) X(5, 0, 32) X(5, 1, 32) X(5, 2, 32) X(5, 3, 32) X(5, 4, 32) X(5, 5, 16) X(5, 6, 8)   \
    X(5, 7, 4) X(5, 8, 2) X(5, 9, 1) X(7, 0, 32) X(7, 1, 32) X(7, 2, 32) X(7, 3, 32) X(7, 4, 32) X(7, 5, 16)    \
    X(7, 6, 8) X(7, 7, 4) X(7, 8, 2) X(7, 9, 1)

int mixed_cols2d_width(int m, int k) {
#define B300_X(M, K, NL) \
    if (m == M && k == K) return NL;
    B300_MIXED_COLS2D(B300_X)
#undef B300_X
    return 0;
}

cudaError_t launch_cols2d_mixed(int m, int k, bool inv, const float2* in, float2* out, int64_t S2, int64_t items,
                                const float2* tw, cudaStream_t st) {
#define B300_X(M, K, NL)                                                                                        \
    if (m == M && k == K) {                                                                                     \
        if (S2 % NL != 0 || items <= 0) return cudaErrorInvalidValue;                                         \
        const int64_t g = items * (S2 / NL);                                                                    \
        if (g > 0x7fffffffLL) return cudaErrorInvalidConfiguration;                                            \
        if (inv)                                                                                                \
            k_cols_mixed<M, K, NL, true, false><<<(unsigned)g, 256, 0, st>>>(in, out, S2, items, tw, nullptr,   \
                                                                               nullptr, 0);                     \
        else                                                                                                    \
            k_cols_mixed<M, K, NL, false, false><<<(unsigned)g, 256, 0, st>>>(in, out, S2, items, tw, nullptr,  \
                                                                                nullptr, 0);                    \
        return cudaGetLastError();                                                                              \
    }
    B300_MIXED_COLS2D(B300_X)
#undef B300_X
    return cudaErrorInvalidValue;
}

namespace {
template <int M, int K>
cudaError_t one(int op, bool inv, const float2* in, float2* out, int64_t nrows, const float2* tw, cudaStream_t st,
                int* info) {
    using MP = MixPlan<M, K>;
    if (op == 0) {  // table entries, lines per CTA
        info[0] = MP::TWSIZE;
        info[1] = MP::NL;
        return cudaSuccess;
    }
    if (op == 1) {  // pass tables, FP64 on the device
        for (int p = 1; p < MP::NPASS; ++p) {
            cudaError_t e = gen_pass_table(out + MP::twoff(p), MP::ns(p), MP::radix(p), st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (nrows <= 0) return cudaSuccess;
    const int64_t g = (nrows + MP::NL - 1) / MP::NL;
    if (g > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (inv) k_rows_mixed<M, K, true><<<(unsigned)g, MP::THREADS, 0, st>>>(in, out, nrows, tw);
    else k_rows_mixed<M, K, false><<<(unsigned)g, MP::THREADS, 0, st>>>(in, out, nrows, tw);
    return cudaGetLastError();
}

// Tables of the power-of-two lines the stage-graph executor runs with the
// same compile-time passes (M = 1): no kernel of their own.
template <int K>
cudaError_t pow2_lines_table(int op, float2* out, cudaStream_t st, int* info) {
    using MP = MixPlan<1, K>;
    if (op == 0) {
        info[0] = MP::TWSIZE;
        info[1] = MP::NL;
        return cudaSuccess;
    }
    if (op != 1) return cudaErrorInvalidValue;
    for (int p = 1; p < MP::NPASS; ++p) {
        cudaError_t e = gen_pass_table(out + MP::twoff(p), MP::ns(p), MP::radix(p), st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t dispatch(int m, int k, int op, bool inv, const float2* in, float2* out, int64_t nrows, const float2* tw,
                     cudaStream_t st, int* info) {
#define B300_X(M, K) \
    if (m == M && k == K) return one<M, K>(op, inv, in, out, nrows, tw, st, info);
    B300_MIXED_CASES(B300_X)
#undef B300_X
    if (m == 1) {
        switch (k) {
#define B300_P(K) \
    case K:       \
        return pow2_lines_table<K>(op, out, st, info);
            B300_P(4) B300_P(5) B300_P(6) B300_P(7) B300_P(8) B300_P(9) B300_P(10) B300_P(11) B300_P(12)
#undef B300_P
            default:
                break;
        }
    }
    return cudaErrorInvalidValue;
}
}  // namespace

int mixed_table_entries(int m, int k) {
    int info[2] = {0, 0};
    return dispatch(m, k, 0, false, nullptr, nullptr, 0, nullptr, 0, info) == cudaSuccess ? info[0] : -1;
}

int mixed_lines_per_cta(int m, int k) {
    int info[2] = {0, 0};
    return dispatch(m, k, 0, false, nullptr, nullptr, 0, nullptr, 0, info) == cudaSuccess ? info[1] : -1;
}

cudaError_t gen_mixed_table(float2* tw, int m, int k, cudaStream_t st) {
    return dispatch(m, k, 1, false, nullptr, tw, 0, nullptr, st, nullptr);
}

cudaError_t launch_rows_mixed(int m, int k, bool inv, const float2* in, float2* out, int64_t nrows, const float2* tw,
                              cudaStream_t st) {
    return dispatch(m, k, 2, inv, in, out, nrows, tw, st, nullptr);
}

}  // namespace b300fft
