// kernels_launch.cuh -- templated launchers of the power-of-two kernels; each
// k_*.cu file instantiates a subset of lengths so the build parallelises.
#pragma once
#include "launch.h"
#include "stockham_pow2.cuh"

namespace b300fft {

constexpr int kThreadsMax = 1024;

inline cudaError_t grid_of(int64_t units, int per, unsigned* g) {
    const int64_t grid = (units + per - 1) / per;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    *g = (unsigned)grid;
    return cudaSuccess;
}

// ---- plain rows --------------------------------------------------------
// Lengths (bit mask of log2 N) whose rows kernel holds 32 elements per thread
// (two radix-16 butterflies per pass at half the threads, 2 CTAs/SM).
// Measured per 2^27 elements: 2^13 407 us vs 447 us with 16 per thread;
// 2^14 538 us vs 550 us.
#ifndef B300_ROWS_RT32_MASK
#define B300_ROWS_RT32_MASK ((1 << 13) | (1 << 14))
#endif
constexpr int rows_rt(int logn) { return logn >= 5 && ((B300_ROWS_RT32_MASK >> logn) & 1) ? 32 : 16; }
constexpr int rows_tpc_rt(int logn) {
    const int t = logn >= 4 ? (1 << logn) / rows_rt(logn) : 1;
    return t >= 256 ? 1 : 256 / t;
}

template <int LOGN>
cudaError_t rows_prepare_l() {
    constexpr int RT = rows_rt(LOGN), TPC = rows_tpc_rt(LOGN);
    const int sm = RowsCfg<LOGN, TPC, RT>::SMEM;
    cudaError_t e =
        cudaFuncSetAttribute(k_rows_pow2<LOGN, TPC, false, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_rows_pow2<LOGN, TPC, true, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

template <int LOGN>
cudaError_t rows_launch_l(bool inv, const float2* in, float2* out, int64_t nrows, const float2* tw, cudaStream_t st) {
    constexpr int RT = rows_rt(LOGN), TPC = rows_tpc_rt(LOGN);
    using CF = RowsCfg<LOGN, TPC, RT>;
    unsigned g;
    if (nrows <= 0) return cudaSuccess;
    if (grid_of(nrows, TPC, &g) != cudaSuccess) return cudaErrorInvalidConfiguration;
    if (inv) k_rows_pow2<LOGN, TPC, true, RT><<<g, CF::THREADS, CF::SMEM, st>>>(in, out, nrows, tw);
    else k_rows_pow2<LOGN, TPC, false, RT><<<g, CF::THREADS, CF::SMEM, st>>>(in, out, nrows, tw);
    return cudaGetLastError();
}

// ---- transposed rows ----------------------------------------------------
template <int LOGN, int TPC>
constexpr bool rowsT_ok() {
    return TPC * P2Plan<LOGN>::T <= kThreadsMax && P2Plan<LOGN>::NPASS >= 2;
}

template <int LOGN, int TPC>
cudaError_t rowsT_one(bool prep, bool inv, const float2* in, float2* out, int64_t nrows, const float2* tw, int64_t n1,
                      cudaStream_t st) {
    if constexpr (!rowsT_ok<LOGN, TPC>()) {
        return cudaErrorInvalidValue;
    } else {
        using CF = RowsTCfg<LOGN, TPC>;
        if (prep) {
            cudaError_t e = cudaFuncSetAttribute(k_rowsT_pow2<LOGN, TPC, false>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM);
            if (e != cudaSuccess) return e;
            return cudaFuncSetAttribute(k_rowsT_pow2<LOGN, TPC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        CF::SMEM);
        }
        if (n1 % TPC != 0) return cudaErrorInvalidValue;
        unsigned g;
        if (nrows <= 0) return cudaSuccess;
        if (grid_of(nrows, TPC, &g) != cudaSuccess) return cudaErrorInvalidConfiguration;
        if (inv) k_rowsT_pow2<LOGN, TPC, true><<<g, CF::THREADS, CF::SMEM, st>>>(in, out, nrows, tw, n1);
        else k_rowsT_pow2<LOGN, TPC, false><<<g, CF::THREADS, CF::SMEM, st>>>(in, out, nrows, tw, n1);
        return cudaGetLastError();
    }
}

template <int LOGN>
cudaError_t rowsT_l(int tpc, bool prep, bool inv, const float2* in, float2* out, int64_t nrows, const float2* tw,
                    int64_t n1, cudaStream_t st) {
    switch (tpc) {
        case 2: return rowsT_one<LOGN, 2>(prep, inv, in, out, nrows, tw, n1, st);
        case 4: return rowsT_one<LOGN, 4>(prep, inv, in, out, nrows, tw, n1, st);
        case 8: return rowsT_one<LOGN, 8>(prep, inv, in, out, nrows, tw, n1, st);
        case 16: return rowsT_one<LOGN, 16>(prep, inv, in, out, nrows, tw, n1, st);
        case 32: return rowsT_one<LOGN, 32>(prep, inv, in, out, nrows, tw, n1, st);
        case 64: return rowsT_one<LOGN, 64>(prep, inv, in, out, nrows, tw, n1, st);
    }
    return cudaErrorInvalidValue;
}

// ---- columns ------------------------------------------------------------
template <int LOGN, int C>
constexpr bool cols_ok() {
    return C * P2Plan<LOGN>::T <= kThreadsMax;
}

template <int LOGN, int C>
cudaError_t cols_one(bool prep, bool inv, bool twd, const float2* in, float2* out, int64_t S, int64_t ncols,
                     int64_t item_stride, int64_t nitems, const float2* tw, const float2* lo, const float2* hi, int sh,
                     cudaStream_t st) {
    if constexpr (!cols_ok<LOGN, C>()) {
        return cudaErrorInvalidValue;
    } else {
        using CF = ColsCfg<LOGN, C>;
        if (prep) {
            cudaError_t e;
            e = cudaFuncSetAttribute(k_cols_pow2<LOGN, C, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     CF::SMEM);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_cols_pow2<LOGN, C, true, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_cols_pow2<LOGN, C, false, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_cols_pow2<LOGN, C, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         CF::SMEM);
            return e;
        }
        if (ncols % C != 0) return cudaErrorInvalidValue;
        const int64_t groups = ncols / C;
        unsigned g;
        if (groups * nitems <= 0) return cudaSuccess;
        if (grid_of(groups * nitems, 1, &g) != cudaSuccess) return cudaErrorInvalidConfiguration;
#define B300_COLS_LAUNCH(I, W) \
    k_cols_pow2<LOGN, C, I, W><<<g, CF::THREADS, CF::SMEM, st>>>(in, out, S, groups, item_stride, nitems, tw, lo, hi, sh)
        if (inv) {
            if (twd) B300_COLS_LAUNCH(true, true);
            else B300_COLS_LAUNCH(true, false);
        } else {
            if (twd) B300_COLS_LAUNCH(false, true);
            else B300_COLS_LAUNCH(false, false);
        }
#undef B300_COLS_LAUNCH
        return cudaGetLastError();
    }
}

template <int LOGN>
cudaError_t cols_l(int c, bool prep, bool inv, bool twd, const float2* in, float2* out, int64_t S, int64_t ncols,
                   int64_t item_stride, int64_t nitems, const float2* tw, const float2* lo, const float2* hi, int sh,
                   cudaStream_t st) {
#define B300_W(W) \
    case W:       \
        return cols_one<LOGN, W>(prep, inv, twd, in, out, S, ncols, item_stride, nitems, tw, lo, hi, sh, st);
    switch (c) { B300_W(1) B300_W(2) B300_W(4) B300_W(8) B300_W(16) B300_W(32) B300_W(64) }
#undef B300_W
    return cudaErrorInvalidValue;
}

}  // namespace b300fft
