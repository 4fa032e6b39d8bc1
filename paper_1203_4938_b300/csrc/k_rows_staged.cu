// k_rows_staged.cu -- instantiations and launcher of the persistent rows
// kernel with bulk-copied input staging (rows_staged.cuh), 2^13 and 2^14.
#include "launch.h"
#include "rows_staged.cuh"

namespace b300fft {

namespace {
template <int LOGN>
cudaError_t one(int op, bool inv, const float2* in, float2* out, int64_t nrows, const float2* tw, int* status,
                int64_t polls, int grid, cudaStream_t st, PersistInfo* info) {
    using CF = StagedCfg<LOGN>;
    auto kf = k_rows_staged<LOGN, false>;
    auto ki = k_rows_staged<LOGN, true>;
    if (op == 0) {
        cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(ki, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kf, CF::THREADS, CF::SMEM);
        if (e != cudaSuccess) return e;
        info->threads = CF::THREADS;
        info->smem = CF::SMEM;
        info->blocks_per_sm = nb;
        return cudaSuccess;
    }
    if (nrows <= 0) return cudaSuccess;
    if (inv) ki<<<grid, CF::THREADS, CF::SMEM, st>>>(in, out, nrows, tw, status, polls);
    else kf<<<grid, CF::THREADS, CF::SMEM, st>>>(in, out, nrows, tw, status, polls);
    return cudaGetLastError();
}

cudaError_t dispatch(int logn, int op, bool inv, const float2* in, float2* out, int64_t nrows, const float2* tw,
                     int* status, int64_t polls, int grid, cudaStream_t st, PersistInfo* info) {
    switch (logn) {
        case 13:
            return one<13>(op, inv, in, out, nrows, tw, status, polls, grid, st, info);
        case 14:
            return one<14>(op, inv, in, out, nrows, tw, status, polls, grid, st, info);
    }
    return cudaErrorInvalidValue;
}
}  // namespace

bool rows_staged_available(int logn) { return logn == 13 || logn == 14; }

cudaError_t rows_staged_prepare(int logn, PersistInfo* info) {
    return dispatch(logn, 0, false, nullptr, nullptr, 0, nullptr, nullptr, 0, 0, 0, info);
}

cudaError_t launch_rows_staged(int logn, bool inv, const float2* in, float2* out, int64_t nrows, const float2* tw,
                               int* status, int64_t polls, int grid, cudaStream_t st) {
    return dispatch(logn, 1, inv, in, out, nrows, tw, status, polls, grid, st, nullptr);
}

}  // namespace b300fft
