// k_2d.cu -- instantiations and launcher of the persistent 2-D kernel
// (persist2d.cuh).  Each (LW, TPC, LH, C) is a candidate square-image tiling.
#include "launch.h"
#include "persist2d.cuh"

namespace b300fft {

#define B300_2D_CONFIGS(X) \
    X(9, 8, 9, 8) X(9, 16, 9, 16) X(10, 8, 10, 8) X(10, 16, 10, 16) X(11, 4, 11, 4) X(11, 8, 11, 8)

namespace {
template <int LW, int TPC, int LH, int C>
cudaError_t one(int op, bool inv, const PersistArgs* a, int grid, cudaStream_t st, PersistInfo* info) {
    using CF = TwoDPersistCfg<LW, TPC, LH, C>;
    auto kf = k_2d_persist<LW, TPC, LH, C, false>;
    auto ki = k_2d_persist<LW, TPC, LH, C, true>;
    if (op == 0) {
        cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(ki, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kf, CF::THREADS, CF::SMEM);
        info->threads = CF::THREADS;
        info->smem = CF::SMEM;
        info->blocks_per_sm = nb;
        return e;
    }
    if (inv) ki<<<grid, CF::THREADS, CF::SMEM, st>>>(*a);
    else kf<<<grid, CF::THREADS, CF::SMEM, st>>>(*a);
    return cudaGetLastError();
}

cudaError_t dispatch(const PersistConfig& c, int op, bool inv, const PersistArgs* a, int grid, cudaStream_t st,
                     PersistInfo* info) {
#define B300_X(LW, TPC, LH, C) \
    if (c.l1 == LW && c.c == TPC && c.l2 == LH && c.tpc == C) return one<LW, TPC, LH, C>(op, inv, a, grid, st, info);
    B300_2D_CONFIGS(B300_X)
#undef B300_X
    return cudaErrorInvalidValue;
}
}  // namespace

// PersistConfig fields reused: l1 = log2 W, c = rows per A tile, l2 = log2 H, tpc = columns per B tile.
bool persist2d_config_available(const PersistConfig& c) {
#define B300_X(LW, TPC, LH, C) \
    if (c.l1 == LW && c.c == TPC && c.l2 == LH && c.tpc == C) return true;
    B300_2D_CONFIGS(B300_X)
#undef B300_X
    return false;
}

cudaError_t persist2d_prepare(const PersistConfig& c, PersistInfo* info) {
    return dispatch(c, 0, false, nullptr, 0, 0, info);
}

cudaError_t launch_2d_persist(const PersistConfig& c, bool inv, const PersistArgs& a, int grid, cudaStream_t st) {
    return dispatch(c, 1, inv, &a, grid, st, nullptr);
}

}  // namespace b300fft
