// k_three.cu -- instantiations and launcher of the three-stage persistent
// kernel (threestep.cuh).  Each (LA, LB1, LB2) is a candidate split of
// log2 N into three stage lengths of 2^6 .. 2^8 points.
#include "launch.h"
#include "threestep.cuh"

namespace b300fft {

#define B300_THREE_CONFIGS(X) X(6, 6, 7) X(7, 7, 6) X(6, 7, 7) X(7, 7, 7) X(7, 7, 8) X(8, 7, 8) X(7, 8, 8) X(8, 8, 8)

namespace {
template <int LA, int LB1, int LB2>
cudaError_t one(int op, bool inv, const ThreeArgs* a, int grid, cudaStream_t st, PersistInfo* info) {
    using CF = ThreeCfg<LA, LB1, LB2>;
    auto kf = k_threestep<LA, LB1, LB2, false>;
    auto ki = k_threestep<LA, LB1, LB2, true>;
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
    if (inv) ki<<<grid, CF::THREADS, CF::SMEM, st>>>(*a);
    else kf<<<grid, CF::THREADS, CF::SMEM, st>>>(*a);
    return cudaGetLastError();
}

cudaError_t dispatch(const ThreeConfig& c, int op, bool inv, const ThreeArgs* a, int grid, cudaStream_t st,
                     PersistInfo* info) {
#define B300_X(LA, LB1, LB2) \
    if (c.la == LA && c.lb1 == LB1 && c.lb2 == LB2) return one<LA, LB1, LB2>(op, inv, a, grid, st, info);
    B300_THREE_CONFIGS(B300_X)
#undef B300_X
    return cudaErrorInvalidValue;
}
}  // namespace

bool three_config_available(const ThreeConfig& c) {
#define B300_X(LA, LB1, LB2) \
    if (c.la == LA && c.lb1 == LB1 && c.lb2 == LB2) return true;
    B300_THREE_CONFIGS(B300_X)
#undef B300_X
    return false;
}

cudaError_t three_prepare(const ThreeConfig& c, PersistInfo* info) {
    return dispatch(c, 0, false, nullptr, 0, 0, info);
}

cudaError_t launch_threestep(const ThreeConfig& c, bool inv, const ThreeArgs& a, int grid, cudaStream_t st) {
    return dispatch(c, 1, inv, &a, grid, st, nullptr);
}

}  // namespace b300fft
