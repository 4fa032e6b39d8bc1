// k_three.cu -- instantiations and launcher of the three-stage persistent
// kernel (threestep.cuh).  Each (LA, LB1, LB2, TILE) is a candidate split of
// log2 N into three stage lengths of 2^6 .. 2^8 points with a tile size.
#include "launch.h"
#include "threestep.cuh"

namespace b300fft {

// (16384-point tiles on 1024 threads compile and are exact, but measured
// 25-30 % slower at 2^21..2^24, so none is instantiated.)
#define B300_THREE_CONFIGS(X)                                                                          \
    X(6, 6, 7, 4096) X(7, 7, 6, 4096) X(6, 7, 7, 4096) X(7, 7, 7, 4096) X(7, 7, 8, 4096) X(8, 7, 8, 4096) \
        X(7, 8, 8, 4096) X(8, 8, 8, 4096)

namespace {
template <int LA, int LB1, int LB2, int TILE>
cudaError_t one(int op, bool inv, const ThreeArgs* a, int grid, cudaStream_t st, PersistInfo* info) {
    using CF = ThreeCfg<LA, LB1, LB2, TILE>;
    auto kf = k_threestep<LA, LB1, LB2, false, TILE>;
    auto ki = k_threestep<LA, LB1, LB2, true, TILE>;
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
    // tensor maps of the L2 prefetches: the input as [batch * N1][N2] (A
    // boxes of CA x N1), the workspace as [batch * N1 * M1][M2] (B1 boxes of
    // CB x M1); unused (and not encoded) when a->prefetch is 0
    CUtensorMap t_in{}, t_b1{};
    ThreeArgs aa = *a;
    if (aa.prefetch) {
        const uint64_t B = (uint64_t)aa.batch, N1 = CF::N1, M1 = CF::M1, M2 = CF::M2, N2 = CF::N2;
        const uint64_t d0[2] = {N2, B * N1}, s0[1] = {N2 * 8};
        const uint32_t b0[2] = {(uint32_t)CF::CA, (uint32_t)N1};
        const uint64_t d1[2] = {M2, B * N1 * M1}, s1[1] = {M2 * 8};
        const uint32_t b1[2] = {(uint32_t)CF::CB, (uint32_t)M1};
        if (!encode_tensor_map(&t_in, aa.in, 2, d0, s0, b0) || !encode_tensor_map(&t_b1, aa.work, 2, d1, s1, b1))
            aa.prefetch = 0;
    }
    if (inv) ki<<<grid, CF::THREADS, CF::SMEM, st>>>(aa, t_in, t_b1);
    else kf<<<grid, CF::THREADS, CF::SMEM, st>>>(aa, t_in, t_b1);
    return cudaGetLastError();
}

cudaError_t dispatch(const ThreeConfig& c, int op, bool inv, const ThreeArgs* a, int grid, cudaStream_t st,
                     PersistInfo* info) {
#define B300_X(LA, LB1, LB2, TILE)                                       \
    if (c.la == LA && c.lb1 == LB1 && c.lb2 == LB2 && c.tile == TILE) \
        return one<LA, LB1, LB2, TILE>(op, inv, a, grid, st, info);
    B300_THREE_CONFIGS(B300_X)
#undef B300_X
    return cudaErrorInvalidValue;
}
}  // namespace

bool three_config_available(const ThreeConfig& c) {
#define B300_X(LA, LB1, LB2, TILE) \
    if (c.la == LA && c.lb1 == LB1 && c.lb2 == LB2 && c.tile == TILE) return true;
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
