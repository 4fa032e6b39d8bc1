// k_persist.cu -- instantiations and launcher of the persistent four-step
// kernel (persist.cuh).  Each (L1, C, L2, TPC) below is a measured or
// candidate configuration for one log2 N (tiles of 4096, 8192 or 16384
// points on 256, 512 or 1024 threads).  The half-width 2^24 shape
// (12, 2, 12, 2) is deliberately absent: a build of it (with a cp.async
// prefetch stage since removed) stopped once with an illegal instruction whose
// cause was not found, so it is neither built nor reachable.
#include "launch.h"
#include "persist.cuh"

namespace b300fft {

#define B300_PERSIST_CONFIGS(X)                                                                             \
    X(6, 32, 7, 16) X(7, 16, 7, 16) X(7, 32, 7, 32) X(7, 32, 8, 16)                                           \
    X(7, 16, 8, 8) X(8, 16, 8, 16) X(8, 8, 8, 8) X(8, 16, 9, 8) X(9, 8, 9, 8) X(8, 16, 10, 4) X(9, 8, 10, 4) \
        X(9, 16, 10, 8) X(10, 4, 10, 4) X(10, 8, 10, 8) X(10, 4, 11, 2) X(11, 4, 10, 8) X(11, 4, 11, 4)     \
            X(11, 2, 11, 2) X(11, 4, 12, 2) X(12, 4, 11, 8) X(12, 4, 12, 4) X(10, 8, 11, 4) X(10, 16, 11, 8)    \
                X(11, 8, 11, 8) X(11, 8, 10, 16) X(10, 16, 10, 16) X(9, 32, 10, 16) X(9, 32, 9, 32)              \
                    X(8, 64, 10, 16) X(8, 64, 9, 32) X(8, 64, 8, 64) X(10, 16, 12, 4) X(11, 8, 12, 4)

namespace {
template <int L1, int C, int L2, int TPC>
cudaError_t one(int op, bool inv, const PersistArgs* a, int grid, cudaStream_t st, PersistInfo* info) {
    using CF = FourStepPersistCfg<L1, C, L2, TPC>;
    auto kf = k_fourstep_persist<L1, C, L2, TPC, false>;
    auto ki = k_fourstep_persist<L1, C, L2, TPC, true>;
    if (op == 0) {  // prepare
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

cudaError_t dispatch(const PersistConfig& c, int op, bool inv, const PersistArgs* a, int grid, cudaStream_t st,
                     PersistInfo* info) {
#define B300_X(L1, C, L2, TPC) \
    if (c.l1 == L1 && c.c == C && c.l2 == L2 && c.tpc == TPC) return one<L1, C, L2, TPC>(op, inv, a, grid, st, info);
    B300_PERSIST_CONFIGS(B300_X)
#undef B300_X
    return cudaErrorInvalidValue;
}
}  // namespace

bool persist_config_available(const PersistConfig& c) {
#define B300_X(L1, C, L2, TPC) \
    if (c.l1 == L1 && c.c == C && c.l2 == L2 && c.tpc == TPC) return true;
    B300_PERSIST_CONFIGS(B300_X)
#undef B300_X
    return false;
}

cudaError_t persist_prepare(const PersistConfig& c, PersistInfo* info) {
    return dispatch(c, 0, false, nullptr, 0, 0, info);
}

cudaError_t launch_fourstep_persist(const PersistConfig& c, bool inv, const PersistArgs& a, int grid,
                                    cudaStream_t st) {
    return dispatch(c, 1, inv, &a, grid, st, nullptr);
}

}  // namespace b300fft
