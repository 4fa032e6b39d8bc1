// k_three_pipe.cu -- instantiations and launcher of the three-stage
// persistent kernel with asynchronous tile loads (pipe3.cuh), and its three
// tensor maps: the input for stage A and two views of the workspace for the
// B1 and B2 stages.
#include "launch.h"
#include "pipe3.cuh"

namespace b300fft {

#define B300_THREE_PIPE_CONFIGS(X) X(6, 6, 7) X(6, 7, 7) X(7, 7, 7) X(7, 7, 8) X(8, 7, 8) X(7, 8, 8) X(8, 8, 8)

namespace {
template <int LA, int LB1, int LB2, int NS>
cudaError_t one(int op, bool inv, const ThreeArgs* a, int grid, cudaStream_t st, PersistInfo* info) {
    using PC = Three3Cfg<LA, LB1, LB2, NS>;
    using CF = ThreeCfg<LA, LB1, LB2>;
    auto kf = k_threestep_pipe<LA, LB1, LB2, NS, false>;
    auto ki = k_threestep_pipe<LA, LB1, LB2, NS, true>;
    if (op == 0) {
        if (!tensor_maps_available()) return cudaErrorNotSupported;
        cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, PC::SMEM);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(ki, cudaFuncAttributeMaxDynamicSharedMemorySize, PC::SMEM);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kf, PC::CTA_THREADS, PC::SMEM);
        if (e != cudaSuccess) return e;
        info->threads = PC::CTA_THREADS;
        info->smem = PC::SMEM;
        info->blocks_per_sm = nb;
        return cudaSuccess;
    }
    constexpr uint64_t N1 = CF::N1, M1 = CF::M1, M2 = CF::M2, N2 = CF::N2;
    const uint64_t B = (uint64_t)a->batch;
    CUtensorMap t_in, t_b1, t_b2;
    {  // input as [B * N1][N2]; stage-A box: CA columns x N1 rows
        const uint64_t dims[2] = {N2, B * N1}, str[1] = {N2 * 8};
        const uint32_t box[2] = {(uint32_t)CF::CA, (uint32_t)N1};
        if (!encode_tensor_map(&t_in, a->in, 2, dims, str, box)) return cudaErrorInvalidValue;
    }
    {  // workspace as [B * N1 * M1][M2]; B1 box: CB columns x M1 rows of one row k1
        const uint64_t dims[2] = {M2, B * N1 * M1}, str[1] = {M2 * 8};
        const uint32_t box[2] = {(uint32_t)CF::CB, (uint32_t)M1};
        if (!encode_tensor_map(&t_b1, a->work, 2, dims, str, box)) return cudaErrorInvalidValue;
    }
    {  // workspace as [B * N1][M1][M2]; B2 box: M2 points of TPC rows k1 at one j1
        const uint64_t dims[3] = {M2, M1, B * N1}, str[2] = {M2 * 8, N2 * 8};
        const uint32_t box[3] = {(uint32_t)M2, 1u, (uint32_t)CF::TPC};
        if (!encode_tensor_map(&t_b2, a->work, 3, dims, str, box)) return cudaErrorInvalidValue;
    }
    if (inv) ki<<<grid, PC::CTA_THREADS, PC::SMEM, st>>>(t_in, t_b1, t_b2, *a);
    else kf<<<grid, PC::CTA_THREADS, PC::SMEM, st>>>(t_in, t_b1, t_b2, *a);
    return cudaGetLastError();
}

cudaError_t dispatch(const ThreeConfig& c, int ns, int op, bool inv, const ThreeArgs* a, int grid, cudaStream_t st,
                     PersistInfo* info) {
#define B300_X(LA, LB1, LB2)                                                              \
    if (c.la == LA && c.lb1 == LB1 && c.lb2 == LB2) {                                     \
        if (ns == 2) return one<LA, LB1, LB2, 2>(op, inv, a, grid, st, info);             \
        if (ns == 3) return one<LA, LB1, LB2, 3>(op, inv, a, grid, st, info);             \
    }
    B300_THREE_PIPE_CONFIGS(B300_X)
#undef B300_X
    return cudaErrorInvalidValue;
}
}  // namespace

bool three_pipe_available(const ThreeConfig& c, int ns) {
    if ((ns != 2 && ns != 3) || c.tile != 4096) return false;
#define B300_X(LA, LB1, LB2) \
    if (c.la == LA && c.lb1 == LB1 && c.lb2 == LB2) return true;
    B300_THREE_PIPE_CONFIGS(B300_X)
#undef B300_X
    return false;
}

cudaError_t three_pipe_prepare(const ThreeConfig& c, int ns, PersistInfo* info) {
    return dispatch(c, ns, 0, false, nullptr, 0, 0, info);
}

cudaError_t launch_threestep_pipe(const ThreeConfig& c, int ns, bool inv, const ThreeArgs& a, int grid,
                                  cudaStream_t st) {
    return dispatch(c, ns, 1, inv, &a, grid, st, nullptr);
}

}  // namespace b300fft
