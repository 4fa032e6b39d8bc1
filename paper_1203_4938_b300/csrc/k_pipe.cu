// k_pipe.cu -- instantiations and launcher of the persistent four-step with
// asynchronous tile loads (pipe.cuh), and the tensor-map encoding its
// first-pass copies read the input through.
#include <cuda.h>

#include <mutex>

#include "launch.h"
#include "pipe.cuh"

namespace b300fft {

// (L1, C, L2, TPC): N = 2^L1 * 2^L2, first-pass tiles of C columns, second-pass
// tiles of TPC rows; every shape here moves 4096 or 8192 points per tile.
#define B300_PIPE_CONFIGS(X)                                                                                  \
    X(7, 32, 8, 16) X(8, 16, 7, 32) X(8, 16, 8, 16) X(8, 16, 9, 8) X(9, 8, 9, 8) X(8, 16, 10, 4) X(9, 8, 10, 4) \
        X(10, 4, 10, 4) X(9, 16, 10, 8) X(10, 8, 10, 8)

namespace {

template <int L1, int C, int L2, int TPC, int NS>
cudaError_t one(int op, bool inv, const PersistArgs* a, int grid, cudaStream_t st, PersistInfo* info) {
    using CF = PipeCfg<L1, C, L2, TPC, NS>;
    auto kf = k_fourstep_pipe<L1, C, L2, TPC, NS, false>;
    auto ki = k_fourstep_pipe<L1, C, L2, TPC, NS, true>;
    if (op == 0) {  // prepare
        if (!tensor_maps_available()) return cudaErrorNotSupported;
        cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(ki, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kf, CF::CTA_THREADS, CF::SMEM);
        if (e != cudaSuccess) return e;
        info->threads = CF::CTA_THREADS;
        info->smem = CF::SMEM;
        info->blocks_per_sm = nb;
        return cudaSuccess;
    }
    // the input viewed as [batch * N1 rows][N2 columns] of 8-byte elements;
    // a first-pass tile is C columns x N1 rows (boxes of at most 256 rows)
    constexpr int64_t N1 = int64_t(1) << L1, N2 = int64_t(1) << L2;
    CUtensorMap tm;
    const uint64_t dims[2] = {(uint64_t)N2, (uint64_t)(a->batch * N1)};
    const uint64_t strides[1] = {(uint64_t)(N2 * 8)};
    const uint32_t box[2] = {(uint32_t)C, (uint32_t)CF::BOX_ROWS};
    if (!encode_tensor_map(&tm, a->in, 2, dims, strides, box)) return cudaErrorInvalidValue;
    if (inv) ki<<<grid, CF::CTA_THREADS, CF::SMEM, st>>>(tm, *a);
    else kf<<<grid, CF::CTA_THREADS, CF::SMEM, st>>>(tm, *a);
    return cudaGetLastError();
}

cudaError_t dispatch(const PersistConfig& c, int ns, int op, bool inv, const PersistArgs* a, int grid,
                     cudaStream_t st, PersistInfo* info) {
#define B300_X(L1, C, L2, TPC)                                                         \
    if (c.l1 == L1 && c.c == C && c.l2 == L2 && c.tpc == TPC) {                        \
        if (ns == 2) return one<L1, C, L2, TPC, 2>(op, inv, a, grid, st, info);        \
        if (ns == 3) return one<L1, C, L2, TPC, 3>(op, inv, a, grid, st, info);        \
    }
    B300_PIPE_CONFIGS(B300_X)
#undef B300_X
    return cudaErrorInvalidValue;
}

}  // namespace

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (the
// library does not link the driver API).
EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}
}  // namespace

bool tensor_maps_available() { return encode_fn() != nullptr; }

bool encode_tensor_map(CUtensorMap* tm, const void* base, int rank, const uint64_t* dims,
                       const uint64_t* strides_bytes, const uint32_t* box) {
    EncodeTiled fn = encode_fn();
    if (!fn || rank < 1 || rank > 5) return false;
    cuuint64_t d[5], st[4];
    cuuint32_t b[5], e[5];
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        b[i] = box[i];
        e[i] = 1;
        if (i + 1 < rank) st[i] = strides_bytes[i];
    }
    return fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, (cuuint32_t)rank, const_cast<void*>(base), d, st, b, e,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool pipe_config_available(const PersistConfig& c, int ns) {
    if (ns != 2 && ns != 3) return false;
#define B300_X(L1, C, L2, TPC) \
    if (c.l1 == L1 && c.c == C && c.l2 == L2 && c.tpc == TPC) return true;
    B300_PIPE_CONFIGS(B300_X)
#undef B300_X
    return false;
}

cudaError_t pipe_prepare(const PersistConfig& c, int ns, PersistInfo* info) {
    return dispatch(c, ns, 0, false, nullptr, 0, 0, info);
}

cudaError_t launch_fourstep_pipe(const PersistConfig& c, int ns, bool inv, const PersistArgs& a, int grid,
                                 cudaStream_t st) {
    return dispatch(c, ns, 1, inv, &a, grid, st, nullptr);
}

}  // namespace b300fft
