// k_cluster.cu -- instantiations and launcher of the thread-block-cluster
// single-pass transforms (cluster.cuh): N = K * 2^LM on K CTAs.
#include "cluster.cuh"
#include "launch.h"

namespace b300fft {

#define B300_CLUSTER_CONFIGS(X) X(12, 8) X(12, 16) X(13, 8) X(13, 16) X(14, 8)

namespace {
template <int LM, int K, bool INV>
cudaError_t setup_one(int* clusters) {
    using CF = ClusterCfg<LM, K>;
    auto f = k_cluster_fft<LM, K, INV>;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM);
    if (e == cudaSuccess && K > 8) e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess || !clusters) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = K;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(K);
    cfg.blockDim = dim3(CF::THREADS);
    cfg.dynamicSmemBytes = CF::SMEM;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(clusters, f, &cfg);
}

template <int LM, int K>
cudaError_t one(int op, bool inv, const float2* in, float2* out, int64_t batch, const float2* tw, const float2* lo,
                const float2* hi, int sh, cudaStream_t st, int* clusters) {
    using CF = ClusterCfg<LM, K>;
    if (op == 0) {
        cudaError_t e = setup_one<LM, K, false>(clusters);
        if (e == cudaSuccess) e = setup_one<LM, K, true>(nullptr);
        return e;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = K;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(K * batch));
    cfg.blockDim = dim3(CF::THREADS);
    cfg.dynamicSmemBytes = CF::SMEM;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (inv) return cudaLaunchKernelEx(&cfg, k_cluster_fft<LM, K, true>, in, out, tw, lo, hi, sh);
    return cudaLaunchKernelEx(&cfg, k_cluster_fft<LM, K, false>, in, out, tw, lo, hi, sh);
}

cudaError_t dispatch(int lm, int k, int op, bool inv, const float2* in, float2* out, int64_t batch, const float2* tw,
                     const float2* lo, const float2* hi, int sh, cudaStream_t st, int* clusters) {
#define B300_X(LM, K) \
    if (lm == LM && k == K) return one<LM, K>(op, inv, in, out, batch, tw, lo, hi, sh, st, clusters);
    B300_CLUSTER_CONFIGS(B300_X)
#undef B300_X
    return cudaErrorInvalidValue;
}
}  // namespace

bool cluster_config_available(int lm, int k) {
#define B300_X(LM, K) \
    if (lm == LM && k == K) return true;
    B300_CLUSTER_CONFIGS(B300_X)
#undef B300_X
    return false;
}

cudaError_t cluster_prepare(int lm, int k, int* max_clusters) {
    return dispatch(lm, k, 0, false, nullptr, nullptr, 0, nullptr, nullptr, nullptr, 0, 0, max_clusters);
}

cudaError_t launch_cluster_fft(int lm, int k, bool inv, const float2* in, float2* out, int64_t batch,
                               const float2* tw, const float2* lo, const float2* hi, int sh, cudaStream_t st) {
    return dispatch(lm, k, 1, inv, in, out, batch, tw, lo, hi, sh, st, nullptr);
}

}  // namespace b300fft
