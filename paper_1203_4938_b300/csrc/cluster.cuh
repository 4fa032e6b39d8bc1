// cluster.cuh -- single-pass transforms of N = K * M points on a thread-block
// cluster of K CTAs that exchange data through distributed shared memory
// (one HBM round trip, no workspace).
//
// Decimation in time with N = K * M (Sec. III-A, Cooley-Tukey; n = r + K*m):
//     F_r[j]      = sum_m x[r + K m] W_M^{m j}                (CTA r, M points)
//     X[q*M + j]  = sum_r W_K^{r q} (W_N^{r j} F_r[j])        (K points per j)
// Steps of CTA c (rank in the cluster) for one transform:
//   1. load x[c*M .. c*M + M) (each thread 16 consecutive elements, 16-byte
//      loads) and store element c*M + e into CTA e mod K's buffer at
//      c*(M/K) + e div K (so CTA r receives its decimated sequence
//      x[r + K m], m < M);
//   2. cluster barrier; the M-point Stockham transform of the buffer
//      (register-staged radix-16 passes, the buffer doubles as the padded
//      exchange area); multiply by W_N^{c j};
//   3. cluster barrier (every CTA is done with its buffer); element j goes to
//      CTA j / S (S = M/K) at [c][j mod S]; cluster barrier;
//   4. K-point DFTs over the K received rows for each of the CTA's S bins j,
//      X[q*M + c*S + j'] -- K contiguous runs of S elements per CTA.
// All CTAs of a cluster run the same code path (one transform per cluster,
// no early exit), so every cluster barrier is reached by all of them; the
// last remote access precedes the last barrier, so no CTA exits while a peer
// can still touch its shared memory.
#pragma once
#include "stockham_pow2.cuh"

namespace b300fft {

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// shared::cluster address of `p` (a shared::cta pointer) in CTA `rank`
__device__ __forceinline__ uint32_t cluster_map(const void* p, uint32_t rank) {
    uint32_t a = (uint32_t)__cvta_generic_to_shared(p), d;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(rank));
    return d;
}
__device__ __forceinline__ void st_cluster(uint32_t addr, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void st_cluster2(uint32_t addr, float2 a, float2 b) {  // 16-byte aligned addr
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a.x), "f"(a.y), "f"(b.x),
                 "f"(b.y)
                 : "memory");
}

template <int LM, int K>
struct ClusterCfg {
    using PL = P2Plan<LM>;
    static constexpr int M = PL::N, T = PL::T, S = M / K;
    static constexpr int THREADS = T;
    static_assert(PL::R == 16 && PL::NPASS >= 2, "M >= 256");
    static_assert(K == 8 || K == 16, "cluster of 8 or 16 CTAs");
    static_assert(S % T == 0, "each thread owns S / T bins of the last step");
    static constexpr int BUF = PL::PADDED;  // float2: dense input / padded exchange / received rows
    static constexpr int SMEM = (BUF + PL::R) * 8;
};

template <int LM, int K, bool INV>
__global__ void __launch_bounds__(ClusterCfg<LM, K>::THREADS, 1024 / ClusterCfg<LM, K>::THREADS)
k_cluster_fft(const float2* __restrict__ in, float2* __restrict__ out, const float2* __restrict__ tw,
              const float2* __restrict__ lo, const float2* __restrict__ hi, int sh) {
    using CF = ClusterCfg<LM, K>;
    using PL = typename CF::PL;
    constexpr int M = CF::M, T = CF::T, S = CF::S;
    constexpr int64_t N = (int64_t)K * M;
    extern __shared__ __align__(16) float2 smem[];
    float2* buf = smem;
    float2* steps = smem + CF::BUF;  // W_N^{c T i}, i < 16
    const int t = threadIdx.x;
    const uint32_t c = cluster_rank();
    const int64_t tr = blockIdx.x / K;
    const float2* x = in + tr * N + (int64_t)c * M;
    float2* y = out + tr * N;

    // 1. contiguous load (elements 16 t .. 16 t + 15 of the chunk); element
    //    e = 16 t + g K + r goes to CTA r at c S + 16 t / K + g
    float2 e[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(x + (int64_t)t * 16) + j);
        e[2 * j] = make_float2(v.x, v.y);
        e[2 * j + 1] = make_float2(v.z, v.w);
    }
    for (int i = t; i < PL::R; i += T) steps[i] = root2(lo, hi, c * (uint32_t)(T * i), sh);
    cluster_barrier();  // every CTA of the cluster runs and may receive
#pragma unroll
    for (int r = 0; r < K; ++r) {
        if constexpr (K == 16) st_cluster(cluster_map(buf + c * S + t, r), e[r]);
        else st_cluster2(cluster_map(buf + c * S + 2 * t, r), e[r], e[8 + r]);
    }
    cluster_barrier();  // the decimated sequence x[c + K m] is complete in buf

    // 2. M-point transform of buf, then the twiddle W_N^{c j}, j = t + T i
    float2 v[PL::R];
#pragma unroll
    for (int i = 0; i < PL::R; ++i) v[i] = buf[t + i * T];
    __syncthreads();  // buf becomes the exchange area
    run_passes<PL, 0, INV, false, 1>(v, t, buf, 0, tw);
    {
        const float2 w0 = root2(lo, hi, c * (uint32_t)t, sh);
#pragma unroll
        for (int i = 0; i < PL::R; ++i) v[i] = twmul<INV>(v[i], cmul(w0, steps[i]));
    }
    cluster_barrier();  // every CTA is done with its buffer
    // 3. bin j = t + T i goes to CTA j / S, row c, column j mod S
#pragma unroll
    for (int i = 0; i < PL::R; ++i)  // t + (i T) % S < S since T divides S
        st_cluster(cluster_map(buf + c * S + t + (i * T) % S, (uint32_t)((i * T) / S)), v[i]);
    cluster_barrier();  // all rows received; no remote access after this point

    // 4. K-point DFTs over the rows for the S bins of this CTA
#pragma unroll
    for (int q = 0; q < S / T; ++q) {
        const int jj = t + q * T;
        float2 u[K];
#pragma unroll
        for (int r = 0; r < K; ++r) u[r] = buf[r * S + jj];
        if constexpr (K == 8) dft8<0, 1, INV>(u);
        else dft16<0, 1, INV>(u);
#pragma unroll
        for (int r = 0; r < K; ++r) __stcs(y + (int64_t)r * M + c * S + jj, u[r]);
    }
}

}  // namespace b300fft
