// rows_staged.cuh -- single-pass power-of-two rows kernel for the lengths
// whose transform fills an SM's register file (2^13, 2^14), with the input of
// the next transform copied into shared memory while the current one computes.
//
// The transform is the same register-staged Stockham FFT as k_rows_pow2
// (stockham_pow2.cuh; Sec. III-A's Cooley-Tukey split into radix-16 passes
// and one closing radix-2/4 pass) with 32 elements per thread (two radix-16
// butterflies per pass).  At these lengths one transform is 64 or 128 KiB of
// registers, so k_rows_pow2 runs one (2^14) or two (2^13) CTAs per SM and
// every CTA waits for its own DRAM loads before it can start.  Here each CTA
// is persistent and owns a staging buffer of one whole transform: thread 0
// has the tensor memory accelerator bulk-copy row r + gridDim.x into it (one
// contiguous copy, mbarrier completion) as soon as the threads have read row
// r into registers, so the load of the next row runs under the passes and
// stores of the current one.
//
// What makes room for the staging buffer is a half-size exchange buffer.
// With two butterflies per thread (b = t and b = t + T, T = N/32 threads),
// every radix-16 pass whose output is exchanged (Ns = 1, 16, 256 <= T) sends
// the outputs of butterfly t to positions < N/2 and those of butterfly t + T
// to the same positions + N/2, and the next pass's gather reads
// x[t + iT], i < 16 from the first half and i >= 16 from the second.  So an
// exchange is done in two rounds through N/2 padded slots: scatter butterfly
// 0's outputs, gather elements 0..15, then butterfly 1's outputs and elements
// 16..31 -- four barriers instead of two, shared memory 1.5 transforms
// instead of 2.06.
//
// The wait for a staged row is bounded (mbarrier polls); when it runs out the
// CTA records FFT_ERR_TIMEOUT in the plan's status word and stops.
//
// Measured per direction on 2^26 elements: 2^14 253 us against 275 us for
// k_rows_pow2 (the default there); 2^13 218 against 211 us (two plain CTAs per
// SM already overlap each other's loads), so 2^13 keeps the plain kernel.
#pragma once
#include "stockham_pow2.cuh"
#include "tma.cuh"

namespace b300fft {

template <int LOGN>
struct StagedCfg {
    using PL = P2Plan<LOGN, 32>;
    static_assert(PL::R == 32 && PL::NPASS >= 2, "two radix-16 butterflies per thread");
    static constexpr int N = PL::N;
    static constexpr int THREADS = PL::T;
    static constexpr int STAGE = N * 8;           // bytes of one staged row
    static constexpr int XHALF = padi(N / 2);     // float2 slots of the half exchange buffer
    static constexpr int SMEM = STAGE + XHALF * 8 + 16;
    static constexpr int MINB = (1024 / THREADS) / 2 > 0 ? (1024 / THREADS) / 2 : 1;  // 2^13: 2, 2^14: 1
};

// Contiguous bulk copy global -> shared with an L2 cache policy.
__device__ __forceinline__ void bulk_load_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                               uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// Outputs of butterfly QQ (registers v[QQ + 2r]) of radix-16 pass P into the
// half buffer, at the positions butterfly t would have in the full buffer.
template <class PL, int P, int QQ>
__device__ __forceinline__ void half_scatter(const float2 (&v)[PL::R], int t, float2* s) {
    constexpr int Ns = PL::ns(P);
    static_assert(PL::radix(P) == 16 && Ns <= PL::T, "half exchange needs Ns <= T");
    if constexpr (Ns % 16 == 0) {
        const int k = t & (Ns - 1);
        float2* p = s + padi((t - k) * 16 + k);
#pragma unroll
        for (int r = 0; r < 16; ++r) p[r * (Ns / 16) * 17] = v[QQ + 2 * r];
    } else {  // Ns == 1: positions 16t + r, padded 17t + r
        float2* p = s + 17 * t;
#pragma unroll
        for (int r = 0; r < 16; ++r) p[r] = v[QQ + 2 * r];
    }
}

// Elements t + iT, i < 16, of the current half.
template <class PL>
__device__ __forceinline__ void half_gather(float2 (&d)[16], int t, const float2* s) {
    static_assert(PL::T % 16 == 0, "gather stride must be a multiple of 16");
    const float2* p = s + padi(t);
#pragma unroll
    for (int i = 0; i < 16; ++i) d[i] = p[i * (PL::T / 16) * 17];
}

// Passes P .. NPASS-1 on v (x[t + iT] of the row) with half exchanges.
template <class PL, int P, bool INV>
__device__ __forceinline__ void staged_passes(float2 (&v)[PL::R], int t, float2* xb, const float2* __restrict__ tw,
                                              const TwPre<PL, P>* pre) {
    pass_compute<PL, P, INV>(v, t, tw, pre);
    if constexpr (P + 1 < PL::NPASS) {
        TwPre<PL, P + 1> next;
        half_scatter<PL, P, 0>(v, t, xb);
        tw_preload<PL, P + 1>(next, t, tw);  // in flight across the barriers
        __syncthreads();
        float2 lo[16];
        half_gather<PL>(lo, t, xb);
        __syncthreads();
        half_scatter<PL, P, 1>(v, t, xb);
        __syncthreads();
        float2 hi[16];
        half_gather<PL>(hi, t, xb);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            v[i] = lo[i];
            v[16 + i] = hi[i];
        }
        if constexpr (P + 2 < PL::NPASS) __syncthreads();  // before the next exchange rewrites the buffer
        staged_passes<PL, P + 1, INV>(v, t, xb, tw, TwPre<PL, P + 1>::ON ? &next : nullptr);
    }
}

template <int LOGN, bool INV>
__global__ void __launch_bounds__(StagedCfg<LOGN>::THREADS, StagedCfg<LOGN>::MINB)
k_rows_staged(const float2* __restrict__ in, float2* __restrict__ out, int64_t nrows, const float2* __restrict__ tw,
              int* status, int64_t polls) {
    using CF = StagedCfg<LOGN>;
    using PL = typename CF::PL;
    constexpr int N = CF::N, T = PL::T;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* const stage = reinterpret_cast<float2*>(smem_raw);
    float2* const xb = reinterpret_cast<float2*>(smem_raw + CF::STAGE);
    uint64_t* const bar = reinterpret_cast<uint64_t*>(smem_raw + CF::STAGE + CF::XHALF * 8);
    const int t = threadIdx.x;
    int64_t row = blockIdx.x;
    if (t == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const uint64_t pol = l2_policy_evict_first();
    if (t == 0 && row < nrows) {
        mbar_arrive_expect_tx(bar, CF::STAGE);
        bulk_load_hint(stage, in + row * N, CF::STAGE, bar, pol);
    }
    uint32_t phase = 0;
    for (; row < nrows; row += gridDim.x) {
        const bool got = mbar_wait(bar, phase, polls);
        phase ^= 1u;
        float2 v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = stage[t + i * T];
        fence_proxy_async_smem();  // these reads before the next copy into the buffer
        if (!tile_and<T>(got)) {   // all threads read a complete row, or all stop
            if (t == 0) {
                atomicCAS(status, 0, 6);
                mbar_wait(bar, phase ^ 1u, polls);  // the late copy, if it still lands
            }
            return;
        }
        const int64_t nxt = row + gridDim.x;
        if (t == 0 && nxt < nrows) {
            mbar_arrive_expect_tx(bar, CF::STAGE);
            bulk_load_hint(stage, in + nxt * N, CF::STAGE, bar, pol);
        }
        staged_passes<PL, 0, INV>(v, t, xb, tw, nullptr);
        float2* dst = out + row * N + t;
#pragma unroll
        for (int i = 0; i < 32; ++i) st_stream(dst + i * T, v[i]);
        __syncthreads();  // the last gathers are done before the next row's first scatter
    }
}

}  // namespace b300fft
