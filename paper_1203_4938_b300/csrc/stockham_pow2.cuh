// stockham_pow2.cuh -- register-staged Stockham autosort FFT for N = 2^n.
//
// The transform is the DFT of the paper's Sec. III-A example, evaluated by
// Cooley-Tukey decimation: N = R_0 * R_1 * ... and every pass performs N/R_p
// radix-R_p butterflies (the paper's small "2^k DFT" node, here radix 16 with
// one closing radix 2/4/8 pass when log2 N is not a multiple of 4).
//
// Stockham pass p (Ns = R_0 * ... * R_{p-1}, L = Ns * R_p), butterfly b:
//     v[r]  = x[b + r * N/R_p]                     (stride-N/R_p gather)
//     v[r] *= W_L^{(b mod Ns) * r}                (skipped for p = 0)
//     v     = DFT_{R_p}(v)
//     y[(b div Ns) * L + (b mod Ns) + r * Ns] = v[r]
// The output of the last pass is in natural order (self-sorting, no bit
// reversal).  Thread t of a transform owns R = 16 registers holding
// x[t + i*T], i < R (T = N/R threads): every pass reads that same pattern, so
// the first pass gathers straight from global memory and the last pass
// scatters straight to it, both coalesced across t.  Between passes the
// exchange goes through shared memory padded by one float2 per 16 (bank
// conflict free for the radix-16 stride patterns used here).
//
// Twiddles come from a per-length table built once per plan in FP64 and
// rounded to FP32: for pass p >= 1 the block [(r-1)*Ns + k] = W_L^{k*r},
// r = 1..R_p-1, k < Ns, so consecutive butterflies read consecutive entries.
#pragma once
#include "butterfly.cuh"

namespace b300fft {

__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }

template <int LOGN>
struct P2Plan {
    static constexpr int N = 1 << LOGN;
    static constexpr int R = N >= 16 ? 16 : N;  // elements per thread
    static constexpr int T = N / R;             // threads per transform
    static constexpr int NP16 = N >= 16 ? LOGN / 4 : 0;
    static constexpr int REM = N >= 16 ? LOGN % 4 : 0;
    static constexpr int NPASS = N >= 16 ? NP16 + (REM ? 1 : 0) : 1;
    __host__ __device__ static constexpr int radix(int p) {
        return N < 16 ? N : (p < NP16 ? 16 : (1 << REM));
    }
    __host__ __device__ static constexpr int ns(int p) {
        int s = 1;
        for (int i = 0; i < p; ++i) s *= radix(i);
        return s;
    }
    __host__ __device__ static constexpr int twoff(int p) {
        int o = 0;
        for (int i = 1; i < p; ++i) o += (radix(i) - 1) * ns(i);
        return o;
    }
    static constexpr int TWSIZE = twoff(NPASS);
    static constexpr int PADDED = N + N / 16;  // float2 per transform in smem
};

__host__ __device__ __forceinline__ constexpr int padi(int a) { return a + (a >> 4); }

// Streaming (evict-first) global accesses for the data; tables use __ldg.
__device__ __forceinline__ float2 ld_stream(const float2* p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream(float2* p, float2 v) { __stcs(p, v); }

template <int R, int S, bool INV>
__device__ __forceinline__ void dft_at(float2* v) {
    dft<R, 0, S, INV>(v);
}

// Multiply the butterfly inputs of pass P by their twiddles and run the
// radix-R_P butterflies.  b0 = t (butterfly index of q = 0); butterfly q is
// b0 + q*T and owns v[q + Q*r].
template <class PL, int P, bool INV>
__device__ __forceinline__ void pass_compute(float2 (&v)[PL::R], int b0, const float2* __restrict__ tw) {
    constexpr int Rp = PL::radix(P), Q = PL::R / Rp, Ns = PL::ns(P);
    if constexpr (P > 0) {
        const float2* twp = tw + PL::twoff(P);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int k = (b0 + q * PL::T) & (Ns - 1);
#pragma unroll
            for (int r = 1; r < Rp; ++r) {
                const float2 w = __ldg(twp + (r - 1) * Ns + k);
                v[q + Q * r] = twmul<INV>(v[q + Q * r], w);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) dft_at<Rp, Q, INV>(v + q);
}

// Scatter the outputs of pass P into the exchange buffer (padded indices).
template <class PL, int P>
__device__ __forceinline__ void pass_scatter(const float2 (&v)[PL::R], int b0, float2* s, int cstride, int coff) {
    constexpr int Rp = PL::radix(P), Q = PL::R / Rp, Ns = PL::ns(P), L = Ns * Rp;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int b = b0 + q * PL::T;
        const int k = b & (Ns - 1);
        const int base = (b - k) * Rp + k;
#pragma unroll
        for (int r = 0; r < Rp; ++r) {
            const int a = (base + r * Ns) * cstride + coff;
            s[padi(a)] = v[q + Q * r];
        }
    }
    (void)L;
}

// Gather the pass inputs x[t + i*T] from the exchange buffer.
template <class PL>
__device__ __forceinline__ void pass_gather(float2 (&v)[PL::R], int t, const float2* s, int cstride, int coff) {
#pragma unroll
    for (int i = 0; i < PL::R; ++i) v[i] = s[padi((t + i * PL::T) * cstride + coff)];
}

// Barrier over the threads that share an exchange buffer.
template <bool WARP_ONLY>
__device__ __forceinline__ void xsync() {
    if constexpr (WARP_ONLY) __syncwarp();
    else __syncthreads();
}

// All passes from P on.  Data layout in the exchange buffer: element a of
// column c at index a*cstride + coff (rows kernel: cstride 1, coff 0).
template <class PL, int P, bool INV, bool WARP_ONLY>
__device__ __forceinline__ void run_passes(float2 (&v)[PL::R], int t, float2* s, int cstride, int coff,
                                           const float2* __restrict__ tw) {
    pass_compute<PL, P, INV>(v, t, tw);
    if constexpr (P + 1 < PL::NPASS) {
        pass_scatter<PL, P>(v, t, s, cstride, coff);
        xsync<WARP_ONLY>();
        pass_gather<PL>(v, t, s, cstride, coff);
        xsync<WARP_ONLY>();
        run_passes<PL, P + 1, INV, WARP_ONLY>(v, t, s, cstride, coff, tw);
    }
}

// ---------------------------------------------------------------------------
// Rows kernel: TPC contiguous transforms of length N per CTA ([batch][N]).
// TRANSPOSE_OUT (four-step second pass): the CTA's TPC rows are consecutive
// k1 of one item of N1*N elements and the result of row k1, bin k2 goes to
// out[item*N1*N + k1 + N1*k2]; it is staged in shared memory so that the
// global stores run TPC consecutive k1 at a time.
// ---------------------------------------------------------------------------
template <int LOGN, int TPC>
struct RowsCfg {
    using PL = P2Plan<LOGN>;
    static constexpr int THREADS = PL::T * TPC;
    static constexpr bool WARP_ONLY = (PL::T <= 32) && (32 % PL::T == 0) && false;
    // transposed staging: row pitch chosen so that TPC rows read at the same
    // column index fall in distinct banks (pitch = 16/TPC mod 16, in float2).
    static constexpr int PITCH_T = ((PL::PADDED + 15) / 16) * 16 + (TPC >= 16 ? 1 : 16 / TPC);
    static constexpr int SMEM_PLAIN = (PL::NPASS > 1 ? PL::PADDED * TPC : 0) * 8;
    static constexpr int SMEM_T = PITCH_T * TPC * 8;
};

template <int LOGN, int TPC, bool INV, bool TRANSPOSE_OUT>
__global__ void __launch_bounds__(RowsCfg<LOGN, TPC>::THREADS)
k_rows_pow2(const float2* __restrict__ in, float2* __restrict__ out, int64_t nrows,
            const float2* __restrict__ tw, int64_t n1) {
    using CF = RowsCfg<LOGN, TPC>;
    using PL = typename CF::PL;
    extern __shared__ float2 smem[];
    const int t = threadIdx.x & (PL::T - 1);
    const int sub = threadIdx.x / PL::T;
    const int64_t row0 = (int64_t)blockIdx.x * TPC;
    const int64_t row = row0 + sub;
    const bool ok = row < nrows;
    const float2* src = in + row * PL::N;
    float2 v[PL::R];
#pragma unroll
    for (int i = 0; i < PL::R; ++i) v[i] = ok ? ld_stream(src + t + i * PL::T) : make_float2(0.f, 0.f);

    constexpr int pitch = TRANSPOSE_OUT ? CF::PITCH_T : PL::PADDED;
    float2* s = smem + sub * pitch;
    run_passes<PL, 0, INV, CF::WARP_ONLY>(v, t, s, 1, 0, tw);

    if constexpr (!TRANSPOSE_OUT) {
        float2* dst = out + row * PL::N;
        if (ok) {
#pragma unroll
            for (int i = 0; i < PL::R; ++i) st_stream(dst + t + i * PL::T, v[i]);
        }
    } else {
        // last pass output is x[t + i*T] in natural order: stage it, then
        // store TPC consecutive k1 for each k2.
#pragma unroll
        for (int i = 0; i < PL::R; ++i) s[padi(t + i * PL::T)] = v[i];
        __syncthreads();
        const int64_t item = row0 / n1;
        const int64_t k10 = row0 - item * n1;
        float2* dst = out + item * n1 * PL::N + k10;
        constexpr int TOT = TPC * PL::N;
#pragma unroll 4
        for (int e = threadIdx.x; e < TOT; e += CF::THREADS) {
            const int c = e % TPC, k2 = e / TPC;
            if (row0 + c < nrows) st_stream(dst + c + n1 * (int64_t)k2, smem[c * pitch + padi(k2)]);
        }
    }
}

// ---------------------------------------------------------------------------
// Columns kernel: C adjacent columns of a row-major [len][S] array per CTA,
// each column a transform of length N = 2^LOGN with element stride S.
// Used for the 2-D column pass (S = W) and the four-step first pass (S = N2),
// where TWIDDLE_OUT multiplies element (k1, n2) by W_{N*S}^{n2*k1} from the
// two-level table W(m) = hi[m >> sh] * lo[m & (2^sh - 1)].
// Thread (c, t): c = threadIdx.x % C is the column (fastest, so each warp
// touches C*8 contiguous bytes per row), t the Stockham thread index.
// ---------------------------------------------------------------------------
template <int LOGN, int C>
struct ColsCfg {
    using PL = P2Plan<LOGN>;
    static constexpr int THREADS = PL::T * C;
    static constexpr int SMEM = (PL::NPASS > 1 ? padi(PL::N * C) : 0) * 8;
};

template <int LOGN, int C, bool INV, bool TWIDDLE_OUT>
__global__ void __launch_bounds__(ColsCfg<LOGN, C>::THREADS)
k_cols_pow2(const float2* __restrict__ in, float2* __restrict__ out, int64_t S, int64_t ngroups_per_item,
            int64_t item_stride, int64_t nitems, const float2* __restrict__ tw,
            const float2* __restrict__ tw_lo, const float2* __restrict__ tw_hi, int sh) {
    using CF = ColsCfg<LOGN, C>;
    using PL = typename CF::PL;
    extern __shared__ float2 smem[];
    const int c = threadIdx.x % C;
    const int t = threadIdx.x / C;
    const int64_t item = blockIdx.x / ngroups_per_item;
    const int64_t g = blockIdx.x - item * ngroups_per_item;
    if (item >= nitems) return;  // uniform per CTA
    const int64_t col = g * C + c;
    const float2* src = in + item * item_stride + col;
    float2 v[PL::R];
#pragma unroll
    for (int i = 0; i < PL::R; ++i) v[i] = ld_stream(src + (int64_t)(t + i * PL::T) * S);

    run_passes<PL, 0, INV, false>(v, t, smem, C, c, tw);

    if constexpr (TWIDDLE_OUT) {
        const uint32_t mask = (1u << sh) - 1u;
#pragma unroll
        for (int i = 0; i < PL::R; ++i) {
            const uint32_t m = (uint32_t)col * (uint32_t)(t + i * PL::T);
            const float2 w = cmul(__ldg(tw_hi + (m >> sh)), __ldg(tw_lo + (m & mask)));
            v[i] = twmul<INV>(v[i], w);
        }
    }
    float2* dst = out + item * item_stride + col;
#pragma unroll
    for (int i = 0; i < PL::R; ++i) st_stream(dst + (int64_t)(t + i * PL::T) * S, v[i]);
}

}  // namespace b300fft
