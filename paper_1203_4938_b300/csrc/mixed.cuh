// mixed.cuh -- batched transforms of mixed-radix lengths L = M * 2^K <= 4096
// (M = 3, 5, 7; M = 1, a power of two, serves the stage-graph executor's
// single-tile lines) with every radix, stride and index known at compile time:
// the Cooley-Tukey split of Sec. III-A applied to the factors 16, ..., 16,
// 2^(K mod 4), M in turn, in self-sorting Stockham order.
//
// One CTA of 256 threads transforms NL lines of one tile.  Pass p (radix R,
// Ns = product of the earlier radices, S = L / R butterflies per line) gives
// butterfly bf = threadIdx.x + 256 j of the tile to this thread.  A thread
// holds the R inputs of all its butterflies in registers, so one shared
// buffer serves every pass: gather, twiddle + butterfly, barrier, scatter,
// barrier.  The first pass gathers straight from global memory and the last
// stores there in natural order, through a layout policy:
//   MixRows  lines are contiguous rows (b fastest across threads);
//   MixCols  lines are adjacent columns of a row-major [L][S2] array (line
//            fastest across threads), stored with the four-step twiddle
//            W_N^{(col0 + line) e} -- the first pass of a four-step.
// (the stage-graph executor adds rows with per-line offsets and rows with
// the four-step's transposed store).  Middle passes map b fastest (shared
// memory only).
//
// Butterfly b of pass p (k = b mod Ns) reads element b + r S of its line,
// multiplies input r by W_{Ns R}^{k r} and writes output r to
// (b - k) R + k + r Ns -- the radix-2 recursion of Sec. III-A generalised to
// radix R, so after the last pass element k of the line is X[k].
#pragma once
#include "butterfly.cuh"
#include "stockham_pow2.cuh"

// CTAs per SM the kernels are compiled for: at 4 (64 registers) no shape
// spills, and against 3 (80 registers) they measured 4-8 % faster.
#ifndef B300_MIX_MINB
#define B300_MIX_MINB 4
#endif

namespace b300fft {

template <int M, int K, int NL_ = 4096 / (M << K)>
struct MixPlan {
    static_assert(M == 3 || M == 5 || M == 7 || (M == 1 && K >= 1), "odd factor 3, 5 or 7 (1: a power of two)");
    static constexpr int L = M << K;
    static_assert(L <= 4096, "one tile per line");
    static constexpr int NP16 = K / 4, REM = K % 4;
    static constexpr int NPASS = NP16 + (REM ? 1 : 0) + (M > 1 ? 1 : 0);
    __host__ __device__ static constexpr int radix(int p) {
        return p < NP16 ? 16 : ((REM && p == NP16) ? (1 << REM) : M);
    }
    __host__ __device__ static constexpr int ns(int p) {
        int s = 1;
        for (int i = 0; i < p; ++i) s *= radix(i);
        return s;
    }
    // pass p's table: entry (r - 1) * Ns + k = W_{Ns R}^{k r}, passes 1.. in order
    __host__ __device__ static constexpr int twoff(int p) {
        int o = 0;
        for (int i = 1; i < p; ++i) o += (radix(i) - 1) * ns(i);
        return o;
    }
    static constexpr int TWSIZE = twoff(NPASS);
    static constexpr int THREADS = 256;
    static constexpr int NL = NL_;                // lines per CTA
    static_assert(NL >= 1 && NL * L <= 4096, "tile of at most 4096 elements");
    static constexpr int LP = (L + (L >> 4)) | 1;  // odd line pitch (> padi(L - 1)): line-fast access conflict free
    static constexpr int SMEM = NPASS > 1 ? NL * LP * 8 : 0;
    static_assert(SMEM <= 48 * 1024, "static shared-memory limit");
};

// Twiddles of one radix-R butterfly: v[r] *= W^{k r}, tp = table + k.
template <int R, bool INV>
__device__ __forceinline__ void mix_twiddle(float2* v, const float2* __restrict__ tp, int Ns) {
    if constexpr (R == 16) {
        // six loads; the other nine are one product of two loaded values
        float2 w[16];
        w[1] = __ldg(tp);
        w[2] = __ldg(tp + Ns);
        w[3] = __ldg(tp + 2 * Ns);
        w[4] = __ldg(tp + 3 * Ns);
        w[8] = __ldg(tp + 7 * Ns);
        w[12] = __ldg(tp + 11 * Ns);
#pragma unroll
        for (int h = 4; h <= 12; h += 4)
#pragma unroll
            for (int l = 1; l <= 3; ++l) w[h + l] = cmul(w[h], w[l]);
#pragma unroll
        for (int r = 1; r < 16; ++r) v[r] = twmul<INV>(v[r], w[r]);
    } else if constexpr (R == 8) {
        float2 w[8];
        w[1] = __ldg(tp);
        w[2] = __ldg(tp + Ns);
        w[4] = __ldg(tp + 3 * Ns);
        w[3] = cmul(w[1], w[2]);
        w[5] = cmul(w[1], w[4]);
        w[6] = cmul(w[2], w[4]);
        w[7] = cmul(w[3], w[4]);
#pragma unroll
        for (int r = 1; r < 8; ++r) v[r] = twmul<INV>(v[r], w[r]);
    } else {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = twmul<INV>(v[r], __ldg(tp + (r - 1) * Ns));
    }
}

// Contiguous rows: line l, element e at base + l L + e.
template <int L>
struct MixRows {
    static constexpr bool LOAD_LF = false, STORE_LF = false;
    const float2* in;
    float2* out;
    __device__ __forceinline__ float2 load(int line, int e) const { return __ldcs(in + line * L + e); }
    __device__ __forceinline__ void store(int line, int e, float2 v) const { __stcs(out + line * L + e, v); }
};

// Adjacent columns of a row-major [L][S2] array (in / out at the tile's first
// column col0).  TW: stored values times W_N^{(col0 + line) e} from the
// two-level table W(m) = hi[m >> sh] * lo[m mod 2^sh] (four-step first pass,
// into the workspace); otherwise plain final stores (2-D column pass).
template <bool INV, bool TW = true>
struct MixCols {
    static constexpr bool LOAD_LF = true, STORE_LF = true;
    const float2* in;
    float2* out;
    int64_t S2;
    uint32_t col0;
    const float2* lo;
    const float2* hi;
    int sh;
    __device__ __forceinline__ float2 load(int line, int e) const { return __ldcs(in + e * S2 + line); }
    __device__ __forceinline__ void store(int line, int e, float2 v) const {
        if constexpr (TW) {
            v = twmul<INV>(v, root2(lo, hi, (col0 + (uint32_t)line) * (uint32_t)e, sh));
            __stcg(out + e * S2 + line, v);
        } else {
            __stcs(out + e * S2 + line, v);
        }
    }
};

// Pass P and every later pass of one tile (nl valid lines; io addresses the
// tile's first line).
template <class MP, int P, bool INV, class IO>
__device__ __forceinline__ void mix_pass(const IO& io, float2* s, int nl, const float2* __restrict__ tw) {
    constexpr int R = MP::radix(P), Ns = MP::ns(P), L = MP::L, S = L / R, NB = MP::NL * S;
    constexpr int T = MP::THREADS, J = (NB + T - 1) / T;
    constexpr bool FIRST = P == 0, LAST = P + 1 == MP::NPASS;
    // line index fastest across threads in the first pass (IO::LOAD_LF) or the
    // last one (IO::STORE_LF); a single pass needs one mapping for both
    static_assert(MP::NPASS > 1 || IO::LOAD_LF == IO::STORE_LF, "one-pass tiles load and store alike");
    constexpr bool LF = (FIRST && IO::LOAD_LF) || (LAST && IO::STORE_LF);
    float2 v[J * R];
    int line[J], b[J];
    bool in_tile[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int bf = threadIdx.x + j * T;
        if constexpr (LF) {
            b[j] = bf / MP::NL;
            line[j] = bf - b[j] * MP::NL;
        } else {
            line[j] = bf / S;
            b[j] = bf - line[j] * S;
        }
        in_tile[j] = NB % T == 0 || j + 1 < J || bf < NB;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 x = make_float2(0.f, 0.f);
            if constexpr (FIRST) {
                if (in_tile[j] && line[j] < nl) x = io.load(line[j], b[j] + r * S);
            } else {
                if (in_tile[j]) x = s[line[j] * MP::LP + padi(b[j] + r * S)];
            }
            v[j * R + r] = x;
        }
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        if constexpr (P > 0) mix_twiddle<R, INV>(v + j * R, tw + MP::twoff(P) + (b[j] & (Ns - 1)), Ns);
        dft<R, 0, 1, INV>(v + j * R);
    }
    if constexpr (LAST) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
            if (in_tile[j] && line[j] < nl) {
#pragma unroll
                for (int r = 0; r < R; ++r) io.store(line[j], b[j] + r * S, v[j * R + r]);
            }
        }
    } else {
        if constexpr (!FIRST) __syncthreads();  // every thread has gathered this pass's inputs
#pragma unroll
        for (int j = 0; j < J; ++j) {
            if (in_tile[j]) {
                const int k = b[j] & (Ns - 1);
                float2* d = s + line[j] * MP::LP;
                const int base = (b[j] - k) * R + k;
#pragma unroll
                for (int r = 0; r < R; ++r) d[padi(base + r * Ns)] = v[j * R + r];
            }
        }
        __syncthreads();
        mix_pass<MP, P + 1, INV>(io, s, nl, tw);
    }
}

// nrows lines of L = M * 2^K elements, [nrows][L] at in / out (out == in allowed:
// a tile reads all its lines before its first store).
template <int M, int K, bool INV>
__global__ void __launch_bounds__(256, B300_MIX_MINB) k_rows_mixed(const float2* __restrict__ in, float2* __restrict__ out,
                                                       int64_t nrows, const float2* __restrict__ tw) {
    using MP = MixPlan<M, K>;
    __shared__ float2 smem[MP::SMEM > 0 ? MP::SMEM / 8 : 1];
    const int64_t row0 = (int64_t)blockIdx.x * MP::NL;
    const int64_t left = nrows - row0;
    const int nl = left < MP::NL ? (int)left : MP::NL;
    const MixRows<MP::L> io{in + row0 * MP::L, out + row0 * MP::L};
    mix_pass<MP, 0, INV>(io, smem, nl, tw);
}

// Column transforms of length L = M * 2^K over `items` row-major [L][S2]
// arrays, NL adjacent columns per CTA (S2 % NL == 0), into `out` (same layout;
// out == in allowed: a tile reads its columns before its first store).  TW:
// the four-step first pass of N = L * S2, times W_N^{n2 k1}; otherwise the
// column pass of a 2-D transform.
template <int M, int K, int NL, bool INV, bool TW = true>
__global__ void __launch_bounds__(256, B300_MIX_MINB) k_cols_mixed(const float2* __restrict__ in, float2* __restrict__ out,
                                                       int64_t S2, int64_t items, const float2* __restrict__ tw,
                                                       const float2* __restrict__ lo, const float2* __restrict__ hi,
                                                       int sh) {
    using MP = MixPlan<M, K, NL>;
    __shared__ float2 smem[MP::SMEM > 0 ? MP::SMEM / 8 : 1];
    const int64_t tiles_per_item = S2 / NL;
    const int64_t item = (int64_t)blockIdx.x / tiles_per_item;
    const int64_t col0 = ((int64_t)blockIdx.x - item * tiles_per_item) * NL;
    const int64_t base = item * MP::L * S2 + col0;
    const MixCols<INV, TW> io{in + base, out + base, S2, (uint32_t)col0, lo, hi, sh};
    mix_pass<MP, 0, INV>(io, smem, NL, tw);
}

}  // namespace b300fft
