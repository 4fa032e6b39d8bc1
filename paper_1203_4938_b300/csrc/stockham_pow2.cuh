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

// RT: elements per thread (16, or 32 = two radix-16 butterflies per pass).
template <int LOGN, int RT = 16>
struct P2Plan {
    static constexpr int N = 1 << LOGN;
    static constexpr int R = N >= RT ? RT : (N >= 16 ? 16 : N);  // elements per thread
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

// Radix-16 passes read 6 of their 15 twiddles and form the rest by one
// complex product (fewer load/store-unit instructions, more FMA work).
#ifndef B300_TW_LOADS6
#define B300_TW_LOADS6 1
#endif
constexpr bool kTwiddleLoads6 = B300_TW_LOADS6 != 0;

// Streaming (evict-first) global accesses for the data; tables use __ldg.
__device__ __forceinline__ float2 ld_stream(const float2* p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream(float2* p, float2 v) { __stcs(p, v); }

// Data-access flavours of the tile functions.
//   Ld::Stream  evict-first load (input read once)
//   Ld::Cg      L2-only load (workspace written earlier in the same launch)
//   St::Stream  evict-first store (final output)
//   St::Keep    store with an L2 evict-last policy (workspace read back soon)
enum class Ld { Stream, Cg };
enum class St { Stream, Keep };

template <Ld K>
__device__ __forceinline__ float2 ldx(const float2* p) {
    if constexpr (K == Ld::Stream) return __ldcs(p);
    else return __ldcg(p);
}
template <St K>
__device__ __forceinline__ void stx(float2* p, float2 v, uint64_t pol) {
    if constexpr (K == St::Stream) {
        __stcs(p, v);
    } else {
        asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y), "l"(pol)
                     : "memory");
    }
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// Shared-memory store that the compiler keeps after the memory operations
// before it: thread 0 of a persistent CTA publishes the next queue item
// (an atomic's result) only after issuing its own loads of the current tile,
// so waiting for the atomic never delays those loads.
__device__ __forceinline__ void st_shared_after(int* p, int v) {
    asm volatile("st.shared.b32 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}

// Drop a 128-byte L2 line without writing it back (scratch data only).
__device__ __forceinline__ void l2_discard_line(const void* p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

template <int R, int S, bool INV>
__device__ __forceinline__ void dft_at(float2* v) {
    dft<R, 0, S, INV>(v);
}

// Twiddles of a radix-16 pass P >= 1 that read six table entries per
// butterfly (W^k, W^2k, W^3k, W^4k, W^8k, W^12k; the other nine are one
// complex product of two of them).  They can be loaded ahead of the pass --
// before the exchange barrier that precedes it, where the data registers are
// free -- so the table loads' latency overlaps the barrier instead of
// stalling the butterflies.
template <class PL, int P>
struct TwPre {
    static constexpr bool ON = P > 0 && P < PL::NPASS && PL::radix(P) == 16 && kTwiddleLoads6;
    static constexpr int Q = ON ? PL::R / 16 : 1;
    float2 w[Q][6];
};

__device__ __forceinline__ float2 ldg_nc_f2(const float2* p) {
    float2 r;
    asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "l"(p));
    return r;
}

// Issue the table loads of pass P for butterflies b0 + q*T (no-op unless
// TwPre<PL, P>::ON).  The loads are volatile so the compiler keeps them ahead
// of the barrier that follows.
template <class PL, int P>
__device__ __forceinline__ void tw_preload(TwPre<PL, P>& pre, int b0, const float2* __restrict__ tw) {
    if constexpr (TwPre<PL, P>::ON) {
        constexpr int Ns = PL::ns(P);
#pragma unroll
        for (int q = 0; q < TwPre<PL, P>::Q; ++q) {
            const float2* tp = tw + PL::twoff(P) + ((b0 + q * PL::T) & (Ns - 1));
            pre.w[q][0] = ldg_nc_f2(tp);
            pre.w[q][1] = ldg_nc_f2(tp + Ns);
            pre.w[q][2] = ldg_nc_f2(tp + 2 * Ns);
            pre.w[q][3] = ldg_nc_f2(tp + 3 * Ns);
            pre.w[q][4] = ldg_nc_f2(tp + 7 * Ns);
            pre.w[q][5] = ldg_nc_f2(tp + 11 * Ns);
        }
    }
}

// Multiply the butterfly inputs of pass P by their twiddles and run the
// radix-R_P butterflies.  b0 = t (butterfly index of q = 0); butterfly q is
// b0 + q*T and owns v[q + Q*r].  `pre`: the pass's table entries loaded
// ahead by tw_preload (null: loaded here).
template <class PL, int P, bool INV>
__device__ __forceinline__ void pass_compute(float2 (&v)[PL::R], int b0, const float2* __restrict__ tw,
                                             const TwPre<PL, P>* pre = nullptr) {
    constexpr int Rp = PL::radix(P), Q = PL::R / Rp, Ns = PL::ns(P);
    if constexpr (P > 0 && Rp == 16 && kTwiddleLoads6) {
        // six table loads (W^k, W^2k, W^3k, W^4k, W^8k, W^12k); the other nine
        // twiddles are one complex product of two table values each
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            float2 w[16];
            if (pre) {
                w[1] = pre->w[q][0];
                w[2] = pre->w[q][1];
                w[3] = pre->w[q][2];
                w[4] = pre->w[q][3];
                w[8] = pre->w[q][4];
                w[12] = pre->w[q][5];
            } else {
                const float2* tp = tw + PL::twoff(P) + ((b0 + q * PL::T) & (Ns - 1));
                w[1] = __ldg(tp);
                w[2] = __ldg(tp + Ns);
                w[3] = __ldg(tp + 2 * Ns);
                w[4] = __ldg(tp + 3 * Ns);
                w[8] = __ldg(tp + 7 * Ns);
                w[12] = __ldg(tp + 11 * Ns);
            }
#pragma unroll
            for (int h = 4; h <= 12; h += 4)
#pragma unroll
                for (int l = 1; l <= 3; ++l) w[h + l] = cmul(w[h], w[l]);
#pragma unroll
            for (int r = 1; r < 16; ++r) v[q + Q * r] = twmul<INV>(v[q + Q * r], w[r]);
        }
    } else if constexpr (P > 0) {
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

// Shared-memory addresses: element a of column c (column stride CS, the
// number of interleaved columns) lives at padi(a*CS + c).  Since
// padi(x + 16m) = padi(x) + 17m, every address below is a per-thread base plus
// a compile-time offset, so each access is one shared load/store with an
// immediate offset.

// Scatter the outputs of pass P into the exchange buffer.
template <class PL, int P, int CS>
__device__ __forceinline__ void pass_scatter(const float2 (&v)[PL::R], int b0, float2* s, int coff) {
    constexpr int Rp = PL::radix(P), Q = PL::R / Rp, Ns = PL::ns(P);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int b = b0 + q * PL::T;
        const int k = b & (Ns - 1);
        const int base = (b - k) * Rp + k;
        if constexpr ((Ns * CS) % 16 == 0) {
            float2* p = s + padi(base * CS + coff);
#pragma unroll
            for (int r = 0; r < Rp; ++r) p[r * (Ns * CS / 16) * 17] = v[q + Q * r];
        } else if constexpr (Ns == 1 && Rp == 16 && 16 % CS == 0) {
            float2* p = s + 17 * b * CS + coff;  // base = 16 b, coff < CS
#pragma unroll
            for (int r = 0; r < Rp; ++r) p[r * CS + ((r * CS) >> 4)] = v[q + Q * r];
        } else {
#pragma unroll
            for (int r = 0; r < Rp; ++r) s[padi((base + r * Ns) * CS + coff)] = v[q + Q * r];
        }
    }
}

// Gather the pass inputs x[t + i*T] from the exchange buffer.
template <class PL, int CS>
__device__ __forceinline__ void pass_gather(float2 (&v)[PL::R], int t, const float2* s, int coff) {
    if constexpr ((PL::T * CS) % 16 == 0) {
        const float2* p = s + padi(t * CS + coff);
#pragma unroll
        for (int i = 0; i < PL::R; ++i) v[i] = p[i * (PL::T * CS / 16) * 17];
    } else {
#pragma unroll
        for (int i = 0; i < PL::R; ++i) v[i] = s[padi((t + i * PL::T) * CS + coff)];
    }
}

// Barrier over the threads of a tile: the whole CTA (NB = 0), or the first
// NB threads on named barrier 1 (tiles run by the consumer warps of a
// warp-specialised kernel, whose producer warp does not take part).
template <int NB>
__device__ __forceinline__ void tile_sync() {
    if constexpr (NB == 0) __syncthreads();
    else asm volatile("bar.sync 1, %0;" ::"n"(NB) : "memory");
}

// Barrier over the first NB threads (named barrier 1) that also returns
// whether `v` holds in every one of them.
template <int NB>
__device__ __forceinline__ bool tile_and(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\t"
        "setp.ne.u32 pi, %1, 0;\n\t"
        "bar.red.and.pred po, 1, %2, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(NB)
        : "memory");
    return r != 0;
}

// Barrier over the threads that share an exchange buffer.
template <bool WARP_ONLY, int NB = 0>
__device__ __forceinline__ void xsync() {
    if constexpr (WARP_ONLY) __syncwarp();
    else tile_sync<NB>();
}

// All passes from P on (CS interleaved columns in the exchange buffer).  With
// LAST_SYNC = false the barrier after the last gather is left out: the caller
// then rewrites the exchange area only after a barrier of its own (tile loop,
// CTA exit, cluster barrier).  Measured: faster for the column tiles of the
// persistent kernels, slower for the single-pass rows kernel.
template <class PL, int P, bool INV, bool WARP_ONLY, int CS, bool LAST_SYNC = true, int NB = 0>
__device__ __forceinline__ void run_passes(float2 (&v)[PL::R], int t, float2* s, int coff,
                                           const float2* __restrict__ tw, const TwPre<PL, P>* pre = nullptr) {
    pass_compute<PL, P, INV>(v, t, tw, pre);
    if constexpr (P + 1 < PL::NPASS) {
        pass_scatter<PL, P, CS>(v, t, s, coff);
        TwPre<PL, P + 1> next;
        tw_preload<PL, P + 1>(next, t, tw);  // in flight across the barrier
        xsync<WARP_ONLY, NB>();
        pass_gather<PL, CS>(v, t, s, coff);
        if constexpr (LAST_SYNC || P + 2 < PL::NPASS) xsync<WARP_ONLY, NB>();
        run_passes<PL, P + 1, INV, WARP_ONLY, CS, LAST_SYNC, NB>(v, t, s, coff, tw,
                                                                  TwPre<PL, P + 1>::ON ? &next : nullptr);
    }
}

// Passes P .. NPASS-2, ending with the scatter of the inputs of the last pass
// into the exchange buffer and a barrier (the caller gathers them with its own
// thread mapping).  Requires NPASS >= 2.
// The twiddles of each following pass are loaded ahead of the barrier before
// it; those of the last pass for its re-mapped butterfly index t_last, into
// `last`.
template <class PL, int P, bool INV, int NB = 0>
__device__ __forceinline__ void run_passes_to_last(float2 (&v)[PL::R], int t, float2* s,
                                                   const float2* __restrict__ tw, const TwPre<PL, P>* pre,
                                                   TwPre<PL, PL::NPASS - 1>& last, int t_last) {
    pass_compute<PL, P, INV>(v, t, tw, pre);
    pass_scatter<PL, P, 1>(v, t, s, 0);
    if constexpr (P + 2 < PL::NPASS) {
        TwPre<PL, P + 1> next;
        tw_preload<PL, P + 1>(next, t, tw);
        tile_sync<NB>();
        pass_gather<PL, 1>(v, t, s, 0);
        tile_sync<NB>();
        run_passes_to_last<PL, P + 1, INV, NB>(v, t, s, tw, TwPre<PL, P + 1>::ON ? &next : nullptr, last, t_last);
    } else {
        tw_preload<PL, PL::NPASS - 1>(last, t_last, tw);
        tile_sync<NB>();
    }
}

// ---------------------------------------------------------------------------
// Tile functions.  Each processes one tile with all threads of the CTA (the
// thread count must equal the tile's THREADS) and may be called repeatedly by
// a persistent CTA; the caller separates consecutive tiles with a barrier.
// ---------------------------------------------------------------------------

// Rows tile: TPC contiguous transforms of length N ([TPC][N] at src/dst);
// rows >= nrows are skipped (their threads still take part in the barriers).
template <int LOGN, int TPC, int RT = 16>
struct RowsCfg {
    using PL = P2Plan<LOGN, RT>;
    static constexpr int THREADS = PL::T * TPC;
    static constexpr int SMEM = (PL::NPASS > 1 ? PL::PADDED * TPC : 0) * 8;
};

template <int LOGN, int TPC, bool INV, Ld LK, St SK, int RT = 16>
__device__ __forceinline__ void rows_tile(const float2* __restrict__ src, float2* __restrict__ dst, int nrows,
                                          const float2* __restrict__ tw, float2* smem, uint64_t pol) {
    using PL = typename RowsCfg<LOGN, TPC, RT>::PL;
    const int t = threadIdx.x & (PL::T - 1);
    const int sub = threadIdx.x / PL::T;
    const bool ok = sub < nrows;
    src += (int64_t)sub * PL::N;
    dst += (int64_t)sub * PL::N;
    float2 v[PL::R];
#pragma unroll
    for (int i = 0; i < PL::R; ++i) v[i] = ok ? ldx<LK>(src + t + i * PL::T) : make_float2(0.f, 0.f);
    run_passes<PL, 0, INV, false, 1>(v, t, smem + sub * PL::PADDED, 0, tw);
    if (ok) {
#pragma unroll
        for (int i = 0; i < PL::R; ++i) stx<SK>(dst + t + i * PL::T, v[i], pol);
    }
}

// Transposed rows tile (four-step second pass).  src = TPC consecutive rows
// k1_0 .. k1_0+TPC-1 of one item ([TPC][N] contiguous); bin k2 of row
// k1_0 + c goes to dst[c + n1*k2] (dst = item base + k1_0).  All passes but
// the last run with thread (row, t); the last pass is re-mapped to thread
// (t', row) with the row index fastest, so the global stores write TPC
// consecutive k1 (TPC*8 bytes) for each k2 straight from registers.  Row
// pitch in shared memory is congruent to 16/TPC (mod 16) float2, so the
// re-mapped gather is bank-conflict free.
template <int LOGN, int TPC>
struct RowsTCfg {
    using PL = P2Plan<LOGN>;
    static constexpr int THREADS = PL::T * TPC;
    static constexpr int PITCH = ((PL::PADDED + 15) / 16) * 16 + (TPC >= 16 ? 1 : 16 / TPC);
    static constexpr int SMEM = PITCH * TPC * 8;
};

// Everything after the load: v holds x[t + i*T] of row `sub` (thread
// (sub, t), t = threadIdx.x mod T).
template <int LOGN, int TPC, bool INV, St SK, int NB = 0>
__device__ __forceinline__ void rowsT_tile_regs(float2 (&v)[P2Plan<LOGN>::R], float2* __restrict__ dst, int64_t n1,
                                                const float2* __restrict__ tw, float2* smem, uint64_t pol) {
    using CF = RowsTCfg<LOGN, TPC>;
    using PL = typename CF::PL;
    static_assert(PL::NPASS >= 2, "transposed rows need at least two passes");
    const int t = threadIdx.x & (PL::T - 1);
    const int sub = threadIdx.x / PL::T;
    const int c = threadIdx.x % TPC;
    const int t2 = threadIdx.x / TPC;
    TwPre<PL, PL::NPASS - 1> last;
    run_passes_to_last<PL, 0, INV, NB>(v, t, smem + sub * CF::PITCH, tw, nullptr, last, t2);
    const float2* sc = smem + c * CF::PITCH;
    if constexpr (PL::T % 16 == 0) {
        const float2* p = sc + padi(t2);
#pragma unroll
        for (int i = 0; i < PL::R; ++i) v[i] = p[i * (PL::T / 16) * 17];
    } else {
#pragma unroll
        for (int i = 0; i < PL::R; ++i) v[i] = sc[padi(t2 + i * PL::T)];
    }
    pass_compute<PL, PL::NPASS - 1, INV>(v, t2, tw, TwPre<PL, PL::NPASS - 1>::ON ? &last : nullptr);
    float2* d0 = dst + c;
#pragma unroll
    for (int i = 0; i < PL::R; ++i) stx<SK>(d0 + n1 * (int64_t)(t2 + i * PL::T), v[i], pol);
}

template <int LOGN, int TPC, bool INV, Ld LK, St SK>
__device__ __forceinline__ void rowsT_tile(const float2* __restrict__ src, float2* __restrict__ dst, int64_t n1,
                                           const float2* __restrict__ tw, float2* smem, uint64_t pol) {
    using PL = P2Plan<LOGN>;
    const int t = threadIdx.x & (PL::T - 1);
    const float2* s0 = src + (int64_t)(threadIdx.x / PL::T) * PL::N;
    float2 v[PL::R];
#pragma unroll
    for (int i = 0; i < PL::R; ++i) v[i] = ldx<LK>(s0 + t + i * PL::T);
    rowsT_tile_regs<LOGN, TPC, INV, SK>(v, dst, n1, tw, smem, pol);
}

// Columns tile: C adjacent columns of a row-major [N][S] array (src/dst point
// at the tile's first column), each column a transform of length N with
// element stride S.  Used for the 2-D column pass (S = W) and the four-step
// first pass (S = N2), where TW multiplies element (k1, n2) by
// W_{N*S}^{n2*k1}, n2 = col0 + c.  With k1 = t + i*T that factor is
// W^{n2*t} * W^{n2*T*i}: the first is read once per thread and the second
// once per (column, i) into shared memory, each from the two-level table
// W(m) = hi[m >> sh] * lo[m & (2^sh - 1)] (m < N*S, no reduction needed).
// Thread (c, t): c = threadIdx.x % C is the column (fastest, so each warp
// touches C*8 contiguous bytes per row), t the Stockham thread index.
template <int LOGN, int C>
struct ColsCfg {
    using PL = P2Plan<LOGN>;
    static constexpr int THREADS = PL::T * C;
    static constexpr int XBUF = PL::NPASS > 1 ? padi(PL::N * C) : 0;  // float2
    static constexpr int SMEM = (XBUF + C * PL::R) * 8;
};

__device__ __forceinline__ float2 root2(const float2* __restrict__ lo, const float2* __restrict__ hi, uint32_t m,
                                        int sh) {
    return cmul(__ldg(hi + (m >> sh)), __ldg(lo + (m & ((1u << sh) - 1u))));
}

// Everything after the load: v holds x[t + i*T] of column c (thread (c, t)).
// With TW the twiddle of element (k1, n2) is W^{tws*n2*k1} of the two-level
// table (tws > 1 reuses a longer transform's table for a divisor length).
// `steps_buf` (C * 16 float2) holds the per-column twiddle steps; null: right
// after the exchange buffer (smem + XBUF).
template <int LOGN, int C, bool INV, bool TW, St SK, int NB = 0>
__device__ __forceinline__ void cols_tile_regs(float2 (&v)[P2Plan<LOGN>::R], float2* __restrict__ dst, int64_t S,
                                               uint32_t col0, const float2* __restrict__ tw,
                                               const float2* __restrict__ tw_lo, const float2* __restrict__ tw_hi,
                                               int sh, float2* smem, uint64_t pol, uint32_t tws = 1,
                                               float2* steps_buf = nullptr) {
    using CF = ColsCfg<LOGN, C>;
    using PL = typename CF::PL;
    const int c = threadIdx.x % C;
    const int t = threadIdx.x / C;
    // [R][C]: W^{n2*T*i} (column fastest: conflict-free reads)
    float2* steps = steps_buf ? steps_buf : smem + CF::XBUF;
    if constexpr (TW) {
        for (int j = threadIdx.x; j < C * PL::R; j += CF::THREADS) {
            const int cc = j % C, ii = j / C;
            steps[ii * C + cc] = root2(tw_lo, tw_hi, (col0 + (uint32_t)cc) * tws * (uint32_t)(ii * PL::T), sh);
        }
        if constexpr (PL::NPASS == 1) tile_sync<NB>();
    }

    run_passes<PL, 0, INV, false, C, false, NB>(v, t, smem, c, tw);

    if constexpr (TW) {
        const float2 w0 = root2(tw_lo, tw_hi, (col0 + (uint32_t)c) * tws * (uint32_t)t, sh);
#pragma unroll
        for (int i = 0; i < PL::R; ++i) v[i] = twmul<INV>(v[i], cmul(w0, steps[i * C + c]));
    }
    dst += c;
#pragma unroll
    for (int i = 0; i < PL::R; ++i) stx<SK>(dst + (int64_t)(t + i * PL::T) * S, v[i], pol);
}

template <int LOGN, int C, bool INV, bool TW, Ld LK, St SK>
__device__ __forceinline__ void cols_tile(const float2* __restrict__ src, float2* __restrict__ dst, int64_t S,
                                          uint32_t col0, const float2* __restrict__ tw,
                                          const float2* __restrict__ tw_lo, const float2* __restrict__ tw_hi, int sh,
                                          float2* smem, uint64_t pol) {
    using PL = P2Plan<LOGN>;
    const int t = threadIdx.x / C;
    src += threadIdx.x % C;
    float2 v[PL::R];
#pragma unroll
    for (int i = 0; i < PL::R; ++i) v[i] = ldx<LK>(src + (int64_t)(t + i * PL::T) * S);
    cols_tile_regs<LOGN, C, INV, TW, SK>(v, dst, S, col0, tw, tw_lo, tw_hi, sh, smem, pol);
}

// ---------------------------------------------------------------------------
// One-tile-per-CTA kernels.
// ---------------------------------------------------------------------------
// RT = 32 (two butterflies per thread) takes ~115 registers: 512 threads/SM.
template <int LOGN, int TPC, bool INV, int RT = 16>
__global__ void __launch_bounds__(RowsCfg<LOGN, TPC, RT>::THREADS,
                                  (RT == 16 ? 1024 : 512) / RowsCfg<LOGN, TPC, RT>::THREADS)
k_rows_pow2(const float2* __restrict__ in, float2* __restrict__ out, int64_t nrows, const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    const int64_t row0 = (int64_t)blockIdx.x * TPC;
    const int64_t left = nrows - row0;
    rows_tile<LOGN, TPC, INV, Ld::Stream, St::Stream, RT>(in + row0 * (1 << LOGN), out + row0 * (1 << LOGN),
                                                          left < TPC ? (int)left : TPC, tw, smem, 0);
}

// nrows = items * n1 rows; the CTA's TPC rows are consecutive k1 of one item.
template <int LOGN, int TPC, bool INV>
__global__ void __launch_bounds__(RowsTCfg<LOGN, TPC>::THREADS, 1024 / RowsTCfg<LOGN, TPC>::THREADS)
k_rowsT_pow2(const float2* __restrict__ in, float2* __restrict__ out, int64_t nrows, const float2* __restrict__ tw,
             int64_t n1) {
    extern __shared__ float2 smem[];
    const int64_t row0 = (int64_t)blockIdx.x * TPC;
    const int64_t item = row0 / n1;
    const int64_t k10 = row0 - item * n1;
    rowsT_tile<LOGN, TPC, INV, Ld::Stream, St::Stream>(in + row0 * (1 << LOGN),
                                                       out + item * n1 * (1 << LOGN) + k10, n1, tw, smem, 0);
}

template <int LOGN, int C, bool INV, bool TWIDDLE_OUT>
__global__ void __launch_bounds__(ColsCfg<LOGN, C>::THREADS, 1024 / ColsCfg<LOGN, C>::THREADS)
k_cols_pow2(const float2* __restrict__ in, float2* __restrict__ out, int64_t S, int64_t ngroups_per_item,
            int64_t item_stride, int64_t nitems, const float2* __restrict__ tw,
            const float2* __restrict__ tw_lo, const float2* __restrict__ tw_hi, int sh) {
    extern __shared__ float2 smem[];
    const int64_t item = blockIdx.x / ngroups_per_item;
    const int64_t g = blockIdx.x - item * ngroups_per_item;
    if (item >= nitems) return;  // uniform per CTA
    const int64_t off = item * item_stride + g * C;
    cols_tile<LOGN, C, INV, TWIDDLE_OUT, Ld::Stream, St::Stream>(in + off, out + off, S, (uint32_t)(g * C), tw,
                                                                 tw_lo, tw_hi, sh, smem, 0);
}

}  // namespace b300fft
