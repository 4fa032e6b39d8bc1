// tc.cuh -- radix-16 Stockham passes whose 16-point DFTs run on the 5th-gen
// tensor cores (tcgen05.mma, kind::f16, FP32 accumulation in TMEM).
//
// One pass of a length-16^k transform does N/16 radix-16 butterflies (the
// paper's Sec. III-A small-DFT node).  Collected over 128 butterflies that is
// a dense real GEMM:
//     D (128 x 32) = A (128 x 32) * B (32 x 32),
//     A[m][k]  = twiddled inputs of butterfly m, k < 16: Re v_k, k >= 16: Im v_{k-16}
//     B^T[n][k] = real embedding of DFT-16:  [[C, S], [-S, C]]  (forward,
//                 C = cos(2 pi jk/16), S = sin(2 pi jk/16); S -> -S inverse)
//     D[m][n]  = Re y_n (n < 16), Im y_{n-16} (n >= 16).
// Precision: each butterfly's inputs are scaled by a power of two so their
// largest component lies in [1, 2) (exact, undone after the GEMM), then
// split a = a_hi + a_lo and b = b_hi + b_lo in FP16 or BF16 (round to
// nearest even); the GEMM accumulates a_hi*b_hi + a_hi*b_lo + a_lo*b_hi in
// FP32 ("plain" modes: a_hi*b_hi only).  Twiddles between passes stay FP32 on
// the CUDA cores.
//
// Operand layout (shared memory, K-major, no swizzle): 8x8 core matrices of
// 16-bit values, 128 contiguous bytes each; core matrix (row block i, k block
// j) at byte (4*i + j)*128, so the leading (K) byte offset is 128 and the
// stride (M/N) byte offset 512.  One MMA covers K = 16 (two k blocks); the
// second K half starts 256 bytes later.  Thread t of the CTA owns butterfly
// row t % 128 of M-tile t / 128 and TMEM lane t % 128 (warp w reads lanes
// 32*(w%4) ...), columns 32 * (t / 128) ... + 31.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "stockham_pow2.cuh"
#include "tma.cuh"  // smem_u32, mbar_init

namespace b300fft {

enum : int { TC_FP16 = 1, TC_BF16 = 2, TC_FP16_PLAIN = 3, TC_BF16_PLAIN = 4 };

template <int MODE>
struct TcMode {
    static constexpr bool BF16 = MODE == TC_BF16 || MODE == TC_BF16_PLAIN;
    static constexpr bool SPLIT = MODE == TC_FP16 || MODE == TC_BF16;
    // instruction descriptor: D f32, A/B f16 (0) or bf16 (1), K-major both,
    // N = 32 (bits 17-22: N>>3), M = 128 (bits 24-28: M>>4)
    static constexpr uint32_t IDESC =
        (1u << 4) | ((BF16 ? 1u : 0u) << 7) | ((BF16 ? 1u : 0u) << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
};

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    constexpr uint64_t LBO = 128, SBO = 512;
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= ((LBO >> 4) & 0x3FFFu) << 16;
    d |= ((SBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of tcgen05; base offset 0; SWIZZLE_NONE
    return d;
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bounded wait for the MMA completion barrier: plain polls without a
// suspend-time hint (the MMAs of one pass take a few hundred cycles); false
// after `polls` polls.
__device__ __forceinline__ bool tc_mma_wait(uint64_t* bar, uint32_t parity, int polls) {
    for (int i = 0; i < polls; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&f)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) f[i] = __uint_as_float(r[i]);
}

// 16-bit value bits and the residual split.
template <bool BF>
__device__ __forceinline__ uint16_t to16(float x, float* back) {
    if constexpr (BF) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        *back = __bfloat162float(h);
        return __bfloat16_as_ushort(h);
    } else {
        const __half h = __float2half_rn(x);
        *back = __half2float(h);
        return __half_as_ushort(h);
    }
}

// Shared state of the tensor-core butterflies of one CTA.
struct TcCtx {
    uint8_t* a_hi;  // [tiles][8 KB] A operand, high parts
    uint8_t* a_lo;  // [tiles][8 KB] A operand, low parts
    uint8_t* b_hi;  // 2 KB  DFT-16 embedding, high parts
    uint8_t* b_lo;  // 2 KB  low parts
    uint64_t* bar;  // MMA completion barrier
    uint32_t tmem;  // TMEM base address (lane 0, first column)
    uint32_t phase;
    int* status;    // device status word (FFT_ERR_TIMEOUT on an expired wait)
};

// byte offset of element (row, k) of a 32-wide K-major core-matrix operand
__device__ __forceinline__ int op_off(int row, int k) { return ((row >> 3) * 4 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2; }

// Element (n, k) of the real embedding of the DFT-16 (direction INV).
__device__ __forceinline__ double dft16_embed(int n, int k, bool inv) {
    const int j = n & 15, i = k & 15;
    double sn, co;
    sincospi(2.0 * (double)((i * j) & 15) / 16.0, &sn, &co);
    if (inv) sn = -sn;
    // forward y = (C - iS) v:  Re y = C Re v + S Im v ;  Im y = -S Re v + C Im v
    if (n < 16) return (k < 16) ? co : sn;
    return (k < 16) ? -sn : co;
}

// Two values rounded to a packed pair of 16-bit values (element k in the low
// half, k + 1 in the high half) and the pair of residuals x - round(x).
template <bool BF>
__device__ __forceinline__ uint32_t to16x2(float x0, float x1, float* r0, float* r1) {
    if constexpr (BF) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
        const float2 b = __bfloat1622float2(h);
        *r0 = x0 - b.x;
        *r1 = x1 - b.y;
        return *reinterpret_cast<const uint32_t*>(&h);
    } else {
        const __half2 h = __floats2half2_rn(x0, x1);
        const float2 b = __half22float2(h);
        *r0 = x0 - b.x;
        *r1 = x1 - b.y;
        return *reinterpret_cast<const uint32_t*>(&h);
    }
}

// Radix-16 butterfly of this thread on the tensor cores.  Called by all
// threads of the CTA together (one butterfly each); v in/out natural order.
// Thread 0 issues the MMAs and waits (bounded) for their completion; the
// other threads wait in the barrier after it, then read their accumulator
// lane.  Returns false (in every thread) when the wait ran out: the results
// are then not read and the caller stops.
template <int MODE>
__device__ __forceinline__ bool tc_dft16(float2 (&v)[16], TcCtx& c, int ntiles) {
    constexpr bool BF = TcMode<MODE>::BF16;
    constexpr bool SPLIT = TcMode<MODE>::SPLIT;
    const int row = threadIdx.x & 127, tile = threadIdx.x >> 7;
    // power-of-two scale: largest component into [1, 2)
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) mx = fmaxf(mx, fmaxf(fabsf(v[i].x), fabsf(v[i].y)));
    int e = 0;
    if (mx > 0.f) e = ((__float_as_int(mx) >> 23) & 0xff) - 127;
    e = e < -120 ? -120 : (e > 120 ? 120 : e);
    const float sc = __int_as_float((127 - e) << 23), inv_sc = __int_as_float((127 + e) << 23);
    uint8_t* ahi = c.a_hi + tile * 8192;
    uint8_t* alo = c.a_lo + tile * 8192;
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = kb * 8 + q * 2;  // k and k + 1 are both real or both imaginary parts
            const float x0 = (k < 16 ? v[k].x : v[k - 16].y) * sc;
            const float x1 = (k < 16 ? v[k + 1].x : v[k - 15].y) * sc;
            float r0, r1;
            hw[q] = to16x2<BF>(x0, x1, &r0, &r1);
            if constexpr (SPLIT) {
                float d0, d1;
                lw[q] = to16x2<BF>(r0, r1, &d0, &d1);
            }
        }
        const int off = op_off(row, kb * 8);
        *reinterpret_cast<uint4*>(ahi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        if constexpr (SPLIT) *reinterpret_cast<uint4*>(alo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    fence_async_smem();
    __syncthreads();
    int late = 0;
    if (threadIdx.x == 0) {
        tc_fence_after();
        constexpr uint32_t ID = TcMode<MODE>::IDESC;
        const uint32_t bh = smem_u32(c.b_hi), bl = smem_u32(c.b_lo);
        for (int t = 0; t < ntiles; ++t) {
            const uint32_t d = c.tmem + 32u * t;
            const uint32_t ah = smem_u32(c.a_hi + t * 8192), al = smem_u32(c.a_lo + t * 8192);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const uint32_t ko = ks * 256;
                tc_mma(d, umma_desc(ah + ko), umma_desc(bh + ko), ID, ks > 0);
                if constexpr (SPLIT) {
                    tc_mma(d, umma_desc(ah + ko), umma_desc(bl + ko), ID, 1);
                    tc_mma(d, umma_desc(al + ko), umma_desc(bh + ko), ID, 1);
                }
            }
        }
        tc_commit(c.bar);
        // bounded wait for the MMAs
        if (!tc_mma_wait(c.bar, c.phase, 1 << 22)) {
            late = 1;
            atomicCAS(c.status, 0, 6);
        }
    }
    if (__syncthreads_or(late)) return false;
    c.phase ^= 1u;
    tc_fence_after();
    float f[32];
    tmem_ld32(c.tmem + ((uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16) + 32u * tile, f);
    tc_fence_before();
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = make_float2(f[j] * inv_sc, f[16 + j] * inv_sc);
    return true;
}

// The 15 twiddles of radix-16 pass P (P >= 1) for butterfly t, loaded as
// volatile loads so they stay ahead of the barrier that follows them.
template <class PL, int P>
__device__ __forceinline__ void tc_tw_load(float2 (&w)[15], int t, const float2* __restrict__ tw) {
    constexpr int Ns = PL::ns(P);
    const float2* twp = tw + PL::twoff(P) + (t & (Ns - 1));
#pragma unroll
    for (int r = 1; r < 16; ++r) w[r - 1] = ldg_nc_f2(twp + (r - 1) * Ns);
}

// Stockham passes of a 16^k transform with tensor-core butterflies.  Same
// thread layout and exchange as run_passes (R = 16, one butterfly per thread);
// each pass's twiddles are loaded before the exchange barrier ahead of it.
// False when an MMA wait ran out (every thread; nothing further is issued).
template <class PL, int P, bool INV, int MODE, int CS>
__device__ __forceinline__ bool tc_run_passes(float2 (&v)[16], int t, float2* s, int coff,
                                              const float2* __restrict__ tw, TcCtx& c, int ntiles,
                                              const float2 (*w)[15] = nullptr) {
    static_assert(PL::R == 16 && PL::radix(P) == 16, "tensor-core passes are radix 16");
    if constexpr (P > 0) {
#pragma unroll
        for (int r = 1; r < 16; ++r) v[r] = twmul<INV>(v[r], (*w)[r - 1]);
    }
    if (!tc_dft16<MODE>(v, c, ntiles)) return false;
    if constexpr (P + 1 < PL::NPASS) {
        pass_scatter<PL, P, CS>(v, t, s, coff);
        float2 wn[15];
        tc_tw_load<PL, P + 1>(wn, t, tw);
        __syncthreads();
        pass_gather<PL, CS>(v, t, s, coff);
        __syncthreads();
        return tc_run_passes<PL, P + 1, INV, MODE, CS>(v, t, s, coff, tw, c, ntiles, &wn);
    }
    return true;
}

// Shared-memory carve-up of a tensor-core CTA (after the FP32 exchange area).
template <int THREADS>
struct TcSmem {
    static constexpr int TILES = THREADS / 128;
    static constexpr int A_BYTES = TILES * 8192;
    static constexpr int BYTES = 2 * A_BYTES + 2 * 2048 + 64;
};

template <int THREADS>
__device__ __forceinline__ TcCtx tc_setup(uint8_t* base, uint32_t* tmem_slot, int* status,
                                          const uint4* __restrict__ bmat) {
    using SM = TcSmem<THREADS>;
    TcCtx c;
    c.a_hi = base;
    c.a_lo = base + SM::A_BYTES;
    c.b_hi = base + 2 * SM::A_BYTES;
    c.b_lo = c.b_hi + 2048;
    c.bar = reinterpret_cast<uint64_t*>(c.b_lo + 2048);
    c.phase = 0;
    c.status = status;
    // B operands (hi then lo, 4 KB) prepared at plan time
    for (int i = threadIdx.x; i < 256; i += THREADS) reinterpret_cast<uint4*>(c.b_hi)[i] = __ldg(bmat + i);
    if (threadIdx.x == 0) mbar_init(c.bar, 1);
    if (threadIdx.x < 32) tmem_alloc(tmem_slot, 32 * SM::TILES < 32 ? 32 : 32 * SM::TILES);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    c.tmem = *tmem_slot;
    return c;
}

// Release the CTA's TMEM.  `failed`: an MMA wait ran out; thread 0 then
// waits once more (bounded) for those MMAs before the columns are freed.
template <int THREADS>
__device__ __forceinline__ void tc_teardown(const TcCtx& c, bool failed = false) {
    if (failed && threadIdx.x == 0) tc_mma_wait(c.bar, c.phase, 1 << 22);
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_fence_after();
        tmem_dealloc(c.tmem, 32 * TcSmem<THREADS>::TILES < 32 ? 32 : 32 * TcSmem<THREADS>::TILES);
    }
}

// ---------------------------------------------------------------------------
// Kernels.  Rows: TPC contiguous transforms of 16^k (k = 2, 3) per CTA with
// TPC * N/16 = THREADS in {128, 256}.  Columns / transposed rows: the
// four-step passes of 65536 = 256 * 256 (16 columns or rows of 256 per CTA).
// ---------------------------------------------------------------------------
// Dynamic shared memory of the four-step tensor-core kernels.
constexpr int tc_cols_smem() { return (padi(256 * 16) + 16 * 16) * 8 + TcSmem<256>::BYTES; }
constexpr int tc_rowsT_smem() { return ((RowsTCfg<8, 16>::SMEM + 127) / 128) * 128 + TcSmem<256>::BYTES; }

template <int LOGN, int TPC>
struct TcRowsCfg {
    using PL = P2Plan<LOGN>;
    static constexpr int THREADS = PL::T * TPC;
    static constexpr int XBYTES = PL::PADDED * TPC * 8;
    static constexpr int SMEM = XBYTES + TcSmem<THREADS>::BYTES;
};

// The kernels are persistent: each CTA allocates its TMEM columns and loads
// the DFT operands once, then takes work units (row groups, column groups)
// blockIdx.x, blockIdx.x + gridDim.x, ...  Resident CTAs per SM (the
// launch-bounds minimum, which registers and shared memory both allow; 64
// TMEM columns each):
constexpr int kTcRowsPerSm = 3, kTcColsPerSm = 2, kTcRowsTPerSm = 3;
template <int LOGN, int TPC, int MODE, bool INV>
__global__ void __launch_bounds__(TcRowsCfg<LOGN, TPC>::THREADS, kTcRowsPerSm)
k_tc_rows(const float2* __restrict__ in, float2* __restrict__ out, int64_t nrows, const float2* __restrict__ tw,
          int* status, const uint4* __restrict__ bmat) {
    using CF = TcRowsCfg<LOGN, TPC>;
    using PL = typename CF::PL;
    static_assert(CF::THREADS == 128 || CF::THREADS == 256, "one butterfly per TMEM lane");
    extern __shared__ __align__(128) uint8_t smem_raw[];
    __shared__ uint32_t tmem_slot;
    float2* xs = reinterpret_cast<float2*>(smem_raw);
    TcCtx c = tc_setup<CF::THREADS>(smem_raw + CF::XBYTES, &tmem_slot, status, bmat);
    const int t = threadIdx.x & (PL::T - 1);
    const int sub = threadIdx.x / PL::T;
    bool ok = true;
    for (int64_t grp = blockIdx.x; ok && grp * TPC < nrows; grp += gridDim.x) {
        const int64_t row = grp * TPC + sub;
        const bool have = row < nrows;
        const float2* src = in + row * PL::N;
        float2 v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = have ? ld_stream(src + t + i * PL::T) : make_float2(0.f, 0.f);
        ok = tc_run_passes<PL, 0, INV, MODE, 1>(v, t, xs + sub * PL::PADDED, 0, tw, c, CF::THREADS / 128);
        if (ok && have) {
            float2* dst = out + row * PL::N;
#pragma unroll
            for (int i = 0; i < 16; ++i) st_stream(dst + t + i * PL::T, v[i]);
        }
        __syncthreads();  // the exchange area is rewritten by the next group
    }
    tc_teardown<CF::THREADS>(c, !ok);
}

// Four-step pass A with tensor cores: C = 16 columns of length 256, stride S,
// output multiplied by W_{256*S}^{n2*k1}; units = column groups of all items.
template <int MODE, bool INV>
__global__ void __launch_bounds__(256, kTcColsPerSm)  // ~100 registers: a 3-CTA cap spills
k_tc_cols256(const float2* __restrict__ in, float2* __restrict__ out, int64_t S, int64_t ngroups_per_item,
             int64_t item_stride, int64_t units, const float2* __restrict__ tw, const float2* __restrict__ lo,
             const float2* __restrict__ hi, int sh, int* status, const uint4* __restrict__ bmat) {
    using PL = P2Plan<8>;
    constexpr int C = 16;
    constexpr int XBYTES = (padi(PL::N * C) + C * PL::R) * 8;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    __shared__ uint32_t tmem_slot;
    float2* xs = reinterpret_cast<float2*>(smem_raw);
    TcCtx c = tc_setup<256>(smem_raw + XBYTES, &tmem_slot, status, bmat);
    const int cc = threadIdx.x % C, t = threadIdx.x / C;
    float2* steps = xs + padi(PL::N * C);
    bool ok = true;
    for (int64_t u = blockIdx.x; ok && u < units; u += gridDim.x) {
        const int64_t item = u / ngroups_per_item;
        const int64_t g = u - item * ngroups_per_item;
        const int64_t col = g * C + cc;
        const float2* src = in + item * item_stride + col;
        float2 v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = ld_stream(src + (int64_t)(t + i * PL::T) * S);
        for (int j = threadIdx.x; j < C * PL::R; j += 256) {
            const int c2 = j % C, ii = j / C;
            steps[ii * C + c2] = root2(lo, hi, (uint32_t)(g * C + c2) * (uint32_t)(ii * PL::T), sh);
        }
        ok = tc_run_passes<PL, 0, INV, MODE, C>(v, t, xs, cc, tw, c, 2);
        if (ok) {
            const float2 w0 = root2(lo, hi, (uint32_t)col * (uint32_t)t, sh);
            float2* dst = out + item * item_stride + col;
#pragma unroll
            for (int i = 0; i < 16; ++i)
                st_stream(dst + (int64_t)(t + i * PL::T) * S, twmul<INV>(v[i], cmul(w0, steps[i * C + cc])));
        }
        __syncthreads();  // steps and the exchange area are rewritten by the next unit
    }
    tc_teardown<256>(c, !ok);
}

// Four-step pass B with tensor cores: TPC = 16 rows of length 256; the last
// pass is re-mapped row-fastest for the transposed store (like rowsT_tile);
// units = groups of 16 rows (nrows = items * n1 rows).
template <int MODE, bool INV>
__global__ void __launch_bounds__(256, kTcRowsTPerSm)
k_tc_rowsT256(const float2* __restrict__ in, float2* __restrict__ out, const float2* __restrict__ tw, int64_t n1,
              int64_t units, int* status, const uint4* __restrict__ bmat) {
    using PL = P2Plan<8>;
    constexpr int TPC = 16;
    using CF = RowsTCfg<8, TPC>;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    __shared__ uint32_t tmem_slot;
    float2* xs = reinterpret_cast<float2*>(smem_raw);
    constexpr int XBYTES = ((CF::SMEM + 127) / 128) * 128;
    TcCtx c = tc_setup<256>(smem_raw + XBYTES, &tmem_slot, status, bmat);
    const int t = threadIdx.x & (PL::T - 1);
    const int sub = threadIdx.x / PL::T;
    const int r = threadIdx.x % TPC, t2 = threadIdx.x / TPC;
    bool ok = true;
    for (int64_t u = blockIdx.x; ok && u < units; u += gridDim.x) {
        const int64_t row0 = u * TPC;
        const int64_t item = row0 / n1;
        const int64_t k10 = row0 - item * n1;
        const float2* s0 = in + (row0 + sub) * PL::N;
        float2 v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = ld_stream(s0 + t + i * PL::T);
        // pass 0 (row-major mapping), exchange
        ok = tc_dft16<MODE>(v, c, 2);
        if (!ok) break;
        float2* sx = xs + sub * CF::PITCH;
        pass_scatter<PL, 0, 1>(v, t, sx, 0);
        // pass 1 re-mapped: row r = threadIdx % 16, butterfly t2 = threadIdx / 16
        float2 w[15];
        tc_tw_load<PL, 1>(w, t2, tw);
        __syncthreads();
        const float2* sc = xs + r * CF::PITCH;
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = sc[padi(t2 + i * PL::T)];
#pragma unroll
        for (int q = 1; q < 16; ++q) v[q] = twmul<INV>(v[q], w[q - 1]);
        ok = tc_dft16<MODE>(v, c, 2);  // its first barrier also ends this unit's gathers
        if (!ok) break;
        float2* d0 = out + item * n1 * PL::N + k10 + r;
#pragma unroll
        for (int i = 0; i < 16; ++i) st_stream(d0 + n1 * (int64_t)(t2 + i * PL::T), v[i]);
    }
    tc_teardown<256>(c, !ok);
}

// Plan-time table of the B operands: out = [hi 2 KB][lo 2 KB] in the
// core-matrix layout, FP64 values rounded once to FP16/BF16 (hi), then the
// residual rounded again (lo).
template <bool BF>
__global__ void k_tc_bmat(uint8_t* out, int inv) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 32 * 32) return;
    const int n = e / 32, k = e % 32;
    const double val = dft16_embed(n, k, inv != 0);
    float back;
    const uint16_t hi = to16<BF>((float)val, &back);
    const uint16_t lo = to16<BF>((float)(val - (double)back), &back);
    *reinterpret_cast<uint16_t*>(out + op_off(n, k)) = hi;
    *reinterpret_cast<uint16_t*>(out + 2048 + op_off(n, k)) = lo;
}

}  // namespace b300fft
