// generic.cuh -- runtime mixed-radix Stockham tiles and the stage-graph
// executor used for non-power-of-two lengths, Bluestein's algorithm and the
// ragged (uneven-length) batch.
//
// A transform is a short chain of *stages*; a stage is a set of independent
// *tiles*; a tile transforms `nl` lines of one length L = R_0*R_1*...
// (radices 2,3,4,5,7,8,16) inside one CTA:
//   1. coalesced load of the tile into shared memory (optionally multiplied
//      by a table, zero at offsets >= in_valid),
//   2. Stockham passes between two shared-memory buffers (the pass formula of
//      the power-of-two kernels, with runtime radices),
//   3. the last pass stores to global memory, optionally multiplied by the
//      four-step twiddle W_{lines*L}^{line*k} or by a table, and only at
//      offsets < out_valid.
// Chains (the paper's Sec. III-A Cooley-Tukey split N = N1*N2, and the
// chirp-z rewrite n*k = (n^2 + k^2 - (k-n)^2)/2 for awkward lengths):
//   single      in -> out                                   (L <= tile max)
//   four-step   A: columns (L=N1, stride N2) x W_N^{n2 k1} -> work1
//               B: rows (L=N2) stored transposed             -> out
//   Bluestein   FFT_M of x*w (zero padded), x filter, IFFT_M, x w,
//               as 2 single-tile stages or 4 four-step stages.
// Every tile of stage s of a transform waits (bounded) for all tiles of
// stage s-1 of the same transform; the executor dequeues tiles from one
// atomic counter in an order where dependencies always come first.
#pragma once
#include "butterfly.cuh"
#include "mixed.cuh"
#include "persist.cuh"

namespace b300fft {

constexpr int kGMaxPass = 8;
constexpr int kGTileMax = 4096;  // complex elements per tile (lines * L)
constexpr int kGMaxLines = 128;
constexpr int kGThreads = 256;
constexpr int kGBuf = kGTileMax + kGTileMax / 16 + kGMaxLines;  // float2 per smem buffer
constexpr int kGSmem = 2 * kGBuf * 8;

struct GShape {
    int L, npass;
    int radix[kGMaxPass];
    int ns[kGMaxPass];
    int64_t tw[kGMaxPass];  // offset of pass p's table in the pool (p >= 1)
};

enum : int { G_PRE_NONE = 0, G_PRE_TABLE = 1, G_PRE_TABLE_CONJ = 2 };
enum : int { G_POST_NONE = 0, G_POST_TW4 = 1, G_POST_TABLE = 2, G_POST_TABLE_CONJ = 3 };
enum : int { G_BUF_IN = 0, G_BUF_OUT = 1, G_BUF_W1 = 2, G_BUF_W2 = 3 };

struct GStage {
    int shape;  // GShape index
    int nlines, lpt, ntiles;
    int in_buf, out_buf;
    int in_line_fast;   // 1: load with the line index fastest (column tiles)
    int out_line_fast;  // 1: last pass with the line index fastest (transposed stores)
    int inv;            // direction of this stage's transform
    int pre, post;
    int sh;
    int tmpl;  // > 0: templated tiles: 2 * log2 N + (0: A, 1: B) of a power-of-two four-step,
               // 100 + log2 N2: second stage (rows of 2^L2) of a mixed-length four-step,
               // 1000 + 16 M + K: single-tile lines of M * 2^K (compile-time passes; M = 1:
               // a power of two),
               // 2000 + 16 M + A: four-step first stage, columns of M * 2^A (compile-time),
               // 3000 + K2: four-step second stage, rows of 2^K2 with the transposed store
               //            (and the post-multiply of Bluestein's transforms),
               // 4000 + K: Bluestein's single-tile stage of M = 2^K (pre / post multiplies),
               // 5000 + A: Bluestein's four-step first stage, columns of 2^A (pre multiply)
    int64_t in_ls, in_es, out_ls, out_es;  // line / element strides (elements)
    int64_t in_valid, out_valid;           // offsets >= these read as 0 / are not stored
    int64_t pre_tab, post_tab;             // table offsets in the pool
    int64_t mtab;                          // compile-time tiles (tmpl >= 1000): their pass table in the pool
    int64_t lo, hi;                        // four-step two-level table in the pool
    int64_t line_tab;  // >= 0: the lines are separate transforms; line l starts at line_off[line_tab + l]
};

struct GTransform {
    int kind;  // index of its first stage in the stage array
    int nstages;
    int ctr;  // first of its nstages-1 dependency counters
    int pad_;
    int64_t in_off, out_off, w1_off, w2_off;
};

struct GExecArgs {
    const float2* in;
    float2* out;
    float2* work;
    const float2* pool;  // twiddle / chirp / filter tables
    const GShape* shapes;
    const GStage* stages;  // for this direction
    const GTransform* xf;
    const uint64_t* items;  // (transform << 32) | (stage << 24) | tile
    int nitems;
    int* ctl;    // [0] queue head, [1 + c] dependency counters
    int* qhead;  // queue head of this launch (ctl[0], or a second head past the counters)
    int* status;
    int64_t spin_limit;
    int single;  // per-stage launch: item = item0 + blockIdx.x, no waits
    int item0;
    int withhold_xf;  // fault injection for tests: transform whose first stage never signals (-1: none)
    const int64_t* line_off;  // element offsets of grouped lines (GStage::line_tab)
};

__device__ __forceinline__ int gpad(int a) { return a + (a >> 4); }

// Division by a runtime divisor d (1 <= d < 2^16) of numerators e < 2^16 as
// one multiply-high: q = floor(e * ceil(2^32 / d) / 2^32), exact whenever
// e * d < 2^32 (the rounding error of the reciprocal stays below 1/d).
struct FastDiv {
    uint32_t d, m;
    __device__ __forceinline__ explicit FastDiv(uint32_t dd)
        : d(dd), m(dd > 1 ? (uint32_t)((0x100000000ull + dd - 1) / dd) : 0u) {}
    __device__ __forceinline__ uint32_t div(uint32_t e) const { return d > 1 ? __umulhi(e, m) : e; }
    __device__ __forceinline__ uint32_t mod(uint32_t e) const { return e - div(e) * d; }
};

// Pass p of a tile: every radix-R butterfly of nl lines.  Intermediate passes
// go src -> dst in shared memory; the last pass stores to global memory.
template <int R, bool INV>
__device__ __forceinline__ void g_pass(const GStage& st, const GShape& sh, int p, const float2* __restrict__ pool,
                                       const float2* src, float2* dst, int Lp, int line0, int nl, bool last,
                                       float2* __restrict__ gout, const int64_t* s_loff) {
    const int L = sh.L;
    const int Ns = sh.ns[p];
    const int stride = L / R;  // butterflies per line
    const int nbf = nl * stride;
    const float2* tw = pool + sh.tw[p];
    const bool lf = last && st.out_line_fast;
    const FastDiv by_nl((uint32_t)nl), by_stride((uint32_t)stride), by_ns((uint32_t)Ns);
    for (int bf = threadIdx.x; bf < nbf; bf += blockDim.x) {
        int line, b;
        if (lf) {
            b = (int)by_nl.div((uint32_t)bf);
            line = bf - b * nl;
        } else {
            line = (int)by_stride.div((uint32_t)bf);
            b = bf - line * stride;
        }
        const float2* s = src + line * Lp;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[gpad(b + r * stride)];
        const int k = (int)by_ns.mod((uint32_t)b);
        if (p > 0) {
            const float2* tp = tw + k;  // block [(r-1)*Ns + k] = W_{Ns R}^{k r}
            if constexpr (R == 16) {
                // six loads; the other nine twiddles are one product of two loaded ones
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
        dft<R, 0, 1, INV>(v);
        if (!last) {
            float2* d = dst + line * Lp;
            const int base = (b - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) d[gpad(base + r * Ns)] = v[r];
        } else {
            // natural order: output element k = b + r*stride of line line0+line
            const int aline = line0 + line;
            const int64_t lo_line = st.line_tab >= 0 ? s_loff[line] : (int64_t)aline * st.out_ls;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int kk = b + r * stride;
                const int64_t off = lo_line + (int64_t)kk * st.out_es;
                if (off >= st.out_valid) continue;
                float2 val = v[r];
                if (st.post == G_POST_TW4) {
                    const uint32_t m = (uint32_t)aline * (uint32_t)kk;
                    val = twmul<INV>(val, root2(pool + st.lo, pool + st.hi, m, st.sh));
                } else if (st.post == G_POST_TABLE) {
                    val = cmul(val, __ldg(pool + st.post_tab + off));
                } else if (st.post == G_POST_TABLE_CONJ) {
                    val = cmulc(val, __ldg(pool + st.post_tab + off));
                }
                __stcg(gout + off, val);
            }
        }
    }
}

// One tile: lines [line0, line0 + nl) of a stage.
template <bool INV>
__device__ void g_tile_dir(const GStage& st, const GShape& sh, const float2* __restrict__ pool,
                           const float2* __restrict__ gin, float2* __restrict__ gout, int line0, int nl,
                           float2* smem, const int64_t* __restrict__ line_off) {
    const int L = sh.L;
    const int Lp = gpad(L) + 1;
    float2* bufA = smem;
    float2* bufB = smem + kGBuf;
    // element offsets of the tile's lines when they are separate transforms
    __shared__ int64_t s_loff[kGMaxLines];
    if (st.line_tab >= 0) {
        for (int l = threadIdx.x; l < nl; l += kGThreads) s_loff[l] = __ldg(line_off + st.line_tab + line0 + l);
        __syncthreads();
    }
    // 1. load (coalesced), pre-multiply, zero beyond in_valid; U loads in
    // flight per thread before their shared-memory stores
    const int tot = nl * L;
    const FastDiv by_nl((uint32_t)nl), by_L((uint32_t)L);
#ifndef B300_G_LOADS
#define B300_G_LOADS 8
#endif
    constexpr int U = B300_G_LOADS;
    for (int e0 = threadIdx.x; e0 < tot; e0 += U * kGThreads) {
        float2 v[U];
        int dst[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * kGThreads;
            v[u] = make_float2(0.f, 0.f);
            dst[u] = -1;
            if (e < tot) {
                int line, i;
                if (st.in_line_fast) {
                    i = (int)by_nl.div((uint32_t)e);
                    line = e - i * nl;
                } else {
                    line = (int)by_L.div((uint32_t)e);
                    i = e - line * L;
                }
                const int64_t lb = st.line_tab >= 0 ? s_loff[line] : (int64_t)(line0 + line) * st.in_ls;
                const int64_t off = lb + (int64_t)i * st.in_es;
                dst[u] = line * Lp + gpad(i);
                if (off < st.in_valid) {
                    v[u] = __ldcg(gin + off);
                    if (st.pre == G_PRE_TABLE) v[u] = cmul(v[u], __ldg(pool + st.pre_tab + off));
                    else if (st.pre == G_PRE_TABLE_CONJ) v[u] = cmulc(v[u], __ldg(pool + st.pre_tab + off));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (dst[u] >= 0) bufA[dst[u]] = v[u];
    }
    __syncthreads();
    // 2./3. Stockham passes; the last one stores to global memory
    const float2* src = bufA;
    float2* dst = bufB;
    for (int p = 0; p < sh.npass; ++p) {
        const bool last = p + 1 == sh.npass;
        switch (sh.radix[p]) {
#define B300_G(RR)                                                                    \
    case RR:                                                                          \
        g_pass<RR, INV>(st, sh, p, pool, src, dst, Lp, line0, nl, last, gout, s_loff);   \
        break;
            B300_G(1) B300_G(2) B300_G(3) B300_G(4) B300_G(5) B300_G(7) B300_G(8) B300_G(16)
#undef B300_G
            default:
                break;
        }
        __syncthreads();
        const float2* t = src;
        src = dst;
        dst = const_cast<float2*>(t);
    }
}

__device__ __forceinline__ const float2* g_buf_in(const GExecArgs& a, const GTransform& x, int sel) {
    switch (sel) {
        case G_BUF_IN: return a.in + x.in_off;
        case G_BUF_OUT: return a.out + x.out_off;
        case G_BUF_W1: return a.work + x.w1_off;
        default: return a.work + x.w2_off;
    }
}
__device__ __forceinline__ float2* g_buf_out(const GExecArgs& a, const GTransform& x, int sel) {
    switch (sel) {
        case G_BUF_OUT: return a.out + x.out_off;
        case G_BUF_W1: return a.work + x.w1_off;
        case G_BUF_W2: return a.work + x.w2_off;
        default: return a.out + x.out_off;  // never written
    }
}

// Power-of-two four-step stage of a transform of N = 2^L1 * 2^L2 with the
// register-staged templated tiles of the batched path (256 threads):
// A = C columns with the W_N twiddle into the transform's work buffer,
// B = TPC rows with the transposed store.  Tables: pre_tab = Stockham table
// of 2^L1, post_tab = of 2^L2, lo / hi / sh = two-level W_N table.
template <int L1, int C, int L2, int TPC>
__device__ __forceinline__ void g_fourstep_tile(const GExecArgs& a, const GTransform& x, const GStage& st, int tile,
                                                float2* smem) {
    static_assert(ColsCfg<L1, C>::THREADS == kGThreads && RowsTCfg<L2, TPC>::THREADS == kGThreads,
                  "templated stages run on the executor's 256 threads");
    constexpr int64_t N1 = int64_t(1) << L1, N2 = int64_t(1) << L2;
    const uint64_t pol = l2_policy_evict_last();
    if (st.tmpl & 1) {
        const float2* src = a.work + x.w1_off + (int64_t)tile * TPC * N2;
        float2* dst = a.out + x.out_off + (int64_t)tile * TPC;
        if (st.inv) rowsT_tile<L2, TPC, true, Ld::Cg, St::Stream>(src, dst, N1, a.pool + st.post_tab, smem, pol);
        else rowsT_tile<L2, TPC, false, Ld::Cg, St::Stream>(src, dst, N1, a.pool + st.post_tab, smem, pol);
    } else {
        const int64_t c0 = (int64_t)tile * C;
        const float2* src = a.in + x.in_off + c0;
        float2* dst = a.work + x.w1_off + c0;
        const float2 *lo = a.pool + st.lo, *hi = a.pool + st.hi;
        if (st.inv)
            cols_tile<L1, C, true, true, Ld::Stream, St::Keep>(src, dst, N2, (uint32_t)c0, a.pool + st.pre_tab, lo, hi,
                                                               st.sh, smem, pol);
        else
            cols_tile<L1, C, false, true, Ld::Stream, St::Keep>(src, dst, N2, (uint32_t)c0, a.pool + st.pre_tab, lo,
                                                                hi, st.sh, smem, pol);
    }
}

// Second stage of a mixed-length four-step (N = N1 * 2^L2, N1 = nlines not a
// power of two): TPC rows of 2^L2 with the transposed store, templated.
template <int L2, int TPC>
__device__ __forceinline__ void g_rowsT_stage(const GExecArgs& a, const GTransform& x, const GStage& st, int tile,
                                              float2* smem) {
    static_assert(RowsTCfg<L2, TPC>::THREADS == kGThreads, "256 threads");
    constexpr int64_t N2 = int64_t(1) << L2;
    const uint64_t pol = l2_policy_evict_last();
    const float2* src = a.work + x.w1_off + (int64_t)tile * TPC * N2;
    float2* dst = a.out + x.out_off + (int64_t)tile * TPC;
    if (st.inv) rowsT_tile<L2, TPC, true, Ld::Cg, St::Stream>(src, dst, (int64_t)st.nlines, a.pool + st.post_tab, smem, pol);
    else rowsT_tile<L2, TPC, false, Ld::Cg, St::Stream>(src, dst, (int64_t)st.nlines, a.pool + st.post_tab, smem, pol);
}

// Lines of the compile-time mixed-radix tiles: kGMixLines(L) per tile, the
// element offset of each line in shared memory past the tile's buffer.
__host__ __device__ constexpr int kGMixLines(int L) { return 4096 / L < kGMaxLines ? 4096 / L : kGMaxLines; }
constexpr int kGMixOffF2 = 6144;  // float2 offset of the line-offset table in the dynamic buffer
static_assert(kGMixOffF2 * 8 + kGMaxLines * 8 <= kGSmem, "line offsets fit the executor's shared memory");

template <int L>
struct MixRowsAt {  // line l, element e at base + off[l] + e
    static constexpr bool LOAD_LF = false, STORE_LF = false;
    const float2* in;
    float2* out;
    const int64_t* off;
    __device__ __forceinline__ float2 load(int line, int e) const { return __ldcs(in + off[line] + e); }
    __device__ __forceinline__ void store(int line, int e, float2 v) const { __stcs(out + off[line] + e, v); }
};

// Single-tile stage of lines of M * 2^K (uniform rows or separate transforms):
// line l of the stage starts at line_off[line_tab + l] (line_tab >= 0) or at
// l * ls.  Not inlined: each tile shape gets its own register allocation.
template <int M, int K>
__device__ __noinline__ void g_mixed_rows(const float2* gin, float2* gout, const int64_t* __restrict__ line_off,
                                          int64_t line_tab, int64_t ls, int nlines, int tile, int inv,
                                          const float2* __restrict__ tw, float2* smem) {
    using MP = MixPlan<M, K, kGMixLines(M << K)>;
    static_assert(MP::SMEM <= kGMixOffF2 * 8, "tile buffer below the line-offset table");
    int64_t* s_off = reinterpret_cast<int64_t*>(smem + kGMixOffF2);
    const int line0 = tile * MP::NL;
    const int nl = min(MP::NL, nlines - line0);
    for (int l = threadIdx.x; l < nl; l += kGThreads)
        s_off[l] = line_tab >= 0 ? __ldg(line_off + line_tab + line0 + l) : (int64_t)(line0 + l) * ls;
    __syncthreads();
    const MixRowsAt<MP::L> io{gin, gout, s_off};
    if (inv) mix_pass<MP, 0, true>(io, smem, nl, tw);
    else mix_pass<MP, 0, false>(io, smem, nl, tw);
}

// Four-step first stage of N = (M * 2^A) * S2: NL adjacent columns, W_N twiddle out.
template <int M, int A, int NL>
__device__ __noinline__ void g_mixed_cols(const float2* gin, float2* gout, int64_t S2, int tile, int inv,
                                          const float2* __restrict__ tw, const float2* __restrict__ lo,
                                          const float2* __restrict__ hi, int sh, float2* smem) {
    using MP = MixPlan<M, A, NL>;
    const int64_t col0 = (int64_t)tile * NL;
    if (inv) {
        const MixCols<true> io{gin + col0, gout + col0, S2, (uint32_t)col0, lo, hi, sh};
        mix_pass<MP, 0, true>(io, smem, NL, tw);
    } else {
        const MixCols<false> io{gin + col0, gout + col0, S2, (uint32_t)col0, lo, hi, sh};
        mix_pass<MP, 0, false>(io, smem, NL, tw);
    }
}

// Rows of a four-step's second stage with the transposed store: line l
// (row k1 = line0 + l of the [N1][L] work buffer) is read contiguously (b
// fastest) and its bin e goes to out[k1 + N1 e] (line fastest: runs of up to
// NL consecutive k1).
// Optional table multiply of a stage's loads or stores (Bluestein's chirp and
// filter): v * t[idx] or v * conj(t[idx]) for idx < valid, zero (loads) or
// nothing (stores) beyond.  t == nullptr: no multiply.
struct TabMul {
    const float2* t;
    int conj;
    int64_t valid;
    __device__ __forceinline__ float2 apply(float2 v, int64_t idx) const {
        if (!t) return v;
        const float2 w = __ldg(t + idx);
        return conj ? cmulc(v, w) : cmul(v, w);
    }
};

template <int L>
struct MixRowsT {
    static constexpr bool LOAD_LF = false, STORE_LF = true;
    const float2* in;  // work buffer at row line0
    float2* out;       // output at k1 = line0
    int64_t n1, line0;
    TabMul post;       // bin k = line0 + line + n1 e
    __device__ __forceinline__ float2 load(int line, int e) const { return __ldcg(in + line * L + e); }
    __device__ __forceinline__ void store(int line, int e, float2 v) const {
        const int64_t k = line0 + line + n1 * e;
        if (k < post.valid) __stcs(out + line + n1 * e, post.apply(v, k));
    }
};

template <int K2>
__device__ __noinline__ void g_mixed_rowsT(const float2* gin, float2* gout, int64_t n1, int tile, int inv,
                                           const float2* __restrict__ tw, float2* smem, const float2* post_t,
                                           int post_conj, int64_t post_valid) {
    const TabMul post{post_t, post_conj, post_valid};
    using MP = MixPlan<1, K2, kGMixLines(1 << K2)>;
    static_assert(MP::SMEM <= kGMixOffF2 * 8, "tile buffer below the line-offset table");
    const int64_t line0 = (int64_t)tile * MP::NL;
    const int nl = (int)(n1 - line0 < MP::NL ? n1 - line0 : MP::NL);
    const MixRowsT<MP::L> io{gin + line0 * MP::L, gout + line0, n1, line0, post};
    if (inv) mix_pass<MP, 0, true>(io, smem, nl, tw);
    else mix_pass<MP, 0, false>(io, smem, nl, tw);
}

// Bluestein's single-tile stage: one line of M = 2^K, loads times the pre
// table (zero beyond pre.valid), stores times the post table (up to post.valid).
template <int L>
struct MixLinePP {
    static constexpr bool LOAD_LF = false, STORE_LF = false;
    const float2* in;
    float2* out;
    TabMul pre, post;
    __device__ __forceinline__ float2 load(int, int e) const {
        return e < pre.valid ? pre.apply(__ldcg(in + e), e) : make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void store(int, int e, float2 v) const {
        if (e < post.valid) __stcg(out + e, post.apply(v, e));
    }
};

template <int K>
__device__ __noinline__ void g_blue_rows(const float2* gin, float2* gout, int inv, const float2* __restrict__ tw,
                                         float2* smem, const float2* pre_t, int pre_conj, int64_t pre_valid,
                                         const float2* post_t, int post_conj, int64_t post_valid) {
    const TabMul pre{pre_t, pre_conj, pre_valid}, post{post_t, post_conj, post_valid};
    using MP = MixPlan<1, K, 1>;
    const MixLinePP<MP::L> io{gin, gout, pre, post};
    if (inv) mix_pass<MP, 0, true>(io, smem, 1, tw);
    else mix_pass<MP, 0, false>(io, smem, 1, tw);
}

// Bluestein's four-step first stage: NL adjacent columns of 2^A (stride S2),
// loads times the pre table (element index col + S2 e, zero beyond
// pre.valid), stores times the W_M twiddle into the work buffer.
template <bool INV>
struct MixColsPre {
    static constexpr bool LOAD_LF = true, STORE_LF = true;
    MixCols<INV, true> c;
    TabMul pre;
    __device__ __forceinline__ float2 load(int line, int e) const {
        const int64_t idx = (int64_t)c.col0 + line + c.S2 * e;
        return idx < pre.valid ? pre.apply(c.load(line, e), idx) : make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void store(int line, int e, float2 v) const { c.store(line, e, v); }
};

template <int A, int NL>
__device__ __noinline__ void g_blue_cols(const float2* gin, float2* gout, int64_t S2, int tile, int inv,
                                         const float2* __restrict__ tw, const float2* __restrict__ lo,
                                         const float2* __restrict__ hi, int sh, float2* smem, const float2* pre_t,
                                         int pre_conj, int64_t pre_valid) {
    const TabMul pre{pre_t, pre_conj, pre_valid};
    using MP = MixPlan<1, A, NL>;
    const int64_t col0 = (int64_t)tile * NL;
    if (inv) {
        const MixColsPre<true> io{{gin + col0, gout + col0, S2, (uint32_t)col0, lo, hi, sh}, pre};
        mix_pass<MP, 0, true>(io, smem, NL, tw);
    } else {
        const MixColsPre<false> io{{gin + col0, gout + col0, S2, (uint32_t)col0, lo, hi, sh}, pre};
        mix_pass<MP, 0, false>(io, smem, NL, tw);
    }
}

// Compile-time mixed tiles of the stage graph (the lengths of the batched
// mixed-radix kernels; columns M * 2^A with the same widths).
#define B300_G_MIXED_ROWS(X)                                                                                    \
    X(1, 4) X(1, 5) X(1, 6) X(1, 7) X(1, 8) X(1, 9) X(1, 10) X(1, 11) X(1, 12) X(3, 0) X(3, 1) X(3, 2) X(3, 3) X(3, 4) X(3, 5) X(3, 6) X(3, 7) X(3, 8) X(3, 9) X(3, 10) X(5, 0) X(5, 1)    \
    X(5, 2) X(5, 3) X(5, 4) X(5, 5) X(5, 6) X(5, 7) X(5, 8) X(5, 9) X(7, 0) X(7, 1) X(7, 2) X(7, 3) X(7, 4)     \
    X(7, 5) X(7, 6) X(7, 7) X(7, 8) X(7, 9)
#define B300_G_MIXED_COLS(X)                                                                           \
    X(3, 2, 256) X(3, 3, 128) X(3, 4, 64) X(3, 5, 32) X(3, 6, 16) X(3, 7, 8) X(5, 2, 128) X(5, 3, 64)      \
    X(5, 4, 32) X(5, 5, 16) X(5, 6, 8) X(7, 2, 128) X(7, 3, 64) X(7, 4, 32) X(7, 5, 16) X(7, 6, 8)

__device__ __forceinline__ void g_mixed_tile(const GExecArgs& a, const GTransform& x, const GStage& st, int tile,
                                             float2* smem) {
    const float2* gin = g_buf_in(a, x, st.in_buf);
    float2* gout = g_buf_out(a, x, st.out_buf);
    const float2* tw = a.pool + st.mtab;
    // table multiplies of the loads / stores (Bluestein stages; none elsewhere)
#define B300_PRE (st.pre != G_PRE_NONE ? a.pool + st.pre_tab : nullptr), (int)(st.pre == G_PRE_TABLE_CONJ), st.in_valid
#define B300_POST                                                                                           \
    (st.post == G_POST_TABLE || st.post == G_POST_TABLE_CONJ ? a.pool + st.post_tab : nullptr),            \
        (int)(st.post == G_POST_TABLE_CONJ), st.out_valid
    switch (st.tmpl) {
#define B300_R(M, K)                                                                                          \
    case 1000 + 16 * M + K:                                                                                   \
        g_mixed_rows<M, K>(gin, gout, a.line_off, st.line_tab, st.in_ls, st.nlines, tile, st.inv, tw, smem); \
        break;
        B300_G_MIXED_ROWS(B300_R)
#undef B300_R
#define B300_T(K2)                                                                     \
    case 3000 + K2:                                                                    \
        g_mixed_rowsT<K2>(gin, gout, (int64_t)st.nlines, tile, st.inv, tw, smem, B300_POST); \
        break;
        B300_T(5) B300_T(6) B300_T(7) B300_T(8) B300_T(9) B300_T(10) B300_T(11) B300_T(12)
#undef B300_T
#define B300_B(K)                                                  \
    case 4000 + K:                                                 \
        g_blue_rows<K>(gin, gout, st.inv, tw, smem, B300_PRE, B300_POST); \
        break;
        B300_B(7) B300_B(8) B300_B(9) B300_B(10) B300_B(11) B300_B(12)
#undef B300_B
#define B300_BC(A, NL)                                                                                           \
    case 5000 + A:                                                                                               \
        g_blue_cols<A, NL>(gin, gout, st.in_es, tile, st.inv, tw, a.pool + st.lo, a.pool + st.hi, st.sh, smem,     \
                           B300_PRE);                                                                            \
        break;
        B300_BC(6, 64) B300_BC(7, 32) B300_BC(8, 16) B300_BC(9, 8)
#undef B300_BC
#define B300_C(M, A, NL)                                                                                          \
    case 2000 + 16 * M + A:                                                                                       \
        g_mixed_cols<M, A, NL>(gin, gout, st.in_es, tile, st.inv, tw, a.pool + st.lo, a.pool + st.hi, st.sh, smem); \
        break;
        B300_G_MIXED_COLS(B300_C)
#undef B300_C
        default:
            break;
    }
#undef B300_PRE
#undef B300_POST
}

template <bool MIX>
__device__ __forceinline__ void g_pow2_tile(const GExecArgs& a, const GTransform& x, const GStage& st, int tile,
                                            float2* smem) {
    if constexpr (MIX) {
        if (st.tmpl >= 1000) {
            g_mixed_tile(a, x, st, tile, smem);
            return;
        }
    }
    if (st.tmpl >= 100) {  // 100 + L2: mixed four-step second stage
        switch (st.tmpl - 100) {
            case 7: g_rowsT_stage<7, 32>(a, x, st, tile, smem); break;
            case 8: g_rowsT_stage<8, 16>(a, x, st, tile, smem); break;
            default: break;
        }
        return;
    }
    switch (st.tmpl >> 1) {
        case 13: g_fourstep_tile<6, 64, 7, 32>(a, x, st, tile, smem); break;
        case 14: g_fourstep_tile<7, 32, 7, 32>(a, x, st, tile, smem); break;
        case 15: g_fourstep_tile<7, 32, 8, 16>(a, x, st, tile, smem); break;
        case 16: g_fourstep_tile<8, 16, 8, 16>(a, x, st, tile, smem); break;
        default: break;
    }
}

// Run queue item p (tile of one stage of one transform).  LEAN: the plan has
// templated power-of-two stages only (no runtime tile is compiled in).
template <bool MIX, bool LEAN>
__device__ __forceinline__ void g_run_item(const GExecArgs& a, int p, float2* smem, int* s_ok) {
    const uint64_t it = a.items[p];
    const int t = (int)(it >> 32);
    const int s = (int)((it >> 24) & 0xff);
    const int tile = (int)(it & 0xffffff);
    const GTransform x = a.xf[t];
    const GStage st = a.stages[x.kind + s];
    const GShape sh = a.shapes[st.shape];
    if (s > 0 && !a.single) {
        if (threadIdx.x == 0) {
            const int need = a.stages[x.kind + s - 1].ntiles;
            int ok = 1;
            int64_t spins = 0;
            while (ld_acquire_gpu(a.ctl + 1 + x.ctr + s - 1) < need) {
                if (++spins > a.spin_limit) {
                    ok = 0;
                    atomicCAS(a.status, 0, 6);
                    break;
                }
                __nanosleep(128);
            }
            *s_ok = ok;
        }
        __syncthreads();
        if (!*s_ok) return;
    }
    if (LEAN || st.tmpl) {
        g_pow2_tile<MIX>(a, x, st, tile, smem);
    } else if constexpr (!LEAN) {
        const int line0 = tile * st.lpt;
        const int nl = min(st.lpt, st.nlines - line0);
        const float2* gin = g_buf_in(a, x, st.in_buf);
        float2* gout = g_buf_out(a, x, st.out_buf);
        if (st.inv) g_tile_dir<true>(st, sh, a.pool, gin, gout, line0, nl, smem, a.line_off);
        else g_tile_dir<false>(st, sh, a.pool, gin, gout, line0, nl, smem, a.line_off);
    }
    if (s + 1 < x.nstages && !a.single) {
        __syncthreads();
        if (threadIdx.x == 0 && !(s == 0 && t == a.withhold_xf)) {
            __threadfence();
            atomicAdd(a.ctl + 1 + x.ctr + s, 1);
        }
    }
}

// Shared memory of the templated power-of-two tiles (the lean executor's buffer).
constexpr int cmax(int x, int y) { return x > y ? x : y; }
constexpr int kGSmemLean =
    cmax(cmax(cmax(ColsCfg<6, 64>::SMEM, ColsCfg<7, 32>::SMEM), cmax(ColsCfg<8, 16>::SMEM, RowsTCfg<7, 32>::SMEM)),
         RowsTCfg<8, 16>::SMEM);

// The lean executor with the compile-time mixed tiles: their buffer and line offsets.
constexpr int kGSmemLeanMix = cmax(kGSmemLean, kGMixOffF2 * 8 + kGMaxLines * 8);

// Persistent executor (single = 0) or one launch per stage group (single = 1:
// block b runs item item0 + b; the stream orders the stages).  MIX: the plan
// has compile-time mixed-radix stages (a separate kernel, so plans without
// them keep the smaller kernel's register allocation).
template <bool MIX, bool LEAN>
__global__ void __launch_bounds__(kGThreads, LEAN ? 4 : 3) k_gexec(GExecArgs a) {
    extern __shared__ float2 smem[];
    __shared__ int s_item[2];
    __shared__ int s_ok;
    if (a.single) {
        g_run_item<MIX, LEAN>(a, a.item0 + blockIdx.x, smem, &s_ok);
        return;
    }
    if (threadIdx.x == 0) s_item[0] = atomicAdd(a.qhead, 1);
    for (int it = 0;; it ^= 1) {
        __syncthreads();
        const int p = s_item[it];
        if (p >= a.nitems) break;
        if (threadIdx.x == 0) s_item[it ^ 1] = atomicAdd(a.qhead, 1);
        g_run_item<MIX, LEAN>(a, p, smem, &s_ok);
    }
}

}  // namespace b300fft
