// threestep.cuh -- persistent three-stage power-of-two FFT for long lengths:
// the four-step split N = N1 * N2 (Sec. III-A, Cooley-Tukey) applied twice,
// N2 = M1 * M2, so every stage works on short transforms (2^6 .. 2^8 points)
// and every tile reads and writes at least 128 contiguous bytes per row.
//
// Input x[n1*N2 + n2]; k = k1 + N1*(j1 + M1*j2) in the output.
//   A  (per column n2):       y[k1][n2] = W_N^{n2 k1} * sum_n1 x[n1 N2 + n2] W_N1^{n1 k1}
//   B1 (per row k1, col m2):  z[k1][j1 M2 + m2] = W_N2^{m2 j1} * sum_m1 y[k1][m1 M2 + m2] W_M1^{m1 j1}
//   B2 (per row k1, j1):      X[k1 + N1 (j1 + M1 j2)] = sum_m2 z[k1][j1 M2 + m2] W_M2^{m2 j2}
// (the second line is the four-step of the length-N2 transform of row k1).
//
// Tiles hold TILE = 4096 points on 256 threads or 16384 points on 1024
// threads (16 complex registers each):
//   A  : CA = TILE / N1 adjacent columns n2 of one transform (stride N2);
//   B1 : CB = TILE / M1 adjacent columns m2 of one row k1 (stride M2), in place;
//   B2 : TPC = TILE / M2 consecutive rows k1 at one j1 (row stride N2); the
//        output is written TPC consecutive k1 (>= 128 bytes) at a time.
// A "group" is TPC consecutive rows k1 of one transform: its B2 tiles need
// exactly its B1 tiles.  Queue order per chunk of transforms follows the
// persistent four-step (A tiles of chunk c+1 before the B tiles of chunk c);
// inside a chunk's B tiles the B1 stage runs D groups ahead of B2:
//     B1(0..D-1), [B1(D), B2(0)], [B1(D+1), B2(1)], ..., B2(G-D..G-1)
// D is chosen so that the tiles between a B1 tile and the first B2 tile that
// needs it outnumber the CTAs in flight (B2 tiles then rarely wait), while
// the D groups of B1 output still fit in L2 when B2 reads them back.
// Dependencies use counters with acquire/release and bounded waits, exactly
// as in persist.cuh (signals are published before any wait; an expired wait
// sets FFT_ERR_TIMEOUT and skips the tile).
#pragma once
#include "persist.cuh"
#include "tma.cuh"

namespace b300fft {

struct ThreeArgs {
    const float2* in;
    float2* out;
    float2* work;
    int* ctl;     // [0] queue head, [1 + c] A tiles done in chunk c, [1 + nch + c*G + g] B1 tiles done in group g
    int* status;  // plan status word
    int64_t batch;
    int64_t cb;  // transforms per chunk
    int nch;     // chunks
    int na, nb;  // A tiles and B tiles (B1 + B2) per chunk
    int G;       // groups per chunk
    int nb1g, nb2g;  // B1 and B2 tiles per group
    int D;           // B1 lookahead in groups (1 <= D <= G)
    const float2* tw_a;
    const float2* tw_b1;
    const float2* tw_b2;
    const float2* lo;  // two-level table of W_N
    const float2* hi;
    int sh;
    int64_t spin_limit;
    int withhold_chunk;
    int prefetch;  // 1: thread 0 brings the next A or B1 tile's box into L2 with one tensor prefetch
};

template <int LA, int LB1, int LB2, int TILE_ = 4096>
struct ThreeCfg {
    static constexpr int TILE = TILE_, THREADS = TILE_ / 16;
    static constexpr int CA = TILE >> LA, CB = TILE >> LB1, TPC = TILE >> LB2;
    static constexpr int64_t N1 = int64_t(1) << LA, M1 = int64_t(1) << LB1, M2 = int64_t(1) << LB2;
    static constexpr int64_t N2 = M1 * M2, N = N1 * N2;
    static_assert(LA >= 6 && LA <= 8 && LB1 >= 6 && LB1 <= 8 && LB2 >= 6 && LB2 <= 8, "stage lengths 2^6 .. 2^8");
    static_assert(CA <= N2 && CB <= M2 && TPC <= N1, "tile wider than its matrix");
    static_assert(ColsCfg<LA, CA>::THREADS == THREADS && ColsCfg<LB1, CB>::THREADS == THREADS &&
                      RowsTCfg<LB2, TPC>::THREADS == THREADS,
                  "all stages use the same thread count");
    static constexpr int S0 = ColsCfg<LA, CA>::SMEM, S1 = ColsCfg<LB1, CB>::SMEM, S2 = RowsTCfg<LB2, TPC>::SMEM;
    static constexpr int SMEM = S0 > S1 ? (S0 > S2 ? S0 : S2) : (S1 > S2 ? S1 : S2);
    static constexpr int RUN_LINES = (int)(M2 * 8 / 128);  // 128-byte lines of one B2 input row
};

enum : int { kStageA = 0, kStageB1 = 1, kStageB2 = 2 };

// Queue position -> (stage, chunk c, group g, tile r within the stage unit).
// Host-callable too (queue-order checks without a GPU).
__host__ __device__ __forceinline__ void three_decode(const ThreeArgs& a, int p, int* stage, int* c, int* g, int* r) {
    bool is_b;
    int rr;
    decode_item(p, a.na, a.nb, a.nch, &is_b, c, &rr);
    if (!is_b) {
        *stage = kStageA;
        *g = 0;
        *r = rr;
        return;
    }
    const int first = a.D * a.nb1g, per = a.nb1g + a.nb2g, mid = (a.G - a.D) * per;
    if (rr < first) {
        *stage = kStageB1;
        *g = rr / a.nb1g;
        *r = rr - *g * a.nb1g;
    } else if (rr - first < mid) {
        const int q = rr - first, blk = q / per, t = q - blk * per;
        if (t < a.nb1g) {
            *stage = kStageB1;
            *g = blk + a.D;
            *r = t;
        } else {
            *stage = kStageB2;
            *g = blk;
            *r = t - a.nb1g;
        }
    } else {
        const int q = rr - first - mid;
        *stage = kStageB2;
        *g = a.G - a.D + q / a.nb2g;
        *r = q % a.nb2g;
    }
}

// The counter (and its target) a tile of `stage` waits for; null for A tiles.
__device__ __forceinline__ const int* three_dep(const ThreeArgs& a, int stage, int c, int g, int* target) {
    if (stage == kStageB1) {
        *target = a.na;
        return a.ctl + 1 + c;
    }
    if (stage == kStageB2) {
        *target = a.nb1g;
        return a.ctl + 1 + a.nch + c * a.G + g;
    }
    return nullptr;
}

__device__ __forceinline__ int three_wait(const ThreeArgs& a, const int* dep, int target) {
    int64_t spins = 0;
    while (ld_acquire_gpu(dep) < target) {
        if (++spins > a.spin_limit) {
            atomicCAS(a.status, 0, 6);
            return 0;
        }
        __nanosleep(128);
    }
    return 1;
}

// One CTA per queue item at a time: the next item is dequeued at the tile
// start, a B tile waits (bounded) for its producers before loading, and a
// producing tile is signalled (and a B2 tile's input lines dropped) right
// after the next loop barrier -- before this CTA can wait on anything.
// Prefetch into L2 the box the tile of queue item p will load (A: the
// input columns, B1: the workspace columns of one row); B2 rows are left to
// the L2 residency of the B1 output.
template <int LA, int LB1, int LB2, int TILE>
__device__ __forceinline__ void three_prefetch(const ThreeArgs& a, int p, const CUtensorMap* t_in,
                                               const CUtensorMap* t_b1) {
    using CF = ThreeCfg<LA, LB1, LB2, TILE>;
    constexpr int GA = (int)(CF::N2 / CF::CA), HB = (int)(CF::M2 / CF::CB), GPT = (int)(CF::N1 / CF::TPC);
    int stage, c, g, r;
    three_decode(a, p, &stage, &c, &g, &r);
    if (stage == kStageA) {
        const int64_t tr = (int64_t)c * a.cb + r / GA;
        if (tr < a.batch) tma_prefetch_2d(t_in, (r % GA) * CF::CA, (int)(tr * CF::N1));
    } else if (stage == kStageB1) {
        const int64_t tr = (int64_t)c * a.cb + g / GPT;
        const int64_t k1 = (int64_t)(g % GPT) * CF::TPC + r / HB;
        if (tr < a.batch) tma_prefetch_2d(t_b1, (r % HB) * CF::CB, (int)((tr * CF::N1 + k1) * CF::M1));
    }
}

template <int LA, int LB1, int LB2, bool INV, int TILE = 4096>
__global__ void __launch_bounds__(TILE / 16, 16384 / TILE)
k_threestep(ThreeArgs a, const __grid_constant__ CUtensorMap t_in, const __grid_constant__ CUtensorMap t_b1) {
    using CF = ThreeCfg<LA, LB1, LB2, TILE>;
    constexpr int CA = CF::CA, CB = CF::CB, TPC = CF::TPC;
    constexpr int64_t N1 = CF::N1, M1 = CF::M1, M2 = CF::M2, N2 = CF::N2, N = CF::N;
    constexpr int TA = (int)(N1 / 16), TB = (int)(M1 / 16), TC = (int)(M2 / 16);  // threads per transform
    constexpr int GA = (int)(N2 / CA);    // A tiles per transform
    constexpr int HB = (int)(M2 / CB);    // B1 tiles per row
    constexpr int GPT = (int)(N1 / TPC);  // groups per transform
    extern __shared__ float2 smem[];
    __shared__ int s_item[2], s_ok;
    const uint64_t pol = l2_policy_evict_last();
    const int total = a.nch * (a.na + a.nb);
    // thread 0: the next queue item (an atomic in flight) and the counter of
    // the previous producing tile still to be signalled (index into ctl, -1:
    // none).  Both are published only after thread 0 has issued its loads of
    // the current tile (or, for a tile that waits, before the wait), so their
    // latency does not delay the tile and no CTA waits on its own signal.
    int nxt = 0, pend = -1;
    const char* drop = nullptr;  // first input row of the previous B2 tile, dropped after the loop barrier
    if (threadIdx.x == 0) s_item[0] = atomicAdd(a.ctl, 1);
    for (int it = 0;; it ^= 1) {
        __syncthreads();  // the previous tile's stores and reads are done
        if (drop) {
            for (int l = threadIdx.x; l < TPC * CF::RUN_LINES; l += CF::THREADS)
                l2_discard_line(drop + (int64_t)(l / CF::RUN_LINES) * N2 * 8 + (int64_t)(l % CF::RUN_LINES) * 128);
            drop = nullptr;
        }
        const int p = s_item[it];
        if (p >= total) break;
        if (threadIdx.x == 0) nxt = atomicAdd(a.ctl, 1);
        int stage, c, g, r;
        three_decode(a, p, &stage, &c, &g, &r);
        if (stage == kStageA) {
            const int64_t tr = (int64_t)c * a.cb + r / GA;
            const uint32_t col0 = (uint32_t)((r % GA) * CA);
            if (tr < a.batch) {
                const float2* src = a.in + tr * N + col0 + threadIdx.x % CA;
                const int t = threadIdx.x / CA;
                float2 v[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = __ldcs(src + (int64_t)(t + i * TA) * N2);
                if (threadIdx.x == 0) {
                    st_shared_after(&s_item[it ^ 1], nxt);
                    if (a.prefetch && nxt < total) three_prefetch<LA, LB1, LB2, TILE>(a, nxt, &t_in, &t_b1);
                    if (pend >= 0) {  // release: the previous tile's stores precede it (loop barrier)
                        __threadfence();
                        atomicAdd(a.ctl + pend, 1);
                        pend = -1;
                    }
                }
                cols_tile_regs<LA, CA, INV, true, St::Keep>(v, a.work + tr * N + col0, N2, col0, a.tw_a, a.lo, a.hi,
                                                            a.sh, smem, pol);
            } else if (threadIdx.x == 0) {
                st_shared_after(&s_item[it ^ 1], nxt);
                if (pend >= 0) {
                    __threadfence();
                    atomicAdd(a.ctl + pend, 1);
                    pend = -1;
                }
            }
            if (threadIdx.x == 0 && c != a.withhold_chunk) pend = 1 + c;
            continue;
        }
        if (threadIdx.x == 0) {
            if (pend >= 0) {  // before waiting: a pending signal may be what the wait needs
                __threadfence();
                atomicAdd(a.ctl + pend, 1);
                pend = -1;
            }
            int target = 0;
            const int* dep = three_dep(a, stage, c, g, &target);
            s_ok = three_wait(a, dep, target);
            st_shared_after(&s_item[it ^ 1], nxt);
            if (a.prefetch && nxt < total) three_prefetch<LA, LB1, LB2, TILE>(a, nxt, &t_in, &t_b1);
        }
        __syncthreads();
        const bool ok = s_ok;
        const int64_t tr = (int64_t)c * a.cb + g / GPT;
        const int64_t k10 = (int64_t)(g % GPT) * TPC;
        if (stage == kStageB1) {
            const int64_t k1 = k10 + r / HB;
            const uint32_t col0 = (uint32_t)((r % HB) * CB);
            float2* base = a.work + tr * N + k1 * N2 + col0;
            if (ok && tr < a.batch) {
                const float2* src = base + threadIdx.x % CB;
                const int t = threadIdx.x / CB;
                float2 v[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = __ldcg(src + (int64_t)(t + i * TB) * M2);
                cols_tile_regs<LB1, CB, INV, true, St::Keep>(v, base, M2, col0, a.tw_b1, a.lo, a.hi, a.sh, smem, pol,
                                                             (uint32_t)N1);
            }
            if (threadIdx.x == 0) pend = 1 + a.nch + c * a.G + g;
        } else if (ok && tr < a.batch) {
            const float2* base = a.work + tr * N + k10 * N2 + (int64_t)r * M2;
            const float2* src = base + (int64_t)(threadIdx.x / TC) * N2 + (threadIdx.x & (TC - 1));
            float2 v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = __ldcg(src + i * TC);
            rowsT_tile_regs<LB2, TPC, INV, St::Stream>(v, a.out + tr * N + k10 + N1 * r, N1 * M1, a.tw_b2, smem, pol);
            drop = reinterpret_cast<const char*>(base);
        }
    }
    if (threadIdx.x == 0 && pend >= 0) {
        __threadfence();
        atomicAdd(a.ctl + pend, 1);
    }
}

}  // namespace b300fft
