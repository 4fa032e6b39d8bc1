// pipe3.cuh -- the persistent three-stage transform (threestep.cuh: the
// four-step split of Sec. III-A applied twice, N = N1 * M1 * M2) with its
// tile loads made asynchronous, as pipe.cuh does for the two-pass kernel.
//
// One producer warp per CTA dequeues items in threestep.cuh's queue order,
// waits (bounded) for a B1 item's chunk or a B2 item's row group, and has
// the tensor memory accelerator copy the item's 4096-point tile into a free
// slot of a ring of NS shared-memory slots:
//   A   CA adjacent columns of N1 rows of the input (row stride N2): a 2-D
//       box {CA, N1} of the input viewed as [batch * N1][N2];
//   B1  CB adjacent columns of M1 rows inside workspace row k1 (row stride
//       M2): a 2-D box {CB, M1} of the workspace viewed as [rows][M2];
//   B2  TPC consecutive rows k1 at one j1 (M2 points each, row stride N2):
//       a 3-D box {M2, 1, TPC} of the workspace viewed as
//       [batch * N1][M1][M2].
// The consumer warps (256 threads) read their 16 registers from the slot,
// run the stage's Stockham passes with the slot as the exchange buffer and
// store from registers, then release the slot and publish the tile (A:
// chunk counter, B1: row-group counter).  All waits are bounded.  Opt-in
// (B300FFT_PIPE=2|3, or the autotuner's pick): the plain three-stage kernel
// measured faster at every size on a B300.
#pragma once
#include "threestep.cuh"
#include "tma.cuh"

namespace b300fft {

template <int LA, int LB1, int LB2, int NS>
struct Three3Cfg {
    using TC = ThreeCfg<LA, LB1, LB2>;
    static constexpr int THREADS = 256, CTA_THREADS = 288, TILE = 4096;
    // a slot holds a stage's padded exchange buffer (or the dense tile); the
    // twiddle steps of the column stages live after the slots
    static constexpr int X0 = ColsCfg<LA, TC::CA>::XBUF * 8, X1 = ColsCfg<LB1, TC::CB>::XBUF * 8, X2 = TC::S2;
    static constexpr int S0 = X0 > X1 ? (X0 > X2 ? X0 : X2) : (X1 > X2 ? X1 : X2);
    static constexpr int SLOT = ((S0 > TILE * 8 ? S0 : TILE * 8) + 1023) / 1024 * 1024;
    static constexpr int STEPS = (TC::CA > TC::CB ? TC::CA : TC::CB) * 16 * 8;
    static constexpr int SMEM = NS * SLOT + STEPS + 1024;
    static constexpr int MINB = 233472 / (SMEM + 1024) > 0 ? 233472 / (SMEM + 1024) : 1;
};

template <int LA, int LB1, int LB2, int NS, bool INV>
__global__ void __launch_bounds__(288, Three3Cfg<LA, LB1, LB2, NS>::MINB)
k_threestep_pipe(const __grid_constant__ CUtensorMap t_in, const __grid_constant__ CUtensorMap t_b1,
                 const __grid_constant__ CUtensorMap t_b2, ThreeArgs a) {
    using CF = ThreeCfg<LA, LB1, LB2>;
    using PC = Three3Cfg<LA, LB1, LB2, NS>;
    constexpr int CA = CF::CA, CB = CF::CB, TPC = CF::TPC;
    constexpr int64_t N1 = CF::N1, M1 = CF::M1, M2 = CF::M2, N2 = CF::N2, N = CF::N;
    constexpr int TA = (int)(N1 / 16), TB = (int)(M1 / 16), TCc = (int)(M2 / 16);
    constexpr int GA = (int)(N2 / CA);    // A tiles per transform
    constexpr int HB = (int)(M2 / CB);    // B1 tiles per row
    constexpr int GPT = (int)(N1 / TPC);  // groups per transform
    constexpr int T = PC::THREADS;
    extern __shared__ unsigned char smem_raw[];
    float2* const slots =
        reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[NS], empty[NS];
    __shared__ int info[NS];  // item; -1 end of queue; <= -2 skipped item -(p + 2)
    const int total = a.nch * (a.na + a.nb);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (threadIdx.x >= T) {  // ---- producer
        if (threadIdx.x != T) return;
        prefetch_tensormap(&t_in);
        prefetch_tensormap(&t_b1);
        prefetch_tensormap(&t_b2);
        const uint64_t pol_in = l2_policy_evict_first();
        const uint64_t pol_w = l2_policy_evict_last();
        // the next item is dequeued one item ahead, so the atomic's latency
        // hides behind the wait for a free slot and the copies of this item
        int p_next = atomicAdd(a.ctl, 1);
        for (int i = 0;; ++i) {
            const int s = i % NS;
            const uint32_t ph = (uint32_t)(i / NS) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u, a.spin_limit)) {
                atomicCAS(a.status, 0, 6);
                return;
            }
            const int p = p_next;
            if (p < total) p_next = atomicAdd(a.ctl, 1);
            int inf = p < total ? p : -1;
            int stage = 0, c = 0, g = 0, r = 0;
            bool load = false;
            int64_t tr = 0;
            if (inf >= 0) {
                three_decode(a, p, &stage, &c, &g, &r);
                tr = (int64_t)c * a.cb + (stage == kStageA ? r / GA : g / GPT);
                load = tr < a.batch;
                if (stage != kStageA && load) {
                    int target = 0;
                    const int* dep = three_dep(a, stage, c, g, &target);
                    int64_t spins = 0;
                    while (ld_acquire_gpu(dep) < target) {
                        if (++spins > a.spin_limit) {
                            atomicCAS(a.status, 0, 6);
                            load = false;
                            inf = -(p + 2);
                            break;
                        }
                        __nanosleep(64);
                    }
                    if (load) fence_proxy_async_global();
                }
            }
            info[s] = inf;
            float2* slot = slots + s * (PC::SLOT / 8);
            if (load) {
                mbar_arrive_expect_tx(&full[s], PC::TILE * 8);
                if (stage == kStageA) {
                    tma_load_2d(slot, &t_in, (r % GA) * CA, (int)(tr * N1), &full[s], pol_in);
                } else if (stage == kStageB1) {
                    const int64_t k1 = (int64_t)(g % GPT) * TPC + r / HB;
                    tma_load_2d(slot, &t_b1, (r % HB) * CB, (int)((tr * N1 + k1) * M1), &full[s], pol_w);
                } else {
                    const int64_t k10 = (int64_t)(g % GPT) * TPC;
                    tma_load_3d(slot, &t_b2, 0, r, (int)(tr * N1 + k10), &full[s], pol_w);
                }
            } else {
                mbar_arrive(&full[s]);
            }
            if (inf == -1) return;
        }
    }

    // ---- consumers
    const uint64_t pol = l2_policy_evict_last();
    for (int i = 0;; ++i) {
        const int s = i % NS;
        const uint32_t ph = (uint32_t)(i / NS) & 1u;
        const bool got = mbar_wait(&full[s], ph, 4 * a.spin_limit);
        const int inf = info[s];
        int p = inf >= 0 ? inf : (inf <= -2 ? -(inf + 2) : 0);
        if (p >= total) p = 0;  // only after a wait that ran out
        float2* slot = slots + s * (PC::SLOT / 8);
        int stage, c, g, r;
        three_decode(a, p, &stage, &c, &g, &r);
        const int64_t tr = (int64_t)c * a.cb + (stage == kStageA ? r / GA : g / GPT);
        const bool run = inf >= 0 && tr < a.batch;
        float2 v[16];
        if (run) {
            if (stage == kStageA) {
                const int cc = threadIdx.x % CA, t = threadIdx.x / CA;
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = slot[(t + q * TA) * CA + cc];
            } else if (stage == kStageB1) {
                const int cc = threadIdx.x % CB, t = threadIdx.x / CB;
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = slot[(t + q * TB) * CB + cc];
            } else {
                const int sub = threadIdx.x / TCc, t = threadIdx.x % TCc;
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = slot[sub * M2 + t + q * TCc];
            }
        }
        if (!tile_and<T>(got)) {  // every dense read done; all consumers agree to go on
            if (threadIdx.x == 0) atomicCAS(a.status, 0, 6);
            break;
        }
        if (inf == -1) break;
        if (stage == kStageA) {
            const uint32_t col0 = (uint32_t)((r % GA) * CA);
            if (run)
                cols_tile_regs<LA, CA, INV, true, St::Keep, T>(v, a.work + tr * N + col0, N2, col0, a.tw_a, a.lo, a.hi,
                                                               a.sh, slot, pol, 1, slots + NS * (PC::SLOT / 8));
            fence_proxy_async_smem();
            tile_sync<T>();
            if (threadIdx.x == 0) {
                mbar_arrive(&empty[s]);
                if (c != a.withhold_chunk) {
                    __threadfence();
                    atomicAdd(a.ctl + 1 + c, 1);
                }
            }
        } else if (stage == kStageB1) {
            const int64_t k1 = (int64_t)(g % GPT) * TPC + r / HB;
            const uint32_t col0 = (uint32_t)((r % HB) * CB);
            if (run)
                cols_tile_regs<LB1, CB, INV, true, St::Keep, T>(v, a.work + tr * N + k1 * N2 + col0, M2, col0, a.tw_b1,
                                                                a.lo, a.hi, a.sh, slot, pol, (uint32_t)N1,
                                                                slots + NS * (PC::SLOT / 8));
            fence_proxy_async_smem();
            tile_sync<T>();
            if (threadIdx.x == 0) {
                mbar_arrive(&empty[s]);
                __threadfence();
                atomicAdd(a.ctl + 1 + a.nch + c * a.G + g, 1);
            }
        } else {
            const int64_t k10 = (int64_t)(g % GPT) * TPC;
            if (run)
                rowsT_tile_regs<LB2, TPC, INV, St::Stream, T>(v, a.out + tr * N + k10 + N1 * r, N1 * M1, a.tw_b2, slot,
                                                              pol);
            fence_proxy_async_smem();
            tile_sync<T>();
            if (threadIdx.x == 0) mbar_arrive(&empty[s]);
            if (run) {  // the tile's input rows are consumed: drop them from L2
                const char* base = reinterpret_cast<const char*>(a.work + tr * N + k10 * N2 + (int64_t)r * M2);
                for (int l = threadIdx.x; l < TPC * CF::RUN_LINES; l += T)
                    l2_discard_line(base + (int64_t)(l / CF::RUN_LINES) * N2 * 8 + (int64_t)(l % CF::RUN_LINES) * 128);
            }
        }
    }
}

}  // namespace b300fft
