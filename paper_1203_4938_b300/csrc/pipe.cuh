// pipe.cuh -- the persistent four-step (persist.cuh: both passes of
// N = N1 * N2, Sec. III-A's Cooley-Tukey split, in one launch with
// L2-resident chunks) with its tile loads made asynchronous.
//
// Each CTA is one producer warp plus the consumer warps of one tile.  The
// producer (one thread) dequeues work items from the same atomic queue as
// persist.cuh, waits (bounded) for a second-pass item's chunk, and has the
// tensor memory accelerator copy the item's whole tile into a free slot of a
// ring of NS shared-memory slots:
//   first pass   C adjacent columns of N1 rows (row stride N2): tiled 2-D
//                tensor copies of C x min(N1, 256) boxes;
//   second pass  TPC consecutive workspace rows of N2 points: contiguous bulk
//                copies.
// Completion is tracked by one mbarrier per slot ("full"); the consumers
// release a slot through a second mbarrier ("empty").  The consumer warps
// read their registers from the slot, run the same register-staged Stockham
// passes as the other kernels with the slot itself as the padded exchange
// buffer (barriers over the consumer threads only), and store the results
// from registers.  Loads of the next items therefore run while the current
// tile computes, instead of every tile's warps waiting for their own global
// loads at the start of the tile.
//
// Selected with B300FFT_PIPE=2|3 (or by the autotuner): on a B300 the plain
// persistent kernel measured 10-40 % faster at every size, because the slots
// leave room for two CTAs (18 warps) per SM instead of four.
//
// Ordering: a first-pass tile's stores are published by bar + fence + atomic
// increment of the chunk counter (as in persist.cuh); the producer acquires
// the counter and issues a proxy fence before its copies read the workspace.
// Consumers fence their generic shared-memory accesses to the async proxy
// before releasing a slot.  All waits are bounded (FFT_ERR_TIMEOUT).
#pragma once
#include "persist.cuh"
#include "tma.cuh"

namespace b300fft {

template <int L1, int C, int L2, int TPC, int NS>
struct PipeCfg {
    static constexpr int THREADS = ColsCfg<L1, C>::THREADS;  // consumer threads
    static_assert(THREADS == RowsTCfg<L2, TPC>::THREADS, "tile shapes must use the same thread count");
    static constexpr int TILE = C << L1;
    static_assert(TILE == (TPC << L2), "both passes move the same number of points per tile");
    static constexpr int CTA_THREADS = THREADS + 32;
    // a slot: the first pass's padded exchange buffer, the second pass's, or
    // the dense tile, whichever is largest; the twiddle steps of a first-pass
    // tile live after the slots
    static constexpr int S0 = ColsCfg<L1, C>::XBUF * 8, S1 = RowsTCfg<L2, TPC>::SMEM, S2 = TILE * 8;
    static constexpr int SLOT = ((S0 > S1 ? (S0 > S2 ? S0 : S2) : (S1 > S2 ? S1 : S2)) + 1023) / 1024 * 1024;
    static constexpr int STEPS = C * 16 * 8;
    static constexpr int SMEM = NS * SLOT + STEPS + 1024;  // + alignment slack of the dynamic buffer
    static constexpr int MINB = 233472 / (SMEM + 1024) > 0 ? 233472 / (SMEM + 1024) : 1;
    static constexpr int BOX_ROWS = (1 << L1) < 256 ? (1 << L1) : 256;
    static constexpr int NBOX = (1 << L1) / BOX_ROWS;
    static constexpr int BULK_PARTS = 4;  // second-pass tile = 4 contiguous bulk copies
    static_assert(C * 8 % 16 == 0 && (TILE * 8 / BULK_PARTS) % 16 == 0, "copy sizes must be multiples of 16 bytes");
};

template <int L1, int C, int L2, int TPC, int NS, bool INV>
__global__ void __launch_bounds__(PipeCfg<L1, C, L2, TPC, NS>::CTA_THREADS, PipeCfg<L1, C, L2, TPC, NS>::MINB)
k_fourstep_pipe(const __grid_constant__ CUtensorMap tin, PersistArgs a) {
    using CF = PipeCfg<L1, C, L2, TPC, NS>;
    constexpr int64_t N1 = int64_t(1) << L1, N2 = int64_t(1) << L2, N = N1 * N2;
    constexpr int GA = (int)(N2 / C);    // first-pass tiles per transform
    constexpr int GB = (int)(N1 / TPC);  // second-pass tiles per transform
    constexpr int T = CF::THREADS;
    constexpr int TA = (int)(N1 / 16), TB = (int)(N2 / 16);  // threads per column / per row
    extern __shared__ unsigned char smem_raw[];
    float2* const slots =
        reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[NS], empty[NS];
    __shared__ int info[NS];  // item of the slot; -1: end of the queue; <= -2: skipped item -(p + 2)
    const int total = a.nch * (a.na + a.nb);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (threadIdx.x >= T) {  // ---- producer warp: one thread issues every copy
        if (threadIdx.x != T) return;
        prefetch_tensormap(&tin);
        const uint64_t pol_in = l2_policy_evict_first();
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
            int64_t tr = 0;
            int j = 0, r = 0;
            bool is_b = false, load = false;
            if (inf >= 0) {
                decode_item(p, a.na, a.nb, a.nch, &is_b, &j, &r);
                tr = (int64_t)j * a.cb + (is_b ? r / GB : r / GA);
                load = tr < a.batch;
                if (is_b && load) {
                    int64_t spins = 0;
                    while (ld_acquire_gpu(a.ctl + 1 + j) < a.na) {
                        if (++spins > a.spin_limit) {
                            atomicCAS(a.status, 0, 6);
                            load = false;
                            inf = -(p + 2);
                            break;
                        }
                        __nanosleep(128);
                    }
                    if (load) fence_proxy_async_global();
                }
            }
            info[s] = inf;
            float2* slot = slots + s * (CF::SLOT / 8);
            if (load) {
                mbar_arrive_expect_tx(&full[s], CF::TILE * 8);
                if (!is_b) {
                    const int x = (r % GA) * C;
#pragma unroll
                    for (int b = 0; b < CF::NBOX; ++b)
                        tma_load_2d(slot + b * CF::BOX_ROWS * C, &tin, x, (int)(tr * N1) + b * CF::BOX_ROWS, &full[s],
                                    pol_in);
                } else {
                    const float2* src = a.work + tr * N + (int64_t)(r % GB) * TPC * N2;
                    constexpr int PART = CF::TILE / CF::BULK_PARTS;
#pragma unroll
                    for (int b = 0; b < CF::BULK_PARTS; ++b)
                        bulk_load(slot + b * PART, src + b * PART, PART * 8, &full[s]);
                }
            } else {
                mbar_arrive(&full[s]);
            }
            if (inf == -1) return;
        }
    }

    // ---- consumer warps
    const uint64_t pol = l2_policy_evict_last();
    for (int i = 0;; ++i) {
        const int s = i % NS;
        const uint32_t ph = (uint32_t)(i / NS) & 1u;
        const bool got = mbar_wait(&full[s], ph, 4 * a.spin_limit);
        // Everything up to the barrier below reads only the slot and the
        // item number, so a thread whose wait ran out does no harm before
        // all consumers agree (barrier with AND reduction) to stop.
        const int inf = info[s];
        int p = inf >= 0 ? inf : (inf <= -2 ? -(inf + 2) : 0);
        if (p >= total) p = 0;  // only after a wait that ran out
        float2* slot = slots + s * (CF::SLOT / 8);
        bool is_b;
        int j, r;
        decode_item(p, a.na, a.nb, a.nch, &is_b, &j, &r);
        const int64_t tr = (int64_t)j * a.cb + (is_b ? r / GB : r / GA);
        const bool run = inf >= 0 && tr < a.batch;
        float2 v[16];
        if (run) {
            if (!is_b) {
                const int c = threadIdx.x % C, t = threadIdx.x / C;
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = slot[(t + q * TA) * C + c];
            } else {
                const int sub = threadIdx.x / TB, t = threadIdx.x % TB;
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = slot[sub * N2 + t + q * TB];
            }
        }
        // every dense read done before the slot becomes the exchange buffer
        if (!tile_and<T>(got)) {
            if (threadIdx.x == 0) atomicCAS(a.status, 0, 6);
            break;
        }
        if (inf == -1) break;
        if (!is_b) {
            const int g = r % GA;
            if (run)
                cols_tile_regs<L1, C, INV, true, St::Keep, T>(v, a.work + tr * N + (int64_t)g * C, N2,
                                                              (uint32_t)(g * C), a.tw_a, a.lo, a.hi, a.sh, slot, pol, 1,
                                                              slots + NS * (CF::SLOT / 8));
            fence_proxy_async_smem();
            tile_sync<T>();  // the tile's stores and slot accesses are done
            if (threadIdx.x == 0) {
                mbar_arrive(&empty[s]);
                if (j != a.withhold_chunk) {
                    __threadfence();
                    atomicAdd(a.ctl + 1 + j, 1);
                }
            }
        } else {
            const int h = r % GB;
            if (run)
                rowsT_tile_regs<L2, TPC, INV, St::Stream, T>(v, a.out + tr * N + (int64_t)h * TPC, N1, a.tw_b, slot,
                                                             pol);
            fence_proxy_async_smem();
            tile_sync<T>();
            if (threadIdx.x == 0) mbar_arrive(&empty[s]);
            if (run) {  // the tile's workspace rows are consumed: drop them from L2
                const char* src = reinterpret_cast<const char*>(a.work + tr * N + (int64_t)h * TPC * N2);
                constexpr int LINES = CF::TILE * 8 / 128;
                for (int l = threadIdx.x; l < LINES; l += T) l2_discard_line(src + (int64_t)l * 128);
            }
        }
    }
}

}  // namespace b300fft
