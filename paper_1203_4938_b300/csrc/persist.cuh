// persist.cuh -- persistent two-stage kernels with per-chunk dependency
// counters: one launch runs both passes of a four-step (or 2-D) transform.
//
// The batch is cut into chunks whose intermediate data fits in L2.  Work
// items are dequeued from one atomic counter in the order
//     A_0, A_1, B_0, A_2, B_1, ..., A_{n-1}, B_{n-2}, B_{n-1}
// (A = first-pass tiles of a chunk, B = second-pass tiles).  An A tile never
// waits; when it is done its CTA bumps the chunk's counter (release).  A B
// tile waits (acquire, bounded) until its chunk's counter reaches the number
// of A tiles per chunk.  Every A tile a B tile depends on was dequeued before
// it by a CTA that is already running, so the waits always end unless a
// counter is withheld; a wait that exceeds `spin_limit` polls sets the plan's
// status word to FFT_ERR_TIMEOUT and the tile is skipped (no trap, no hang).
//
// Four-step: pass A writes the workspace with an L2 evict-last policy; pass B
// reads it with L2-only loads and then discards those L2 lines, so the
// workspace normally never reaches DRAM and the transform costs about one
// HBM round trip instead of two.
#pragma once
#include "stockham_pow2.cuh"

namespace b300fft {

struct PersistArgs {
    const float2* in;
    float2* out;
    float2* work;
    int* ctl;     // [0] = queue head, [1 + j] = finished A tiles of chunk j
    int* status;  // plan status word (FFT_ERR_TIMEOUT = 6 on an expired wait)
    int64_t batch;
    int64_t cb;  // transforms per chunk
    int nch;     // chunks
    int na, nb;  // A and B tiles per chunk
    const float2* tw_a;
    const float2* tw_b;
    const float2* lo;
    const float2* hi;
    int sh;
    int64_t spin_limit;
    int withhold_chunk;  // debug fault injection: chunk whose A tiles never signal (-1: none)
};

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Position p of the queue -> (is_b, chunk, tile).  Host-callable too, so the
// queue order can be checked without a GPU.
__host__ __device__ __forceinline__ void decode_item(int p, int na, int nb, int nch, bool* is_b, int* chunk, int* tile) {
    if (p < na) {
        *is_b = false;
        *chunk = 0;
        *tile = p;
        return;
    }
    const int q = p - na;
    const int blk = q / (na + nb), r = q - blk * (na + nb);
    if (blk < nch - 1) {
        if (r < na) {
            *is_b = false;
            *chunk = blk + 1;
            *tile = r;
        } else {
            *is_b = true;
            *chunk = blk;
            *tile = r - na;
        }
    } else {
        *is_b = true;
        *chunk = nch - 1;
        *tile = r;
    }
}

// Four-step, N = 2^L1 * 2^L2: A tile = C columns (length 2^L1, stride 2^L2)
// with the inter-pass twiddle; B tile = TPC rows (length 2^L2) with the
// transposed store.  Both tile shapes use C*2^L1/16 = TPC*2^L2/16 threads.
template <int L1, int C, int L2, int TPC>
struct FourStepPersistCfg {
    static constexpr int THREADS = ColsCfg<L1, C>::THREADS;
    static_assert(THREADS == RowsTCfg<L2, TPC>::THREADS, "tile shapes must use the same thread count");
    static constexpr int SMEM =
        ColsCfg<L1, C>::SMEM > RowsTCfg<L2, TPC>::SMEM ? ColsCfg<L1, C>::SMEM : RowsTCfg<L2, TPC>::SMEM;
};

template <int L1, int C, int L2, int TPC, bool INV>
__global__ void __launch_bounds__(FourStepPersistCfg<L1, C, L2, TPC>::THREADS,
                                  1024 / FourStepPersistCfg<L1, C, L2, TPC>::THREADS)
k_fourstep_persist(PersistArgs a) {
    constexpr int64_t N1 = int64_t(1) << L1, N2 = int64_t(1) << L2, N = N1 * N2;
    constexpr int GA = (int)(N2 / C);    // A tiles per transform
    constexpr int GB = (int)(N1 / TPC);  // B tiles per transform
    constexpr int T = FourStepPersistCfg<L1, C, L2, TPC>::THREADS;
    using PA = P2Plan<L1>;
    using PB = P2Plan<L2>;
    extern __shared__ float2 smem[];
    __shared__ int s_item[2];
    __shared__ int s_ok;
    const uint64_t pol = l2_policy_evict_last();
    const int total = a.nch * (a.na + a.nb);
    // thread 0's bookkeeping: the next queue item (an atomic in flight) and a
    // finished A tile's chunk counter still to be signalled; both are
    // published only after this thread has issued its loads of the current
    // tile, so their latency never delays them, and the signal always
    // precedes any wait of this CTA (no deadlock)
    int nxt = 0;
    int pend = -1;  // chunk whose counter thread 0 still has to bump
    if (threadIdx.x == 0) s_item[0] = atomicAdd(a.ctl, 1);
    for (int it = 0;; it ^= 1) {
        __syncthreads();  // previous tile done with smem; s_item[it] visible
        const int p = s_item[it];
        if (p >= total) break;
        if (threadIdx.x == 0) {
            nxt = atomicAdd(a.ctl, 1);
            if (pend >= 0) {
                __threadfence();
                atomicAdd(a.ctl + 1 + pend, 1);
                pend = -1;
            }
        }
        bool is_b;
        int j, r;
        decode_item(p, a.na, a.nb, a.nch, &is_b, &j, &r);
        if (!is_b) {
            const int64_t tr = (int64_t)j * a.cb + r / GA;
            const int g = r % GA;
            if (tr < a.batch) {
                const float2* src = a.in + tr * N + (int64_t)g * C + threadIdx.x % C;
                const int t = threadIdx.x / C;
                float2 v[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = __ldcs(src + (int64_t)(t + i * PA::T) * N2);
                if (threadIdx.x == 0) st_shared_after(&s_item[it ^ 1], nxt);
                cols_tile_regs<L1, C, INV, true, St::Keep>(v, a.work + tr * N + (int64_t)g * C, N2,
                                                           (uint32_t)(g * C), a.tw_a, a.lo, a.hi, a.sh, smem, pol);
            } else if (threadIdx.x == 0) {
                st_shared_after(&s_item[it ^ 1], nxt);
            }
            // the tile's stores are ordered before the signal by the next loop
            // barrier; thread 0 signals after its loads of the next tile
            if (threadIdx.x == 0 && j != a.withhold_chunk) pend = j;
        } else {
            // The wait stays after the loop barrier: the pending signal must
            // cover every thread's stores of the previous tile (a barrier),
            // and it must be published before waiting -- two CTAs that each
            // waited while holding the first-pass signal the other needs
            // (a tile of chunk c+1 pending, waiting on c; and vice versa)
            // would never proceed.
            if (threadIdx.x == 0) {
                if (pend >= 0) {  // before waiting: a pending signal may be what the wait needs
                    __threadfence();
                    atomicAdd(a.ctl + 1 + pend, 1);
                    pend = -1;
                }
                int ok = 1;
                int64_t spins = 0;
                while (ld_acquire_gpu(a.ctl + 1 + j) < a.na) {
                    if (++spins > a.spin_limit) {
                        ok = 0;
                        atomicCAS(a.status, 0, 6);
                        break;
                    }
                    __nanosleep(128);
                }
                s_ok = ok;
                st_shared_after(&s_item[it ^ 1], nxt);  // the atomic returned during the waits above
            }
            __syncthreads();
            const int64_t tr = (int64_t)j * a.cb + r / GB;
            const int h = r % GB;
            if (s_ok && tr < a.batch) {
                const float2* src = a.work + tr * N + (int64_t)h * TPC * N2;
                rowsT_tile<L2, TPC, INV, Ld::Cg, St::Stream>(src, a.out + tr * N + (int64_t)h * TPC, N1, a.tw_b,
                                                             smem, pol);
                // the tile's workspace rows are consumed -- every thread used
                // its loaded values before the tile's exchange barrier -- so
                // drop them from L2
                constexpr int LINES = (int)(TPC * N2 * 8 / 128);
                for (int l = threadIdx.x; l < LINES; l += T)
                    l2_discard_line(reinterpret_cast<const char*>(src) + (int64_t)l * 128);
            }
        }
    }
    if (threadIdx.x == 0 && pend >= 0) {
        __threadfence();
        atomicAdd(a.ctl + 1 + pend, 1);
    }
    (void)PB::T;
}

}  // namespace b300fft
