// persist2d.cuh -- the 2-D transform (rows, then columns; the image-shaped
// form of the Sec. III-A DFT) in one persistent launch whose intermediate
// stays in L2: the queue and dependency counters of persist.cuh, with
//   A tiles = TPC consecutive rows of length W of one image (rows_tile), written
//             to `out` with an L2 evict-last policy;
//   B tiles = C adjacent columns of length H of one image (cols_tile, no
//             twiddle), read from L2 and written back in place.
// The batch is cut into chunks of images whose rows fit in L2; a chunk's B
// tiles wait (bounded) for all of its A tiles.
#pragma once
#include "persist.cuh"

namespace b300fft {

template <int LW, int TPC, int LH, int C>
struct TwoDPersistCfg {
    static constexpr int THREADS = RowsCfg<LW, TPC>::THREADS;
    static_assert(THREADS == ColsCfg<LH, C>::THREADS, "row and column tiles must use the same thread count");
    static constexpr int SMEM =
        RowsCfg<LW, TPC>::SMEM > ColsCfg<LH, C>::SMEM ? RowsCfg<LW, TPC>::SMEM : ColsCfg<LH, C>::SMEM;
};

template <int LW, int TPC, int LH, int C, bool INV>
__global__ void __launch_bounds__(TwoDPersistCfg<LW, TPC, LH, C>::THREADS,
                                  1024 / TwoDPersistCfg<LW, TPC, LH, C>::THREADS)
k_2d_persist(PersistArgs a) {
    constexpr int64_t W = int64_t(1) << LW, H = int64_t(1) << LH, HW = H * W;
    constexpr int GA = (int)(H / TPC);  // row tiles per image
    constexpr int GB = (int)(W / C);    // column tiles per image
    extern __shared__ float2 smem[];
    __shared__ int s_item[2];
    __shared__ int s_ok;
    const uint64_t pol = l2_policy_evict_last();
    const int total = a.nch * (a.na + a.nb);
    if (threadIdx.x == 0) s_item[0] = atomicAdd(a.ctl, 1);
    for (int it = 0;; it ^= 1) {
        __syncthreads();
        const int p = s_item[it];
        if (p >= total) break;
        if (threadIdx.x == 0) s_item[it ^ 1] = atomicAdd(a.ctl, 1);
        bool is_b;
        int j, r;
        decode_item(p, a.na, a.nb, a.nch, &is_b, &j, &r);
        if (!is_b) {
            const int64_t img = (int64_t)j * a.cb + r / GA;
            if (img < a.batch) {
                const int64_t off = img * HW + (int64_t)(r % GA) * TPC * W;
                rows_tile<LW, TPC, INV, Ld::Stream, St::Keep>(a.in + off, a.out + off, TPC, a.tw_a, smem, pol);
            }
            __syncthreads();
            if (threadIdx.x == 0 && j != a.withhold_chunk) {
                __threadfence();
                atomicAdd(a.ctl + 1 + j, 1);
            }
        } else {
            if (threadIdx.x == 0) {
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
            }
            __syncthreads();
            const int64_t img = (int64_t)j * a.cb + r / GB;
            if (s_ok && img < a.batch) {
                const int64_t off = img * HW + (int64_t)(r % GB) * C;
                cols_tile<LH, C, INV, false, Ld::Cg, St::Stream>(a.out + off, a.out + off, W, 0, a.tw_b, nullptr,
                                                                 nullptr, 0, smem, pol);
            }
        }
    }
}

}  // namespace b300fft
