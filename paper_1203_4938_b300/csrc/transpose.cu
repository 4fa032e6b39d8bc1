// transpose.cu -- batched complex transpose, out[b][c][r] = in[b][r][c].
//
// Used by the general 2-D plan: the 2-D DFT is the 1-D DFT of Sec. III-A
// along every row and then along every column; for sides the in-place column
// kernels do not cover, the column pass runs as a transpose, a 1-D plan over
// the W transposed rows of length H, and a transpose back.
// HBM-bound: each element is read once and written once (16 bytes).  A CTA
// of 32 x 8 threads moves 32 x 32 tiles through shared memory (one padding
// column, so the column-order reads spread over the banks), 256-byte row
// segments on both sides; the grid is a multiple of the SM count and strides
// over the tiles.
//
// The six-step form of a 1-D transform too long for one plan (N = N1 * N2,
// Sec. III-A's split of a DFT into DFTs of the factors) also uses a fused
// variant that multiplies each element by the four-step twiddle W_N^(n2*k1)
// on its way through the tile.
#include <cuda_runtime.h>
#include <stdint.h>

#include "butterfly.cuh"
#include "launch.h"

namespace b300fft {

namespace {

constexpr int kT = 32;      // tile side
constexpr int kRowsPT = 4;  // rows per thread (blockDim.y = kT / kRowsPT)

__global__ void __launch_bounds__(kT * (kT / kRowsPT))
    k_transpose(const float2* __restrict__ in, float2* __restrict__ out, int64_t rows, int64_t cols, int64_t tr,
                int64_t tc, int64_t tiles) {
    __shared__ float2 t[kT][kT + 1];
    const int x = threadIdx.x, y = threadIdx.y;
    for (int64_t q = blockIdx.x; q < tiles; q += gridDim.x) {
        const int64_t per = tr * tc;
        const int64_t b = q / per, rem = q - b * per;
        const int64_t i0 = (rem / tc) * kT, j0 = (rem % tc) * kT;
        const float2* src = in + b * rows * cols;
        float2* dst = out + b * rows * cols;
#pragma unroll
        for (int k = 0; k < kRowsPT; ++k) {
            const int r = y + k * (kT / kRowsPT);
            if (i0 + r < rows && j0 + x < cols) t[r][x] = __ldcs(src + (i0 + r) * cols + j0 + x);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kRowsPT; ++k) {
            const int c = y + k * (kT / kRowsPT);
            if (j0 + c < cols && i0 + x < rows) __stcs(dst + (j0 + c) * rows + i0 + x, t[x][c]);
        }
        __syncthreads();
    }
}

// Z[b][k1][n2] = Y[b][n2][k1] * W_N^(n2 * k1): rows = N2, cols = N1.  The
// exponent is reduced mod N in 64 bits once per thread and tile and then
// stepped by n2 * 8 (mod N) for the thread's four columns; the root is the
// product of two FP64-generated tables, W_N^(m mod 2^sh) and W_N^(2^sh *
// floor(m / 2^sh)).
template <bool INV>
__global__ void __launch_bounds__(kT * (kT / kRowsPT))
    k_twiddle_transpose(const float2* __restrict__ in, float2* __restrict__ out, int64_t rows, int64_t cols,
                        int64_t tr, int64_t tc, int64_t tiles, uint64_t n, const float2* __restrict__ lo,
                        const float2* __restrict__ hi, int sh) {
    __shared__ float2 t[kT][kT + 1];
    const int x = threadIdx.x, y = threadIdx.y;
    const uint32_t mask = (1u << sh) - 1u;
    for (int64_t q = blockIdx.x; q < tiles; q += gridDim.x) {
        const int64_t per = tr * tc;
        const int64_t b = q / per, rem = q - b * per;
        const int64_t i0 = (rem / tc) * kT, j0 = (rem % tc) * kT;
        const float2* src = in + b * rows * cols;
        float2* dst = out + b * rows * cols;
#pragma unroll
        for (int k = 0; k < kRowsPT; ++k) {
            const int r = y + k * (kT / kRowsPT);
            if (i0 + r < rows && j0 + x < cols) t[r][x] = __ldcs(src + (i0 + r) * cols + j0 + x);
        }
        __syncthreads();
        // store side: element (n2 = i0 + x, k1 = j0 + c), c = y + 8k
        const uint64_t n2 = (uint64_t)(i0 + x);
        uint64_t e = (n2 * (uint64_t)(j0 + y)) % n;
        const uint64_t step = (n2 * (uint64_t)(kT / kRowsPT)) % n;
#pragma unroll
        for (int k = 0; k < kRowsPT; ++k) {
            const int c = y + k * (kT / kRowsPT);
            if (j0 + c < cols && i0 + x < rows) {
                const uint32_t m = (uint32_t)e;
                const float2 w = cmul(__ldg(hi + (m >> sh)), __ldg(lo + (m & mask)));
                __stcs(dst + (j0 + c) * rows + i0 + x, twmul<INV>(t[x][c], w));
            }
            e += step;
            if (e >= n) e -= n;
        }
        __syncthreads();
    }
}

int transpose_grid(int64_t tiles) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    const int64_t cap = (int64_t)sms * 8;  // 8 CTAs of 256 threads per SM
    return (int)(tiles < cap ? tiles : cap);
}

}  // namespace

cudaError_t launch_twiddle_transpose(const float2* in, float2* out, int64_t rows, int64_t cols, int64_t batch,
                                     int64_t n, const float2* lo, const float2* hi, int sh, bool inv,
                                     cudaStream_t st) {
    if (rows < 1 || cols < 1 || batch < 1 || n < 1 || n > (int64_t(1) << 32) || sh < 1 || sh > 31)
        return cudaErrorInvalidValue;
    const int64_t tr = (rows + kT - 1) / kT, tc = (cols + kT - 1) / kT, tiles = tr * tc * batch;
    const dim3 blk(kT, kT / kRowsPT);
    if (inv)
        k_twiddle_transpose<true><<<transpose_grid(tiles), blk, 0, st>>>(in, out, rows, cols, tr, tc, tiles,
                                                                         (uint64_t)n, lo, hi, sh);
    else
        k_twiddle_transpose<false><<<transpose_grid(tiles), blk, 0, st>>>(in, out, rows, cols, tr, tc, tiles,
                                                                          (uint64_t)n, lo, hi, sh);
    return cudaGetLastError();
}

cudaError_t launch_transpose(const float2* in, float2* out, int64_t rows, int64_t cols, int64_t batch,
                             cudaStream_t st) {
    if (rows < 1 || cols < 1 || batch < 1) return cudaErrorInvalidValue;
    const int64_t tr = (rows + kT - 1) / kT, tc = (cols + kT - 1) / kT, tiles = tr * tc * batch;
    k_transpose<<<transpose_grid(tiles), dim3(kT, kT / kRowsPT), 0, st>>>(in, out, rows, cols, tr, tc, tiles);
    return cudaGetLastError();
}

}  // namespace b300fft
