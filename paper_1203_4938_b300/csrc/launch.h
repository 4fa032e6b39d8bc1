// launch.h -- host-side entry points of the kernel translation units, used by
// the plan/ABI layer (fft_api.cu).  Internal to the library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace b300fft {

// Largest power-of-two length a single CTA transforms on its own.
constexpr int kRowsMaxLog = 14;
// Largest column length of the columns kernel.
constexpr int kColsMaxLog = 12;

// --- power-of-two Stockham tables (twiddle.cu) ---------------------------
// Number of FP32 twiddle entries the register-staged kernels read for 2^logn.
int pow2_table_entries(int logn);
// Fill tw[0 .. pow2_table_entries(logn)) on `st` (FP64 evaluation).
cudaError_t gen_pow2_table(float2* tw, int logn, cudaStream_t st);
// out[i] = W_n^((i * mult) mod n) = exp(-2 pi i (i*mult mod n)/n), i < count.
cudaError_t gen_root_table(float2* out, int64_t count, int64_t mult, int64_t n, cudaStream_t st);

// --- rows kernel (k_rows.cu) ----------------------------------------------
// Transforms-per-CTA the rows kernel uses for 2^logn (plain and transposed).
int rows_tpc(int logn, bool transposed);
// Dynamic shared memory bytes of that configuration.
int rows_smem(int logn, bool transposed);
int rows_threads(int logn, bool transposed);
// Raise the dynamic shared-memory limit of the kernels a plan will use.
cudaError_t rows_prepare(int logn, bool transposed);
// nrows transforms of length 2^logn, [nrows][2^logn] -> same layout, or with
// transposed=true the four-step output layout (see stockham_pow2.cuh).
cudaError_t launch_rows(int logn, bool inv, bool transposed, const float2* in, float2* out, int64_t nrows,
                        const float2* tw, int64_t n1, cudaStream_t st);

// --- columns kernel (k_cols.cu) -------------------------------------------
// C = adjacent columns per CTA.  cols_width is the default for a length (the
// only width with the four-step twiddle); cols_width_for picks the widest
// instantiated width (default, 4 or 1) that divides ncols.
int cols_width(int logn);
int cols_width_for(int logn, int64_t ncols);
int cols_smem(int logn, int c);
int cols_threads(int logn, int c);
cudaError_t cols_prepare(int logn, int c);
// Column transforms of length 2^logn over `ncols` adjacent columns of each of
// `nitems` row-major [2^logn][S] arrays (item_stride elements apart).  With
// twiddle_out (default width only), element (k1, n2) is multiplied by
// W_{2^logn * S}^{n2*k1} from the two-level table (lo, hi, sh).
cudaError_t launch_cols(int logn, int c, bool inv, bool twiddle_out, const float2* in, float2* out, int64_t S,
                        int64_t ncols, int64_t item_stride, int64_t nitems, const float2* tw, const float2* lo,
                        const float2* hi, int sh, cudaStream_t st);

}  // namespace b300fft
