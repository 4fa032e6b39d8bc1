// launch.h -- host-side entry points of the kernel translation units, used by
// the plan/ABI layer (fft_api.cu).  Internal to the library.
#pragma once
#include <cuda.h>  // CUtensorMap (descriptor type only; the driver API is not linked)
#include <cuda_runtime.h>
#include <stdint.h>

namespace b300fft {

// Largest power-of-two length a single CTA transforms on its own.
constexpr int kRowsMaxLog = 14;
// Whether plans of 2^logn use the staged persistent rows kernel by default
// (measured per direction on 2^26 elements: 2^14 253 vs 275 us, 2^13 218 vs
// 211 us -- two plain CTAs per SM already overlap each other's loads).
constexpr int rows_staged_default(int logn) { return logn == 14 ? 1 : 0; }
// Largest column length of the columns kernel.
constexpr int kColsMaxLog = 12;

// --- power-of-two Stockham tables (twiddle.cu) ---------------------------
// Number of FP32 twiddle entries the register-staged kernels read for 2^logn.
int pow2_table_entries(int logn);
// Fill tw[0 .. pow2_table_entries(logn)) on `st` (FP64 evaluation).
cudaError_t gen_pow2_table(float2* tw, int logn, cudaStream_t st);
// out[i] = W_n^((i * mult) mod n) = exp(-2 pi i (i*mult mod n)/n), i < count.
cudaError_t gen_root_table(float2* out, int64_t count, int64_t mult, int64_t n, cudaStream_t st);
// One Stockham pass block: out[(r-1)*Ns + k] = W_{Ns*R}^{k*r}, r < R, k < Ns.
cudaError_t gen_pass_table(float2* out, int Ns, int R, cudaStream_t st);
// Bluestein chirp w[n] = exp(-pi i (n^2 mod 2N)/N), n < N.
cudaError_t gen_chirp(float2* out, int64_t n, cudaStream_t st);
// Bluestein filter FFT_M(b)/M (FP64, rounded once); scratch = 2*M double2.
cudaError_t gen_bluestein_filter(float2* out, int64_t n, int64_t M, bool inverse, double2* scratch,
                                 cudaStream_t st);

// --- rows kernel (k_rows.cu) ----------------------------------------------
// nrows contiguous transforms of length 2^logn, [nrows][2^logn] -> same layout.
int rows_tpc(int logn);
int rows_threads(int logn);
cudaError_t rows_prepare(int logn);  // raise the dynamic shared-memory limit
// --- single-pass mixed radix, L = M * 2^K <= 4096, M = 3, 5, 7 (k_mixed.cu) ----
bool mixed_supported(int64_t n, int* m, int* k);
int mixed_table_entries(int m, int k);
int mixed_lines_per_cta(int m, int k);
cudaError_t gen_mixed_table(float2* tw, int m, int k, cudaStream_t st);
cudaError_t launch_rows_mixed(int m, int k, bool inv, const float2* in, float2* out, int64_t nrows, const float2* tw,
                              cudaStream_t st);
// Four-step first pass for N = M * 2^a * S2: columns of length M * 2^a over
// `items` row-major [M * 2^a][S2] arrays, mixed_cols_width(m, a) columns per
// CTA (0: no kernel for that length), times W_N^{n2 k1} from (lo, hi, sh).
int mixed_cols_width(int m, int a);
// out[b][c][r] = in[b][r][c] for [batch][rows][cols] complex64 (transpose.cu);
// in != out.
cudaError_t launch_transpose(const float2* in, float2* out, int64_t rows, int64_t cols, int64_t batch,
                             cudaStream_t st);
// out[b][c][r] = in[b][r][c] * W_n^{r*c} (conjugated when inv); lo / hi: the
// two-level root tables of n (2^sh and ceil(n / 2^sh) entries); in != out.
cudaError_t launch_twiddle_transpose(const float2* in, float2* out, int64_t rows, int64_t cols, int64_t batch,
                                     int64_t n, const float2* lo, const float2* hi, int sh, bool inv,
                                     cudaStream_t st);
// 2-D column pass: columns of length M * 2^K (no twiddle), mixed_cols2d_width
// columns per CTA (S2 must be a multiple of it).
int mixed_cols2d_width(int m, int k);
cudaError_t launch_cols2d_mixed(int m, int k, bool inv, const float2* in, float2* out, int64_t S2, int64_t items,
                                const float2* tw, cudaStream_t st);
cudaError_t launch_cols_mixed(int m, int a, bool inv, const float2* in, float2* out, int64_t S2, int64_t items,
                              const float2* tw, const float2* lo, const float2* hi, int sh, cudaStream_t st);

// One-pass FFT convolution of rows of 2^logn (conv.cu): forward passes, times
// hs (or conj(hs)) and scale, inverse passes; tw = the rows plan's table.
cudaError_t launch_conv_rows(int logn, bool corr, const float2* in, float2* out, int64_t nrows, const float2* tw,
                             const float2* hs, float scale, cudaStream_t st);

cudaError_t launch_rows(int logn, bool inv, const float2* in, float2* out, int64_t nrows, const float2* tw,
                        cudaStream_t st);

// --- transposed rows (k_rowsT.cu) -------------------------------------------
// Four-step second pass: nrows = items * n1 rows of length 2^logn, `tpc` rows
// per CTA (2..64, n1 % tpc == 0); row k1 of item j, bin k2 goes to
// out[j*n1*2^logn + k1 + n1*k2].
int rowsT_threads(int logn, int tpc);
cudaError_t rowsT_prepare(int logn, int tpc);
cudaError_t launch_rowsT(int logn, int tpc, bool inv, const float2* in, float2* out, int64_t nrows, const float2* tw,
                         int64_t n1, cudaStream_t st);

// --- columns kernel (k_cols.cu) -------------------------------------------
// C = adjacent columns per CTA, a power of two in [1, 64] with
// C * 2^logn / 16 <= 1024 threads.  cols_width is the default for a length;
// cols_width_for the widest valid width that divides ncols (0 if none).
bool cols_width_valid(int logn, int c);
int cols_width(int logn);
int cols_width_for(int logn, int64_t ncols);
int cols_threads(int logn, int c);
cudaError_t cols_prepare(int logn, int c);
// Column transforms of length 2^logn over `ncols` adjacent columns of each of
// `nitems` row-major [2^logn][S] arrays (item_stride elements apart).  With
// twiddle_out, element (k1, n2) is multiplied by W_{2^logn * S}^{n2*k1} from
// the two-level table (lo, hi, sh).
cudaError_t launch_cols(int logn, int c, bool inv, bool twiddle_out, const float2* in, float2* out, int64_t S,
                        int64_t ncols, int64_t item_stride, int64_t nitems, const float2* tw, const float2* lo,
                        const float2* hi, int sh, cudaStream_t st);

// --- persistent four-step (k_persist.cu) -----------------------------------
struct PersistArgs;  // persist.cuh
struct PersistConfig {
    int l1, c, l2, tpc;  // N = 2^l1 * 2^l2; column width c, transposed rows per CTA tpc
};
struct PersistInfo {
    int threads = 0, smem = 0, blocks_per_sm = 0;
};
bool persist_config_available(const PersistConfig& c);
cudaError_t persist_prepare(const PersistConfig& c, PersistInfo* info);
cudaError_t launch_fourstep_persist(const PersistConfig& c, bool inv, const PersistArgs& a, int grid,
                                    cudaStream_t st);

// --- persistent rows kernel with bulk-copied input staging (k_rows_staged.cu)
// nrows contiguous transforms of 2^logn (13 or 14); `in` must be 16-byte
// aligned (the copies read whole rows); grid <= nrows persistent CTAs; a
// staged row that does not arrive within `polls` waits of ~1 us sets
// *status = FFT_ERR_TIMEOUT.
bool rows_staged_available(int logn);
cudaError_t rows_staged_prepare(int logn, PersistInfo* info);
cudaError_t launch_rows_staged(int logn, bool inv, const float2* in, float2* out, int64_t nrows, const float2* tw,
                               int* status, int64_t polls, int grid, cudaStream_t st);

// --- tensor maps of the asynchronous tile copies (k_pipe.cu) -----------------
// Encode a tiled tensor map over 8-byte elements (complex64): dims[0] is the
// innermost extent, strides_bytes[i] the byte stride of dimension i + 1, box
// the copied box (each extent <= 256).  False when the driver's encoder is
// unavailable or refuses the layout.
bool tensor_maps_available();
bool encode_tensor_map(CUtensorMap* tm, const void* base, int rank, const uint64_t* dims,
                       const uint64_t* strides_bytes, const uint32_t* box);

// --- persistent four-step with asynchronous tile loads (k_pipe.cu) ----------
// The same decomposition as launch_fourstep_persist, run by a producer warp
// (tensor-memory-accelerator copies into a ring of ns = 2 or 3 shared-memory
// slots) and the consumer warps of one tile per CTA.
bool pipe_config_available(const PersistConfig& c, int ns);
cudaError_t pipe_prepare(const PersistConfig& c, int ns, PersistInfo* info);
cudaError_t launch_fourstep_pipe(const PersistConfig& c, int ns, bool inv, const PersistArgs& a, int grid,
                                 cudaStream_t st);

// --- persistent 2-D (k_2d.cu) --------------------------------------------------
// PersistConfig fields: l1 = log2 W, c = rows per row tile, l2 = log2 H,
// tpc = columns per column tile.
bool persist2d_config_available(const PersistConfig& c);
cudaError_t persist2d_prepare(const PersistConfig& c, PersistInfo* info);
cudaError_t launch_2d_persist(const PersistConfig& c, bool inv, const PersistArgs& a, int grid, cudaStream_t st);

// --- persistent three-stage (k_three.cu) ------------------------------------
// N = 2^la * 2^lb1 * 2^lb2, each stage length in 2^6 .. 2^8, tiles of 4096 or
// 16384 points.
struct ThreeArgs;  // threestep.cuh
struct ThreeConfig {
    int la, lb1, lb2;
    int tile = 4096;  // points per tile: 4096 (256 threads) or 16384 (1024 threads)
};
bool three_config_available(const ThreeConfig& c);
cudaError_t three_prepare(const ThreeConfig& c, PersistInfo* info);
cudaError_t launch_threestep(const ThreeConfig& c, bool inv, const ThreeArgs& a, int grid, cudaStream_t st);
// The same with asynchronous tile loads (pipe3.cuh) into a ring of ns = 2 or 3 slots.
bool three_pipe_available(const ThreeConfig& c, int ns);
cudaError_t three_pipe_prepare(const ThreeConfig& c, int ns, PersistInfo* info);
cudaError_t launch_threestep_pipe(const ThreeConfig& c, int ns, bool inv, const ThreeArgs& a, int grid,
                                  cudaStream_t st);

// --- thread-block-cluster single pass (k_cluster.cu) --------------------------
// N = K * 2^lm (K = 8 or 16 CTAs per transform, DSMEM exchanges).
bool cluster_config_available(int lm, int k);
// raise the kernel attributes; *max_clusters = co-resident clusters (0: cannot run)
cudaError_t cluster_prepare(int lm, int k, int* max_clusters);
cudaError_t launch_cluster_fft(int lm, int k, bool inv, const float2* in, float2* out, int64_t batch,
                               const float2* tw, const float2* lo, const float2* hi, int sh, cudaStream_t st);

}  // namespace b300fft
