/*
 * fft.h -- C ABI of the B300 batched complex-to-complex FFT library
 * (libb300fft.so, sm_103a).
 *
 * The operation is the discrete Fourier transform of the paper's Sec. III-A
 * example ("Discrete Fourier Transform Example"): for every length-N sequence
 * x of a batch,
 *
 *     X[k] = sum_{n<N} x[n] * exp(-2*pi*i*n*k/N)     (FFT_FORWARD)
 *     X[k] = sum_{n<N} x[n] * exp(+2*pi*i*n*k/N)     (FFT_INVERSE)
 *
 * unnormalised in both directions, output in natural order.  The paper builds
 * the DFT of N = N1*N2 points from DFTs of sizes N1 and N2 (Cooley-Tukey) and
 * ships a flow of many small DFTs to the data-parallel device; here every
 * level runs on the GPU.  The 2-D form (dims = 2, lengths = {H, W}) is the
 * separable transform X[k1,k2] = sum x[n1,n2] W_H^(n1*k1) W_W^(n2*k2) over
 * image-shaped data, the shape of the paper's Sec. III-B image example.
 *
 * Element type: complex64 = interleaved float pairs (re, im) -- the paper's
 * float2 -- for input and output at every precision setting.
 *
 * Layouts:
 *   1-D     [batch][N], contiguous.
 *   2-D     [batch][H][W], row-major, contiguous.
 *   ragged  the transforms are packed back to back; transform t starts at
 *           element offset sum_{u<t} lengths[u].
 *
 * Ownership: the caller owns the input and output device buffers and the CUDA
 * stream.  A plan owns its twiddle/chirp tables, its workspace, any captured
 * CUDA graph and a device status word; fft_plan_destroy frees them.
 * fft_exec allocates nothing and does not synchronise.
 *
 * Errors: argument errors are returned synchronously as fft_status values.
 * Errors found by a kernel (e.g. a bounded wait that ran out) are written to
 * the plan's device status word and returned by fft_plan_check after the
 * caller has synchronised the stream.  No kernel traps.
 *
 * Threads: plans may be created and destroyed from any thread; one plan must
 * not be executed concurrently on two streams when it uses a workspace
 * (fft_plan_workspace_bytes > 0).
 */
#ifndef B300_FFT_H
#define B300_FFT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FFT_API __attribute__((visibility("default")))
#else
#define FFT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fft_plan_s *fft_plan;

typedef enum {
    FFT_OK = 0,
    FFT_ERR_INVALID_ARG = 1,  /* bad dims, length, batch, direction or NULL pointer */
    FFT_ERR_UNSUPPORTED = 2,  /* valid request this library does not implement      */
    FFT_ERR_ALLOC = 3,        /* device or host allocation failed at plan time       */
    FFT_ERR_MISALIGNED = 4,   /* input or output pointer not 16-byte aligned         */
    FFT_ERR_CUDA = 5,         /* a CUDA runtime call failed                          */
    FFT_ERR_TIMEOUT = 6,      /* a bounded device-side wait expired                  */
    FFT_ERR_BAD_HANDLE = 7    /* NULL, destroyed or foreign plan handle              */
} fft_status;

/* Arithmetic of the transform; input and output are complex64 in every mode. */
typedef enum {
    FFT_FP32 = 0,          /* FP32 Stockham passes on the CUDA cores             */
    FFT_TC_FP16 = 1,       /* radix-16 stages as FP16 tensor-core GEMMs, hi+lo   */
    FFT_TC_BF16 = 2,       /* radix-16 stages as BF16 tensor-core GEMMs, hi+lo   */
    FFT_TC_FP16_PLAIN = 3, /* FP16 tensor-core stages without the lo correction  */
    FFT_TC_BF16_PLAIN = 4  /* BF16 tensor-core stages without the lo correction  */
} fft_precision;

enum { FFT_FORWARD = -1, FFT_INVERSE = +1 };

/* Create a plan for `batch` transforms of the given shape.
 *   dims     1 or 2.
 *   lengths  dims entries: {N} or {H, W}; every entry >= 1.
 *   batch    number of transforms (>= 1).
 *   precision one of fft_precision (tensor-core modes: 1-D, N = 16^k, k >= 2).
 * Computes the twiddle tables on the device in FP64 and rounds them once to
 * FP32; allocates the workspace a multi-pass length needs.  Synchronises the
 * current device once.  2-D: sides that are powers of two (W <= 2^14,
 * H <= 2^12) or 3/5/7 * 2^k <= 4096 run as a rows pass and an in-place column
 * pass; any other pair of lengths that a 1-D plan supports runs as a 1-D plan
 * over the rows, a transpose, a 1-D plan over the columns and a transpose
 * back (a batch*H*W complex workspace).  1-D lengths above 2^24 points
 * that factor as N1 * N2 with both factors supported run as a six-step
 * (transpose, N1-point plan, twiddle + transpose, N2-point plan, transpose;
 * a batch*N complex workspace).  Returns NULL on error;
 * fft_last_error() says why. */
FFT_API fft_plan fft_plan_create(int dims, const int64_t *lengths, int64_t batch, int precision);

/* Create a plan for `count` 1-D transforms of uneven lengths, packed back to
 * back (see Layouts).  lengths: host array of `count` entries, each in
 * [1, 2^20].  The whole batch runs as one persistent kernel launch, captured
 * once into a CUDA graph at plan time.  precision must be FFT_FP32. */
FFT_API fft_plan fft_plan_create_ragged(const int64_t *lengths, int64_t count, int precision);

/* Create a plan for `batch` real transforms of even length n (half spectrum).
 * fft_exec with FFT_FORWARD maps real input [batch][n] (floats) to complex
 * output [batch][n/2+1] (bins 0..n/2 of the DFT of the paper's Sec. III-A;
 * the rest follow from X[n-k] = conj(X[k])); FFT_INVERSE maps [batch][n/2+1]
 * complex (a Hermitian half spectrum) to [batch][n] real, unnormalised, so
 * inverse(forward(x)) = n x.  Built on the complex plan of length n/2 (any
 * length fft_plan_create supports) plus one split pass; the plan holds an
 * n/2 * batch complex workspace.  NULL on error (odd n: FFT_ERR_UNSUPPORTED). */
FFT_API fft_plan fft_plan_create_real(int64_t n, int64_t batch);

/* Spectrum product of FFT convolution / correlation (the paper's Sec. III-A
 * names convolution among the DFT's uses):
 *     out[t][k] = scale * a[t][k] * b[k]          (conj_b = 0: convolution)
 *     out[t][k] = scale * a[t][k] * conj(b[k])    (conj_b != 0: correlation)
 * for t < batch, k < n; a, out: [batch][n] complex64 (out == a allowed),
 * b: [n] complex64 broadcast over the batch; device pointers, 16-byte
 * aligned.  With a = DFT(x), b = DFT(h) and scale = 1/n, the inverse
 * transform of out is the circular convolution (correlation) of x with h.
 * Asynchronous on `stream`. */
FFT_API fft_status fft_spectrum_product(const void *a, const void *b, void *out, int64_t n, int64_t batch,
                                        float scale, int conj_b, void *stream);

/* FFT convolution / correlation of every row in one call (Sec. III-A names
 * convolution among the DFT's uses):
 *     out[t] = scale * IDFT( DFT(x[t]) * H )          (conj_h = 0)
 *     out[t] = scale * IDFT( DFT(x[t]) * conj(H) )    (conj_h != 0)
 * with the unnormalised transforms of `plan` (an FP32 complex plan: 1-D of
 * n points, or 2-D of n = H * W points, the circular 2-D filtering of every
 * image; batch rows or images; ragged, real and tensor-core plans:
 * FFT_ERR_INVALID_ARG).
 * x, out: [batch][n] complex64; hspec: H = DFT(h), [n] complex64 (2-D:
 * [H][W]); device pointers, 16-byte aligned; out == x allowed.  scale = 1/n
 * gives the circular convolution (correlation) of x with h.  1-D plans of a power of two
 * n <= 2^14 run one fused pass per row (forward passes, product, inverse
 * passes in the tile: one HBM round trip); other plans run the forward
 * transform, fft_spectrum_product and the inverse transform through `out`.
 * Asynchronous on `stream`; allocates nothing. */
FFT_API fft_status fft_convolve(fft_plan plan, const void *x, const void *hspec, void *out, float scale, int conj_h,
                                void *stream);

/* The GPU steps of the image example (Sec. III-B), fused in one pass (no
 * paper formulas are given; the readings below are the standard ones):
 *   1. JFIF (ITU-R BT.601 full range) YCbCr of 8-bit RGB:
 *        Y = .299 R + .587 G + .114 B, Cb = 128 - .168736 R - .331264 G + .5 B,
 *        Cr = 128 + .5 R - .418688 G - .081312 B;
 *   2. Cb, Cr downscaled to a quarter of the pixels (mean of each 2x2 block);
 *   3. directional derivative of Y along (ux, uy): ux dY/dx + uy dY/dy with
 *      central differences inside, one-sided first differences on the border.
 * rgb: [batch][h][w][3] uint8 (interleaved R, G, B), 2-byte aligned;
 * y, d: [batch][h][w] float32; cb, cr: [batch][h/2][w/2] float32, 4-byte
 * aligned; device pointers (misaligned: FFT_ERR_MISALIGNED).
 * h, w even, 2 <= h <= 2^19, 2 <= w <= 2^24, batch <= 65535 (else
 * FFT_ERR_INVALID_ARG).  Asynchronous on `stream`; allocates nothing. */
FFT_API fft_status fft_image_steps(const void *rgb, int64_t batch, int64_t h, int64_t w, float ux, float uy,
                                   void *y, void *cb, void *cr, void *d, void *stream);

/* FP32 FMA throughput probe (measurement aid, not part of a transform): the
 * non-tensor arithmetic ceiling that the butterfly work is compared with.
 * Launches `blocks` CTAs of 256 threads; each thread runs 16 independent
 * FMA chains for `iters` rounds, i.e. blocks * 256 * 16 * iters FMAs
 * (2 flops each).  out: device float32 [blocks * 256], 4-byte aligned; every
 * element is set to 120 + 16 * iters (exact).  1 <= blocks <= 2^24,
 * 1 <= iters <= 2^20 (else FFT_ERR_INVALID_ARG).  Asynchronous on `stream`. */
FFT_API fft_status fft_probe_fma(void *out, int64_t blocks, int64_t iters, void *stream);

/* Status of the last fft_plan_create* call on this host thread. */
FFT_API fft_status fft_last_error(void);

/* Enqueue the transform of `in` into `out` on `stream` (a cudaStream_t, or
 * NULL for the legacy default stream).  in and out are device pointers,
 * 16-byte aligned, holding the plan's elements; in == out is allowed.
 * direction: FFT_FORWARD or FFT_INVERSE.  Asynchronous; allocates nothing. */
FFT_API fft_status fft_exec(fft_plan plan, const void *in, void *out, int direction, void *stream);

/* Same result and arguments as fft_exec, but for plans built by the
 * stage-graph executor (ragged plans and non-power-of-two lengths) it enqueues
 * one kernel launch per (stage, length) group, in dependency order, instead of
 * the single persistent launch: the per-size-launch baseline the persistent
 * form is compared against.  For other plans it is fft_exec. */
FFT_API fft_status fft_exec_per_size(fft_plan plan, const void *in, void *out, int direction, void *stream);

/* Read and clear the plan's device status word, and those of the plans a
 * real or transposing 2-D plan runs inside it; returns the first nonzero one
 * (synchronous; call it after the stream that ran fft_exec has been
 * synchronised). */
FFT_API fft_status fft_plan_check(fft_plan plan);

/* Free every resource of the plan.  Synchronises the device first. */
FFT_API fft_status fft_plan_destroy(fft_plan plan);

/* Bytes of device workspace the plan holds, with those of the plans it runs
 * inside it (0 for single-pass plans). */
FFT_API size_t fft_plan_workspace_bytes(fft_plan plan);

/* Static English text for a status value. */
FFT_API const char *fft_status_string(fft_status status);

/* Number of kernel launches one fft_exec of this plan enqueues (a captured
 * graph counts its kernels).  0 for an invalid handle. */
FFT_API int fft_plan_kernel_count(fft_plan plan);

/* Enqueue only kernel `k` (0 <= k < fft_plan_kernel_count) of the sequence
 * fft_exec would enqueue, with the same arguments; intermediate results live
 * in the plan's workspace, so running k = 0, 1, ... in order on one stream is
 * exactly fft_exec.  For per-kernel timing and profiling. */
FFT_API fft_status fft_exec_kernel(fft_plan plan, int k, const void *in, void *out, int direction, void *stream);

/* Allocation-free 1-D transform.  The paper has no counterpart to this entry
 * point; it exists for callers that cannot call cudaMalloc -- code that runs
 * after its host has fixed every device allocation (an embedded engine, a
 * plugin whose host forbids allocation, a loop that budgets all device memory
 * at start-up) -- and so cannot create a plan, whose tables and workspace are
 * allocated.  It computes the same transform as a plan for (1, {n}, batch)
 * with the same two-pass kernels, but keeps its workspace and twiddle tables
 * in arrays that are part of the library image: every GPU on which the
 * library's device code is loaded holds them (about 32.1 MiB) until the
 * process exits.  Under CUDA's default lazy module loading that memory is
 * committed at the first call on each device, not when the library is
 * loaded: make one call per device before the host fixes its device-memory
 * budget (and before any stream capture).
 *   in, out    device pointers, 16-byte aligned, batch * n complex64 each
 *              ([batch][n]); in == out is allowed.
 *   n          a power of two, 2^13 <= n <= 2^22.
 *   batch      >= 1 with n * batch <= 2^22 (the size of the static
 *              workspace); larger requests return FFT_ERR_INVALID_ARG.
 *   direction  FFT_FORWARD or FFT_INVERSE;  stream  a cudaStream_t or NULL.
 * Allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
 * The first call on a device looks up the device addresses of the static
 * arrays and sets kernel attributes for that device.  Every call on a device
 * shares the same arrays: the twiddle tables are rebuilt on the stream only
 * when n differs from the previous call's on that device, and the workspace
 * is fully overwritten before it is read, so calls whose execution overlaps
 * on the GPU -- on different streams, or from different threads -- race and
 * give wrong results; order them on one stream.  Asynchronous like fft_exec. */
FFT_API fft_status fft_exec_pow2_static(const void *in, void *out, int64_t n, int64_t batch, int direction,
                                        void *stream);

/* Human-readable one-line description of the plan's decomposition (kernel
 * family, radix sequence, tile shape) copied into buf (NUL-terminated,
 * truncated to cap bytes).  Returns the full length, or -1 on a bad handle. */
FFT_API int fft_plan_describe(fft_plan plan, char *buf, size_t cap);

#ifdef __cplusplus
}
#endif
#endif /* B300_FFT_H */
