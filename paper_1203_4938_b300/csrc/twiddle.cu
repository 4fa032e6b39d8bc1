// twiddle.cu -- plan-time twiddle tables, evaluated on the GPU in FP64 and
// rounded once to FP32 (the rounding of these factors sets the FFT's error
// floor, so they are never built by recurrence and never in FP32).
//
// W_L^m = exp(-2*pi*i*m/L) for the DFT of the paper's Sec. III-A example; the
// inverse transform conjugates at use.
#include "launch.h"
#include "stockham_pow2.cuh"

namespace b300fft {

// exp(-2 pi i m / L), m already reduced to [0, L).
__device__ __forceinline__ float2 root_fp64(int64_t m, int64_t L) {
    double s, c;
    sincospi(2.0 * (double)m / (double)L, &s, &c);
    return make_float2((float)c, (float)(-s));
}

// One Stockham pass block: out[(r-1)*Ns + k] = W_{Ns*R}^{k*r}.
__global__ void k_tw_pass(float2* out, int Ns, int R) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t cnt = (int64_t)(R - 1) * Ns;
    if (i >= cnt) return;
    const int64_t r = i / Ns + 1, k = i - (r - 1) * Ns;
    out[i] = root_fp64(k * r, (int64_t)Ns * R);
}

// out[i] = W_n^((i*mult) mod n)
__global__ void k_tw_roots(float2* out, int64_t count, int64_t mult, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int64_t m = (int64_t)(((__int128)i * mult) % n);
    out[i] = root_fp64(m, n);
}

namespace {
struct PassList {
    int n = 0;
    int radix[8];
};
template <int LOGN>
PassList passes_of() {
    using PL = P2Plan<LOGN>;
    PassList p;
    p.n = PL::NPASS;
    for (int i = 0; i < PL::NPASS; ++i) p.radix[i] = PL::radix(i);
    return p;
}
PassList pow2_passes(int logn) {
    switch (logn) {
#define B300_CASE(L) \
    case L:          \
        return passes_of<L>();
        B300_CASE(0) B300_CASE(1) B300_CASE(2) B300_CASE(3) B300_CASE(4) B300_CASE(5) B300_CASE(6)
        B300_CASE(7) B300_CASE(8) B300_CASE(9) B300_CASE(10) B300_CASE(11) B300_CASE(12)
        B300_CASE(13) B300_CASE(14)
#undef B300_CASE
        default:
            return PassList{};
    }
}
}  // namespace

int pow2_table_entries(int logn) {
    PassList p = pow2_passes(logn);
    int ns = 1, total = 0;
    for (int i = 0; i < p.n; ++i) {
        if (i > 0) total += (p.radix[i] - 1) * ns;
        ns *= p.radix[i];
    }
    return total;
}

cudaError_t gen_pow2_table(float2* tw, int logn, cudaStream_t st) {
    PassList p = pow2_passes(logn);
    if (p.n == 0) return cudaErrorInvalidValue;
    int ns = 1, off = 0;
    for (int i = 0; i < p.n; ++i) {
        if (i > 0) {
            const int cnt = (p.radix[i] - 1) * ns;
            k_tw_pass<<<(cnt + 255) / 256, 256, 0, st>>>(tw + off, ns, p.radix[i]);
            off += cnt;
        }
        ns *= p.radix[i];
    }
    return cudaGetLastError();
}

cudaError_t gen_root_table(float2* out, int64_t count, int64_t mult, int64_t n, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_tw_roots<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(out, count, mult, n);
    return cudaGetLastError();
}

}  // namespace b300fft

// ---------------------------------------------------------------------------
// Tables of the generic (mixed-radix) passes and of Bluestein's algorithm.
// ---------------------------------------------------------------------------
namespace b300fft {

cudaError_t gen_pass_table(float2* out, int Ns, int R, cudaStream_t st) {
    const int cnt = (R - 1) * Ns;
    if (cnt <= 0) return cudaSuccess;
    k_tw_pass<<<(cnt + 255) / 256, 256, 0, st>>>(out, Ns, R);
    return cudaGetLastError();
}

// Bluestein chirp w[n] = exp(-pi i (n^2 mod 2N) / N), n < N, the index
// reduced exactly in 64-bit integers before the FP64 evaluation.
__global__ void k_chirp(float2* out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t m = (int64_t)(((__int128)i * i) % (2 * n));
    double s, c;
    sincospi((double)m / (double)n, &s, &c);
    out[i] = make_float2((float)c, (float)(-s));
}

// Bluestein kernel sequence b of length M (FP64): b[m] = exp(sg*pi i (m^2 mod
// 2N)/N) for m < N and b[M-m] = b[m] for 0 < m < N, zero elsewhere.  With
// sg = +1 this is conj(w) (forward transform), with sg = -1 it is w (inverse).
__global__ void k_bluestein_seq(double2* b, int64_t n, int64_t M, int sg) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    int64_t m = -1;
    if (i < n) m = i;
    else if (i > M - n) m = M - i;
    double2 v = make_double2(0.0, 0.0);
    if (m >= 0) {
        const int64_t q = (int64_t)(((__int128)m * m) % (2 * n));
        double s, c;
        sincospi((double)q / (double)n, &s, &c);
        v = make_double2(c, sg * s);
    }
    b[i] = v;
}

// One radix-2 Stockham pass in FP64 (forward), plan time only.
__global__ void k_fp64_radix2(const double2* __restrict__ src, double2* __restrict__ dst, int64_t M, int64_t Ns) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M / 2) return;
    const int64_t k = j % Ns;
    double s, c;
    sincospi(-(double)k / (double)Ns, &s, &c);  // W_{2Ns}^k
    const double2 a = src[j], b0 = src[j + M / 2];
    const double2 b = make_double2(b0.x * c - b0.y * s, b0.x * s + b0.y * c);
    const int64_t d = (j / Ns) * 2 * Ns + k;
    dst[d] = make_double2(a.x + b.x, a.y + b.y);
    dst[d + Ns] = make_double2(a.x - b.x, a.y - b.y);
}

__global__ void k_round_scale(const double2* __restrict__ src, float2* __restrict__ out, int64_t M, double scale) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    out[i] = make_float2((float)(src[i].x * scale), (float)(src[i].y * scale));
}

cudaError_t gen_chirp(float2* out, int64_t n, cudaStream_t st) {
    k_chirp<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n);
    return cudaGetLastError();
}

// out[0..M) = FFT_M(b)/M in FP64, rounded once to FP32 (the Bluestein filter).
// scratch: 2*M double2 of device memory.
cudaError_t gen_bluestein_filter(float2* out, int64_t n, int64_t M, bool inverse, double2* scratch,
                                 cudaStream_t st) {
    double2* a = scratch;
    double2* b = scratch + M;
    const unsigned g = (unsigned)((M + 255) / 256);
    k_bluestein_seq<<<g, 256, 0, st>>>(a, n, M, inverse ? -1 : +1);
    for (int64_t ns = 1; ns < M; ns *= 2) {
        k_fp64_radix2<<<(unsigned)((M / 2 + 255) / 256), 256, 0, st>>>(a, b, M, ns);
        double2* t = a;
        a = b;
        b = t;
    }
    k_round_scale<<<g, 256, 0, st>>>(a, out, M, 1.0 / (double)M);
    return cudaGetLastError();
}

}  // namespace b300fft
