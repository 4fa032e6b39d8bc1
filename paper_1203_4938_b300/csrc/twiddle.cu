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
