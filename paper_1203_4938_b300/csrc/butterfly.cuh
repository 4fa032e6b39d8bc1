// butterfly.cuh -- in-register small DFTs (the "DFT of size 2^k computed in a
// program node" of the paper's Sec. III-A example, generalised to radices
// 2, 3, 4, 5, 7, 8 and 16) and complex helpers for the Stockham passes.
//
// Sign convention: forward uses exp(-2*pi*i*n*k/R), inverse exp(+...); both
// unnormalised.  A butterfly works on R registers v[base + stride*r], r < R,
// in place, with compile-time indices so the "strided register" view costs
// nothing after unrolling.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace b300fft {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// multiply by the table twiddle w (forward) or its conjugate (inverse)
template <bool INV>
__device__ __forceinline__ float2 twmul(float2 a, float2 w) { return INV ? cmulc(a, w) : cmul(a, w); }
// multiply by -i (forward) or +i (inverse): W_4^1 of the chosen direction
template <bool INV>
__device__ __forceinline__ float2 rot4(float2 a) { return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// Exact values of cos/sin at multiples of pi/8 (mathematical constants).
#define B300_C8 0.70710678118654752440f   // cos(pi/4)
#define B300_C16 0.92387953251128675613f  // cos(pi/8)
#define B300_S16 0.38268343236508977173f  // sin(pi/8)

// Multiply by W_16^m of the chosen direction, m in [0, 16), compile-time m.
template <int M, bool INV>
__device__ __forceinline__ float2 w16(float2 a) {
    constexpr int m = M & 15;
    // forward W_16^m = cos(2 pi m/16) - i sin(2 pi m/16); inverse conjugates.
    if constexpr (m == 0) return a;
    else if constexpr (m == 4) return rot4<INV>(a);
    else if constexpr (m == 8) return make_float2(-a.x, -a.y);
    else if constexpr (m == 12) return rot4<!INV>(a);
    else {
        constexpr float cs[16] = {1.f, B300_C16, B300_C8, B300_S16, 0.f, -B300_S16, -B300_C8, -B300_C16,
                                  -1.f, -B300_C16, -B300_C8, -B300_S16, 0.f, B300_S16, B300_C8, B300_C16};
        constexpr float sn[16] = {0.f, B300_S16, B300_C8, B300_C16, 1.f, B300_C16, B300_C8, B300_S16,
                                  0.f, -B300_S16, -B300_C8, -B300_C16, -1.f, -B300_C16, -B300_C8, -B300_S16};
        const float c = cs[m];
        const float s = INV ? sn[m] : -sn[m];  // forward: -sin
        return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
    }
}

template <int B, int S, bool INV>
__device__ __forceinline__ void dft2(float2* v) {
    float2 a = v[B], b = v[B + S];
    v[B] = cadd(a, b);
    v[B + S] = csub(a, b);
}

template <int B, int S, bool INV>
__device__ __forceinline__ void dft4(float2* v) {
    float2 a0 = v[B], a1 = v[B + S], a2 = v[B + 2 * S], a3 = v[B + 3 * S];
    float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
    float2 t2 = cadd(a1, a3), t3 = rot4<INV>(csub(a1, a3));
    v[B] = cadd(t0, t2);
    v[B + 2 * S] = csub(t0, t2);
    v[B + S] = cadd(t1, t3);
    v[B + 3 * S] = csub(t1, t3);
}

// DFT-8 = one radix-2 step over two DFT-4s of the even and odd samples.
template <int B, int S, bool INV>
__device__ __forceinline__ void dft8(float2* v) {
    float2 e[4] = {v[B], v[B + 2 * S], v[B + 4 * S], v[B + 6 * S]};
    float2 o[4] = {v[B + S], v[B + 3 * S], v[B + 5 * S], v[B + 7 * S]};
    dft4<0, 1, INV>(e);
    dft4<0, 1, INV>(o);
    o[1] = w16<2, INV>(o[1]);
    o[2] = w16<4, INV>(o[2]);
    o[3] = w16<6, INV>(o[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[B + k * S] = cadd(e[k], o[k]);
        v[B + (k + 4) * S] = csub(e[k], o[k]);
    }
}

// DFT-16 = radix-4 decimation in time: D_m = DFT4(x[m], x[m+4], x[m+8], x[m+12]);
// E_m[k1] = W16^(m k1) D_m[k1];  X[k1 + 4 k2] = DFT4 over m of E_m[k1].
template <int B, int S, bool INV>
__device__ __forceinline__ void dft16(float2* v) {
    float2 u[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) u[i] = v[B + i * S];
    dft4<0, 4, INV>(u);
    dft4<1, 4, INV>(u);
    dft4<2, 4, INV>(u);
    dft4<3, 4, INV>(u);
    // u[m + 4*k1] = D_m[k1]
    u[1 + 4 * 1] = w16<1, INV>(u[1 + 4 * 1]);
    u[1 + 4 * 2] = w16<2, INV>(u[1 + 4 * 2]);
    u[1 + 4 * 3] = w16<3, INV>(u[1 + 4 * 3]);
    u[2 + 4 * 1] = w16<2, INV>(u[2 + 4 * 1]);
    u[2 + 4 * 2] = w16<4, INV>(u[2 + 4 * 2]);
    u[2 + 4 * 3] = w16<6, INV>(u[2 + 4 * 3]);
    u[3 + 4 * 1] = w16<3, INV>(u[3 + 4 * 1]);
    u[3 + 4 * 2] = w16<6, INV>(u[3 + 4 * 2]);
    u[3 + 4 * 3] = w16<9, INV>(u[3 + 4 * 3]);
    dft4<0, 1, INV>(u);
    dft4<4, 1, INV>(u);
    dft4<8, 1, INV>(u);
    dft4<12, 1, INV>(u);
    // u[4*k1 + k2] = X[k1 + 4*k2]
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[B + (k1 + 4 * k2) * S] = u[4 * k1 + k2];
}

// ---- odd radices: direct evaluation with symmetric pairing -----------------
// X[k] = x0 + sum_{j=1}^{(R-1)/2} [ (x_j + x_{R-j}) cos(2 pi jk/R)
//                                  -/+ i (x_j - x_{R-j}) sin(2 pi jk/R) ]
// The cos/sin values are rounded mathematical constants of the radix.
template <int R>
struct OddRadix;
template <>
struct OddRadix<3> {
    static constexpr int H = 1;
    __host__ __device__ static constexpr float c(int j) { return -0.5f; }
    __host__ __device__ static constexpr float s(int j) { return 0.86602540378443864676f; }
};
template <>
struct OddRadix<5> {
    static constexpr int H = 2;
    // cos/sin(2 pi m/5), m = 1, 2
    __host__ __device__ static constexpr float c(int m) { return m == 1 ? 0.30901699437494742410f : -0.80901699437494742410f; }
    __host__ __device__ static constexpr float s(int m) { return m == 1 ? 0.95105651629515357212f : 0.58778525229247312917f; }
};
template <>
struct OddRadix<7> {
    static constexpr int H = 3;
    // cos/sin(2 pi m/7), m = 1, 2, 3
    __host__ __device__ static constexpr float c(int m) {
        return m == 1 ? 0.62348980185873353053f : (m == 2 ? -0.22252093395631440429f : -0.90096886790241912624f);
    }
    __host__ __device__ static constexpr float s(int m) {
        return m == 1 ? 0.78183148246802980871f : (m == 2 ? 0.97492791218182360702f : 0.43388373911755812048f);
    }
};

template <int R, int B, int S, bool INV>
__device__ __forceinline__ void dft_odd(float2* v) {
    using O = OddRadix<R>;
    constexpr int H = O::H;
    float2 sp[H], sm[H];
    const float2 x0 = v[B];
#pragma unroll
    for (int j = 1; j <= H; ++j) {
        sp[j - 1] = cadd(v[B + j * S], v[B + (R - j) * S]);
        sm[j - 1] = csub(v[B + j * S], v[B + (R - j) * S]);
    }
    float2 sum = x0;
#pragma unroll
    for (int j = 0; j < H; ++j) sum = cadd(sum, sp[j]);
    float2 out[R];
    out[0] = sum;
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        float2 a = x0, b = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 1; j <= H; ++j) {
            const int m = (j * k) % R;  // compile-time after unrolling
            const int mm = m <= H ? m : R - m;
            const float c = O::c(mm);
            const float sg = m <= H ? 1.f : -1.f;  // sin(2 pi m/R) = sg * s(mm)
            const float s = sg * O::s(mm);
            a.x = fmaf(sp[j - 1].x, c, a.x);
            a.y = fmaf(sp[j - 1].y, c, a.y);
            b.x = fmaf(sm[j - 1].x, s, b.x);
            b.y = fmaf(sm[j - 1].y, s, b.y);
        }
        // forward: X[k] = a - i b, X[R-k] = a + i b ; inverse swaps.
        const float2 mib = make_float2(b.y, -b.x);  // -i*b
        out[k] = INV ? csub(a, mib) : cadd(a, mib);
        out[R - k] = INV ? cadd(a, mib) : csub(a, mib);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) v[B + k * S] = out[k];
}

template <int R, int B, int S, bool INV>
__device__ __forceinline__ void dft(float2* v) {
    if constexpr (R == 1) {
    } else if constexpr (R == 2) dft2<B, S, INV>(v);
    else if constexpr (R == 4) dft4<B, S, INV>(v);
    else if constexpr (R == 8) dft8<B, S, INV>(v);
    else if constexpr (R == 16) dft16<B, S, INV>(v);
    else dft_odd<R, B, S, INV>(v);
}

}  // namespace b300fft
