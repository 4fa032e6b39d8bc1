// real.cu -- real-to-complex and complex-to-real transforms (half spectrum),
// built on the complex plans: a length-N real sequence is packed as the N/2
// complex values z[n] = x[2n] + i x[2n+1], transformed with the N/2-point
// C2C plan, and split into the N/2+1 non-redundant bins (the input of the
// paper's Sec. III-B image example is real, which this form exploits):
//     E[k] = (Z[k] + conj(Z[N/2-k])) / 2,   O[k] = (Z[k] - conj(Z[N/2-k])) / (2i)
//     X[k] = E[k] + W_N^k O[k],             k = 0 .. N/2   (Z[N/2] = Z[0]).
// The complex-to-real direction inverts the split (unnormalised, like the
// complex inverse: C2R(R2C(x)) = N x):
//     E[k] = X[k] + conj(X[N/2-k]),   O[k] = (X[k] - conj(X[N/2-k])) W_N^{-k}
//     Z[k] = E[k] + i O[k],  then the N/2-point inverse C2C, then unpack.
// The split twiddles W_N^k (k < N/2) are an FP64-built table.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>

#include "butterfly.cuh"
#include "launch.h"
#include "plan.h"
#include "stockham_pow2.cuh"

namespace b300fft {

// Fused forms for h = N/2 = 2^LOGN <= 4096 (one tile per transform, TPC
// transforms per 256-thread CTA): the split happens inside the tile after
// the last radix pass (Z[h-k] comes from the exchange buffer), the merge
// inside the tile before the first one -- one HBM round trip instead of two.
template <int LOGN, int TPC, bool C2R>
__global__ void __launch_bounds__(RowsCfg<LOGN, TPC>::THREADS) k_real_rows(const float2* __restrict__ in,
                                                                           float2* __restrict__ out, int64_t nrows,
                                                                           const float2* __restrict__ tw,
                                                                           const float2* __restrict__ w) {
    using PL = P2Plan<LOGN>;
    constexpr int h = PL::N, T = PL::T;
    static_assert(PL::NPASS >= 2, "the exchange buffer carries the mirrored bins");
    extern __shared__ float2 smem[];
    const int t = threadIdx.x & (T - 1), sub = threadIdx.x / T;
    const int64_t row = (int64_t)blockIdx.x * TPC + sub;
    const bool ok = row < nrows;
    float2* s = smem + sub * PL::PADDED;
    float2 v[PL::R];
    if constexpr (!C2R) {
        const float2* src = in + row * h;
#pragma unroll
        for (int i = 0; i < PL::R; ++i) v[i] = ok ? __ldcs(src + t + i * T) : make_float2(0.f, 0.f);
        run_passes<PL, 0, false, false, 1>(v, t, s, 0, tw);  // Z[t + i T]; the exchange area is free again
#pragma unroll
        for (int i = 0; i < PL::R; ++i) s[padi(t + i * T)] = v[i];
        __syncthreads();
        if (ok) {
            float2* dst = out + row * (h + 1);
#pragma unroll
            for (int i = 0; i < PL::R; ++i) {
                const int k = t + i * T;
                const float2 zk = v[i], zm = s[padi((h - k) & (h - 1))];
                const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
                const float2 o = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
                __stcs(dst + k, cadd(e, cmul(o, __ldg(w + k))));
            }
            if (t == 0) __stcs(dst + h, make_float2(v[0].x - v[0].y, 0.f));  // X[h] = E[0] - O[0]
        }
    } else {
        const float2* src = in + row * (h + 1);
#pragma unroll
        for (int i = 0; i < PL::R; ++i) {
            const int k = t + i * T;
            float2 z = make_float2(0.f, 0.f);
            if (ok) {
                const float2 xk = __ldg(src + k), xm = __ldg(src + h - k);
                const float2 e = make_float2(xk.x + xm.x, xk.y - xm.y);                       // X[k] + conj(X[h-k])
                const float2 o = cmulc(make_float2(xk.x - xm.x, xk.y + xm.y), __ldg(w + k));  // (X[k] - conj) W^-k
                z = make_float2(e.x - o.y, e.y + o.x);                                        // E + i O
            }
            v[i] = z;
        }
        run_passes<PL, 0, true, false, 1>(v, t, s, 0, tw);
        if (ok) {
            float2* dst = out + row * h;
#pragma unroll
            for (int i = 0; i < PL::R; ++i) __stcs(dst + t + i * T, v[i]);
        }
    }
}

namespace {
template <int LOGN>
cudaError_t real_rows_one(bool prep, bool c2r, const float2* in, float2* out, int64_t nrows, const float2* tw,
                          const float2* w, cudaStream_t st) {
    constexpr int TPC = (256 >> (LOGN - 4)) > 0 ? (256 >> (LOGN - 4)) : 1;  // 256 threads per CTA
    using CF = RowsCfg<LOGN, TPC>;
    if (prep) {
        cudaError_t e = cudaFuncSetAttribute(k_real_rows<LOGN, TPC, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_real_rows<LOGN, TPC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     CF::SMEM);
        return e;
    }
    if (nrows <= 0) return cudaSuccess;
    const int64_t g = (nrows + TPC - 1) / TPC;
    if (g > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (c2r) k_real_rows<LOGN, TPC, true><<<(unsigned)g, CF::THREADS, CF::SMEM, st>>>(in, out, nrows, tw, w);
    else k_real_rows<LOGN, TPC, false><<<(unsigned)g, CF::THREADS, CF::SMEM, st>>>(in, out, nrows, tw, w);
    return cudaGetLastError();
}

// log2 h with a fused kernel (one tile per transform, at least two passes)
cudaError_t real_rows(int logh, bool prep, bool c2r, const float2* in, float2* out, int64_t nrows, const float2* tw,
                      const float2* w, cudaStream_t st) {
    switch (logh) {
#define B300_C(L) \
    case L:       \
        return real_rows_one<L>(prep, c2r, in, out, nrows, tw, w, st);
        B300_C(5) B300_C(6) B300_C(7) B300_C(8) B300_C(9) B300_C(10) B300_C(11) B300_C(12)
#undef B300_C
        default:
            return cudaErrorInvalidValue;
    }
}
}  // namespace

// Z (batch x h, complex, natural order) -> X (batch x (h+1)); h = N/2.
__global__ void k_r2c_split(const float2* __restrict__ z, float2* __restrict__ x, int64_t h, int64_t batch,
                            const float2* __restrict__ w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = h / 2 + 1;  // pairs (k, h-k) for k = 0 .. h/2
    if (i >= per * batch) return;
    const int64_t b = i / per, k = i - b * per;
    const float2* zb = z + b * h;
    float2* xb = x + b * (h + 1);
    const float2 zk = zb[k == h ? 0 : k];
    const int64_t m = (h - k) % h;  // Z[h - k], with Z[h] = Z[0]
    const float2 zm = zb[m];
    // bin k
    {
        const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        const float2 o = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
        xb[k] = cadd(e, cmul(o, __ldg(w + k)));
    }
    // bin h - k (the mirrored pair), unless it is bin k itself
    if (h - k != k) {
        const int64_t k2 = h - k;
        const float2 a = zb[k2 == h ? 0 : k2], c = zb[(h - k2) % h];
        const float2 e = make_float2(0.5f * (a.x + c.x), 0.5f * (a.y - c.y));
        const float2 o = make_float2(0.5f * (a.y + c.y), -0.5f * (a.x - c.x));
        const float2 wk = k2 == h ? make_float2(-1.f, 0.f) : __ldg(w + k2);
        xb[k2] = cadd(e, cmul(o, wk));
    }
}

// X (batch x (h+1)) -> Z (batch x h): the pre-processing of the inverse.
__global__ void k_c2r_merge(const float2* __restrict__ x, float2* __restrict__ z, int64_t h, int64_t batch,
                            const float2* __restrict__ w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= h * batch) return;
    const int64_t b = i / h, k = i - b * h;
    const float2* xb = x + b * (h + 1);
    const float2 xk = xb[k], xm = xb[h - k];
    const float2 e = make_float2(xk.x + xm.x, xk.y - xm.y);                   // X[k] + conj(X[h-k])
    const float2 o = cmulc(make_float2(xk.x - xm.x, xk.y + xm.y), __ldg(w + k));  // (X[k] - conj(X[h-k])) W^-k
    z[b * h + k] = make_float2(e.x - o.y, e.y + o.x);                            // E + i O
}

namespace {
cudaError_t grid_launch(int64_t n, unsigned* g) {
    const int64_t blocks = (n + 255) / 256;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    *g = (unsigned)(blocks > 0 ? blocks : 1);
    return cudaSuccess;
}
}  // namespace

// Real plan: owns a complex plan of length N/2 (same batch) and the split table.
fft_status build_real_plan(fft_plan_s* p, int64_t n, int64_t batch) {
    if (n < 2 || (n & 1)) return FFT_ERR_UNSUPPORTED;
    const int64_t h = n / 2;
    const int64_t lens[1] = {h};
    p->inner = fft_plan_create(1, lens, batch, FFT_FP32);
    if (!p->inner) return fft_last_error();
    p->kind = PlanKind::Real;
    if (cudaMalloc(&p->d_tables, sizeof(float2) * (size_t)h) != cudaSuccess) return FFT_ERR_ALLOC;
    if (gen_root_table(p->d_tables, h, 1, n, 0) != cudaSuccess) return FFT_ERR_CUDA;  // W_N^k, k < N/2
    // complex scratch of N/2 per transform (the packed spectrum)
    p->work_bytes = sizeof(float2) * (size_t)h * (size_t)batch;
    if (cudaMalloc(&p->d_work, p->work_bytes) != cudaSuccess) return FFT_ERR_ALLOC;
    p->kernels = 1 + fft_plan_kernel_count(p->inner);
    char inner[200];
    fft_plan_describe(p->inner, inner, sizeof inner);
    // h = 2^5 .. 2^12 with the single-pass complex plan: the fused kernels
    const char* fz = std::getenv("B300FFT_REAL_FUSED");
    p->real_fused = (!fz || std::atoi(fz) != 0) && p->inner->kind == PlanKind::Rows && p->inner->logn_a >= 5 &&
                    p->inner->logn_a <= 12 &&
                    real_rows(p->inner->logn_a, true, false, nullptr, nullptr, 0, nullptr, nullptr, 0) == cudaSuccess;
    if (p->real_fused) {
        p->kernels = 1;
        std::snprintf(p->desc, sizeof p->desc, "real N=%lld fused (complex N/2 = 2^%d rows + split in one pass)",
                      (long long)n, p->inner->logn_a);
        return FFT_OK;
    }
    std::snprintf(p->desc, sizeof p->desc, "real N=%lld via complex N/2 [%s] + split", (long long)n, inner);
    return FFT_OK;
}

// forward: in = real [batch][N] (as floats), out = complex [batch][N/2+1]
// inverse: in = complex [batch][N/2+1], out = real [batch][N]
fft_status exec_real(fft_plan_s* p, const void* in, void* out, bool inv, cudaStream_t st) {
    const int64_t h = p->len[0] / 2, batch = p->batch;
    float2* z = p->d_work;
    unsigned g;
    if (p->real_fused && in != out) {  // in place: the two-pass form (a fused tile would overwrite unread rows)
        const fft_plan_s* q = p->inner;
        return real_rows(q->logn_a, false, inv, static_cast<const float2*>(in), static_cast<float2*>(out), batch,
                         q->d_tables + q->off_a, p->d_tables, st) == cudaSuccess
                   ? FFT_OK
                   : FFT_ERR_CUDA;
    }
    if (!inv) {
        // real x viewed as h complex values per transform (x[2n] + i x[2n+1])
        fft_status s = fft_exec(p->inner, in, z, FFT_FORWARD, st);
        if (s != FFT_OK) return s;
        if (grid_launch((h / 2 + 1) * batch, &g) != cudaSuccess) return FFT_ERR_CUDA;
        k_r2c_split<<<g, 256, 0, st>>>(z, static_cast<float2*>(out), h, batch, p->d_tables);
        return cudaGetLastError() == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
    }
    if (grid_launch(h * batch, &g) != cudaSuccess) return FFT_ERR_CUDA;
    k_c2r_merge<<<g, 256, 0, st>>>(static_cast<const float2*>(in), z, h, batch, p->d_tables);
    if (cudaGetLastError() != cudaSuccess) return FFT_ERR_CUDA;
    // inverse C2C of the merged spectrum; its complex output is the real result interleaved
    return fft_exec(p->inner, z, out, FFT_INVERSE, st);
}

}  // namespace b300fft
