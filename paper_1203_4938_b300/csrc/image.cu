// image.cu -- the GPU steps of the image example (Sec. III-B), fused into one
// pass over the pixels:
//   1. chroma + luminance: JFIF (ITU-R BT.601 full range) YCbCr of 8-bit RGB,
//        Y  = .299 R + .587 G + .114 B
//        Cb = 128 - .168736 R - .331264 G + .5 B
//        Cr = 128 + .5 R - .418688 G - .081312 B
//   2. chroma downscaled to a quarter of the pixels: mean of each 2x2 block;
//   3. directional derivative of Y along the unit vector (ux, uy):
//        ux dY/dx + uy dY/dy, central differences inside the image and
//        one-sided first differences on its border.
// The paper names the steps, not their formulas; the ones above are the
// standard chroma/luminance split with a 1/4-size chroma layer.
//
// One CTA makes a 32 x 128 output tile.  Each thread owns 2x2 pixel quads
// (h, w even, so a quad is wholly inside or outside the image): it loads the
// quad's two 6-byte row pieces with 16-bit loads, writes the four luminances
// to shared memory and the two chroma means straight to global memory.  The
// one-pixel luminance halo around the tile (border pixels clamped) is
// converted separately; after one barrier the tile writes Y and the
// derivative with 512-byte rows (16-byte stores when w % 4 == 0 and the
// outputs are 16-byte aligned).  HBM traffic per pixel: 3 bytes in,
// 4 + 4 + 2 x 1 bytes out (halo bytes are re-read from L2 by the
// neighbouring tiles).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fft.h"

namespace b300fft {

constexpr int kImgTW = 128, kImgTH = 32, kImgThreads = 256;

__device__ __forceinline__ float luma(float r, float g, float b) { return fmaf(0.299f, r, fmaf(0.587f, g, 0.114f * b)); }
__device__ __forceinline__ float chroma_b(float r, float g, float b) {
    return fmaf(-0.168736f, r, fmaf(-0.331264f, g, fmaf(0.5f, b, 128.0f)));
}
__device__ __forceinline__ float chroma_r(float r, float g, float b) {
    return fmaf(0.5f, r, fmaf(-0.418688f, g, fmaf(-0.081312f, b, 128.0f)));
}

template <bool VEC>
__global__ void __launch_bounds__(kImgThreads) k_image_steps(const uint8_t* __restrict__ rgb, int64_t h, int64_t w,
                                                             float ux, float uy, float* __restrict__ Y,
                                                             float* __restrict__ CB, float* __restrict__ CR,
                                                             float* __restrict__ D) {
    __shared__ float sy[kImgTH + 2][kImgTW + 3];  // luminance with a one-pixel halo (+1 pad)
    const int64_t img = blockIdx.z;
    const int64_t x0 = (int64_t)blockIdx.x * kImgTW, y0 = (int64_t)blockIdx.y * kImgTH;
    const uint8_t* src = rgb + img * h * w * 3;
    const int64_t h2 = h / 2, w2 = w / 2;
    float* cbo = CB + img * h2 * w2;
    float* cro = CR + img * h2 * w2;
    // steps 1 and 2 on the tile's quads: every load of the thread's quads is
    // issued first (24 16-bit loads in flight), then the arithmetic
    constexpr int QW = kImgTW / 2, NQ = (kImgTH / 2) * QW, KQ = NQ / kImgThreads;
    uint32_t raw[KQ][6];
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
        const int qd = threadIdx.x + k * kImgThreads;
        const int qy = qd / QW, qx = qd - qy * QW;
        const int64_t gy = y0 + 2 * qy, gx = x0 + 2 * qx;
        const bool in = gy < h && gx < w;
#pragma unroll
        for (int row = 0; row < 2; ++row) {
            // 6 bytes R G B R G B at an even byte offset: three 16-bit loads
            const uint16_t* p = reinterpret_cast<const uint16_t*>(src + ((gy + row) * w + gx) * 3);
#pragma unroll
            for (int q = 0; q < 3; ++q) raw[k][3 * row + q] = in ? (uint32_t)__ldg(p + q) : 0u;
        }
    }
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
        const int qd = threadIdx.x + k * kImgThreads;
        const int qy = qd / QW, qx = qd - qy * QW;
        const int64_t gy = y0 + 2 * qy, gx = x0 + 2 * qx;
        if (gy >= h || gx >= w) continue;
        float r[4], g[4], b[4];
#pragma unroll
        for (int row = 0; row < 2; ++row) {
            const uint32_t a0 = raw[k][3 * row], a1 = raw[k][3 * row + 1], a2 = raw[k][3 * row + 2];
            r[2 * row] = (float)(a0 & 255u);
            g[2 * row] = (float)(a0 >> 8);
            b[2 * row] = (float)(a1 & 255u);
            r[2 * row + 1] = (float)(a1 >> 8);
            g[2 * row + 1] = (float)(a2 & 255u);
            b[2 * row + 1] = (float)(a2 >> 8);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) sy[2 * qy + 1 + (i >> 1)][2 * qx + 1 + (i & 1)] = luma(r[i], g[i], b[i]);
        const float sb = (chroma_b(r[0], g[0], b[0]) + chroma_b(r[1], g[1], b[1])) +
                         (chroma_b(r[2], g[2], b[2]) + chroma_b(r[3], g[3], b[3]));
        const float sr = (chroma_r(r[0], g[0], b[0]) + chroma_r(r[1], g[1], b[1])) +
                         (chroma_r(r[2], g[2], b[2]) + chroma_r(r[3], g[3], b[3]));
        __stcs(cbo + (gy / 2) * w2 + gx / 2, 0.25f * sb);
        __stcs(cro + (gy / 2) * w2 + gx / 2, 0.25f * sr);
    }
    // luminance of the halo ring (clamped at the image border)
    constexpr int RING = 2 * (kImgTW + 2) + 2 * kImgTH;
    for (int q = threadIdx.x; q < RING; q += kImgThreads) {
        int ly, lx;
        if (q < 2 * (kImgTW + 2)) {
            ly = q < kImgTW + 2 ? 0 : kImgTH + 1;
            lx = q < kImgTW + 2 ? q : q - (kImgTW + 2);
        } else {
            const int t = q - 2 * (kImgTW + 2);
            ly = 1 + (t >> 1);
            lx = (t & 1) ? kImgTW + 1 : 0;
        }
        int64_t gy = y0 + ly - 1, gx = x0 + lx - 1;
        gy = gy < 0 ? 0 : (gy >= h ? h - 1 : gy);
        gx = gx < 0 ? 0 : (gx >= w ? w - 1 : gx);
        const uint8_t* p = src + (gy * w + gx) * 3;
        sy[ly][lx] = luma((float)__ldg(p), (float)__ldg(p + 1), (float)__ldg(p + 2));
    }
    __syncthreads();
    // Y and step 3
    float* yo = Y + img * h * w;
    float* dout = D + img * h * w;
    if constexpr (VEC) {  // w % 4 == 0, 16-byte aligned outputs: four pixels per thread and store
#pragma unroll
        for (int k = 0; k < kImgTH * kImgTW / 4 / kImgThreads; ++k) {
            const int q = threadIdx.x + k * kImgThreads;
            const int ly = q / (kImgTW / 4), lx = 4 * (q - ly * (kImgTW / 4));
            const int64_t gy = y0 + ly, gx = x0 + lx;
            if (gy >= h || gx >= w) continue;
            float row[6], up[4], dn[4];
#pragma unroll
            for (int i = 0; i < 6; ++i) row[i] = sy[ly + 1][lx + i];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                up[i] = sy[ly][lx + 1 + i];
                dn[i] = sy[ly + 2][lx + 1 + i];
            }
            float dv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float c = row[i + 1];
                float ddx = 0.5f * (row[i + 2] - row[i]);
                if (i == 0 && gx == 0) ddx = row[2] - c;
                if (i == 3 && gx + 3 == w - 1) ddx = c - row[3];
                const float ddy = gy == 0 ? dn[i] - c : (gy == h - 1 ? c - up[i] : 0.5f * (dn[i] - up[i]));
                dv[i] = fmaf(ux, ddx, uy * ddy);
            }
            __stcs(reinterpret_cast<float4*>(yo + gy * w + gx), make_float4(row[1], row[2], row[3], row[4]));
            __stcs(reinterpret_cast<float4*>(dout + gy * w + gx), make_float4(dv[0], dv[1], dv[2], dv[3]));
        }
        return;
    }
#pragma unroll 4
    for (int q = threadIdx.x; q < kImgTH * kImgTW; q += kImgThreads) {
        const int ly = q / kImgTW, lx = q - ly * kImgTW;
        const int64_t gy = y0 + ly, gx = x0 + lx;
        if (gy >= h || gx >= w) continue;
        const float c = sy[ly + 1][lx + 1];
        const float l = sy[ly + 1][lx], r = sy[ly + 1][lx + 2];
        const float u = sy[ly][lx + 1], dn = sy[ly + 2][lx + 1];
        const float ddx = gx == 0 ? r - c : (gx == w - 1 ? c - l : 0.5f * (r - l));
        const float ddy = gy == 0 ? dn - c : (gy == h - 1 ? c - u : 0.5f * (dn - u));
        __stcs(yo + gy * w + gx, c);
        __stcs(dout + gy * w + gx, fmaf(ux, ddx, uy * ddy));
    }
}

}  // namespace b300fft

using namespace b300fft;

extern "C" fft_status fft_image_steps(const void* rgb, int64_t batch, int64_t h, int64_t w, float ux, float uy,
                                      void* y, void* cb, void* cr, void* d, void* stream) {
    if (!rgb || !y || !cb || !cr || !d || batch < 1 || h < 2 || w < 2 || (h & 1) || (w & 1)) return FFT_ERR_INVALID_ARG;
    if (batch > 65535 || h > (int64_t(1) << 19) || w > (int64_t(1) << 24) || batch * h * w > (int64_t(1) << 36))
        return FFT_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(rgb) & 1) || (reinterpret_cast<uintptr_t>(y) & 3) ||
        (reinterpret_cast<uintptr_t>(cb) & 3) ||
        (reinterpret_cast<uintptr_t>(cr) & 3) || (reinterpret_cast<uintptr_t>(d) & 3))
        return FFT_ERR_MISALIGNED;
    const dim3 grid((unsigned)((w + kImgTW - 1) / kImgTW), (unsigned)((h + kImgTH - 1) / kImgTH), (unsigned)batch);
    const bool vec = (w % 4) == 0 && !(reinterpret_cast<uintptr_t>(y) & 15) && !(reinterpret_cast<uintptr_t>(d) & 15);
    auto kern = vec ? k_image_steps<true> : k_image_steps<false>;
    kern<<<grid, kImgThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const uint8_t*>(rgb), h, w, ux, uy, static_cast<float*>(y), static_cast<float*>(cb),
        static_cast<float*>(cr), static_cast<float*>(d));
    return cudaGetLastError() == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
}
