/* c_abi_demo.c -- the library used from plain C through include/fft.h and
 * the CUDA runtime only (no Python, no torch).
 *
 * 1. A batch of 8 transforms of N = 4096: transform t holds the pure tone
 *    x[n] = exp(2 pi i f_t n / N); its forward DFT (Sec. III-A, sign -) is
 *    N at bin f_t and 0 elsewhere.  The inverse of that spectrum is N * x.
 * 2. A 2-D plan 96 x 1000 on an impulse at (r0, c0): every output bin has
 *    modulus 1.
 * 3. Argument errors: a NULL pointer, a misaligned pointer and a destroyed
 *    handle come back as status values.
 * Exit status 0 when every check holds; the largest errors are printed.
 * Bounds: 1e-6 of N on every bin of the tone spectra, 4e-6 on every element
 * of the round trip (unit-modulus data; the per-transform relative L2 bar of
 * 1e-6 allows a few times that on the largest element), 2e-6 on the
 * modulus of every 2-D bin. */
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "fft.h"

#define CHECK(cond, msg)                                  \
    do {                                                  \
        if (!(cond)) {                                    \
            fprintf(stderr, "c_abi_demo: %s\n", msg);     \
            return 1;                                     \
        }                                                 \
    } while (0)

static const double kTwoPi = 6.283185307179586476925286766559;

int main(void) {
    enum { N = 4096, B = 8, H = 96, W = 1000 };
    const int64_t n = N;
    float *h = (float *)malloc(sizeof(float) * 2 * N * B);
    CHECK(h != NULL, "host allocation");
    for (int t = 0; t < B; ++t) {
        const int f = 37 * t + 5;
        for (int j = 0; j < N; ++j) {
            const double a = kTwoPi * (double)(((int64_t)f * j) % N) / N;
            h[2 * (t * N + j)] = (float)cos(a);
            h[2 * (t * N + j) + 1] = (float)sin(a);
        }
    }
    void *d_in = NULL, *d_out = NULL;
    CHECK(cudaMalloc(&d_in, sizeof(float) * 2 * N * B) == cudaSuccess, "cudaMalloc in");
    CHECK(cudaMalloc(&d_out, sizeof(float) * 2 * N * B) == cudaSuccess, "cudaMalloc out");
    CHECK(cudaMemcpy(d_in, h, sizeof(float) * 2 * N * B, cudaMemcpyHostToDevice) == cudaSuccess, "copy in");

    fft_plan p = fft_plan_create(1, &n, B, FFT_FP32);
    CHECK(p != NULL, fft_status_string(fft_last_error()));
    CHECK(fft_exec(p, d_in, d_out, FFT_FORWARD, NULL) == FFT_OK, "fft_exec forward");
    CHECK(cudaDeviceSynchronize() == cudaSuccess, "sync");
    CHECK(fft_plan_check(p) == FFT_OK, "device status");
    float *y = (float *)malloc(sizeof(float) * 2 * N * B);
    CHECK(y != NULL, "host allocation");
    CHECK(cudaMemcpy(y, d_out, sizeof(float) * 2 * N * B, cudaMemcpyDeviceToHost) == cudaSuccess, "copy out");
    double err = 0.0;
    for (int t = 0; t < B; ++t) {
        const int f = 37 * t + 5;
        for (int k = 0; k < N; ++k) {
            const double re = y[2 * (t * N + k)] - (k == f ? (double)N : 0.0), im = y[2 * (t * N + k) + 1];
            const double e = sqrt(re * re + im * im) / N;
            if (e > err) err = e;
        }
    }
    printf("tone spectrum max error / N: %.3e\n", err);
    CHECK(err <= 1e-6, "tone spectrum");

    /* inverse of the spectrum, in place: N * x */
    CHECK(fft_exec(p, d_out, d_out, FFT_INVERSE, NULL) == FFT_OK, "fft_exec inverse");
    CHECK(cudaMemcpy(y, d_out, sizeof(float) * 2 * N * B, cudaMemcpyDeviceToHost) == cudaSuccess, "copy out");
    double err2 = 0.0;
    for (int i = 0; i < N * B; ++i) {
        const double re = y[2 * i] / N - h[2 * i], im = y[2 * i + 1] / N - h[2 * i + 1];
        const double e = sqrt(re * re + im * im);
        if (e > err2) err2 = e;
    }
    printf("round trip max error: %.3e\n", err2);
    CHECK(err2 <= 4e-6, "round trip");

    /* argument errors */
    CHECK(fft_exec(p, NULL, d_out, FFT_FORWARD, NULL) == FFT_ERR_INVALID_ARG, "NULL input accepted");
    CHECK(fft_exec(p, (char *)d_in + 8, d_out, FFT_FORWARD, NULL) == FFT_ERR_MISALIGNED, "misaligned accepted");
    CHECK(fft_plan_destroy(p) == FFT_OK, "destroy");
    CHECK(fft_exec(p, d_in, d_out, FFT_FORWARD, NULL) == FFT_ERR_BAD_HANDLE, "destroyed handle accepted");

    /* 2-D impulse: |X[k1, k2]| = 1 everywhere */
    const int64_t hw[2] = {H, W};
    float *img = (float *)calloc(2 * H * W, sizeof(float));
    CHECK(img != NULL, "host allocation");
    img[2 * (17 * W + 333)] = 1.0f;
    void *d_img = NULL;
    CHECK(cudaMalloc(&d_img, sizeof(float) * 2 * H * W) == cudaSuccess, "cudaMalloc image");
    CHECK(cudaMemcpy(d_img, img, sizeof(float) * 2 * H * W, cudaMemcpyHostToDevice) == cudaSuccess, "copy image");
    fft_plan q = fft_plan_create(2, hw, 1, FFT_FP32);
    CHECK(q != NULL, fft_status_string(fft_last_error()));
    char desc[256];
    fft_plan_describe(q, desc, sizeof desc);
    printf("2-D plan: %s\n", desc);
    CHECK(fft_exec(q, d_img, d_img, FFT_FORWARD, NULL) == FFT_OK, "fft_exec 2-D");
    CHECK(cudaMemcpy(img, d_img, sizeof(float) * 2 * H * W, cudaMemcpyDeviceToHost) == cudaSuccess, "copy image");
    CHECK(fft_plan_check(q) == FFT_OK, "device status 2-D");
    double err3 = 0.0;
    for (int i = 0; i < H * W; ++i) {
        const double m = sqrt((double)img[2 * i] * img[2 * i] + (double)img[2 * i + 1] * img[2 * i + 1]);
        if (fabs(m - 1.0) > err3) err3 = fabs(m - 1.0);
    }
    printf("2-D impulse max | |X| - 1 |: %.3e\n", err3);
    CHECK(err3 <= 2e-6, "2-D impulse");
    CHECK(fft_plan_destroy(q) == FFT_OK, "destroy 2-D");

    cudaFree(d_in);
    cudaFree(d_out);
    cudaFree(d_img);
    free(h);
    free(y);
    free(img);
    printf("c_abi_demo: ok\n");
    return 0;
}
