// k_tc.cu -- plans and launches of the tensor-core radix-16 path (tc.cuh):
// N = 256 and 4096 in one CTA, N = 65536 as the four-step 256 x 256.
#include <cstdio>
#include <cstdlib>

#include "launch.h"
#include "plan.h"
#include "tc.cuh"

namespace b300fft {

namespace {

// Raise the shared-memory limits and size the persistent grids of the plan's
// kernels.
template <int MODE>
cudaError_t prep_mode(fft_plan_s* p) {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f, int bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    };
    set((const void*)k_tc_rows<8, 16, MODE, false>, TcRowsCfg<8, 16>::SMEM);
    set((const void*)k_tc_rows<8, 16, MODE, true>, TcRowsCfg<8, 16>::SMEM);
    set((const void*)k_tc_rows<12, 1, MODE, false>, TcRowsCfg<12, 1>::SMEM);
    set((const void*)k_tc_rows<12, 1, MODE, true>, TcRowsCfg<12, 1>::SMEM);
    set((const void*)k_tc_cols256<MODE, false>, tc_cols_smem());
    set((const void*)k_tc_cols256<MODE, true>, tc_cols_smem());
    set((const void*)k_tc_rowsT256<MODE, false>, tc_rowsT_smem());
    set((const void*)k_tc_rowsT256<MODE, true>, tc_rowsT_smem());
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // Persistent grids: SMs x the kernels' resident CTAs per SM (their launch
    // bounds; the occupancy query reports one per SM for these kernels, and
    // one per SM measured 1.7x slower).  B300FFT_TC_GRID overrides the CTAs
    // per SM (0: one CTA per work unit).
    const char* env = std::getenv("B300FFT_TC_GRID");
    const int per_sm = env && *env ? std::atoi(env) : -1;
    auto grid = [&](int resident) {
        p->tc_per_sm = per_sm > 0 ? per_sm : resident;
        return per_sm == 0 ? 0x7fffffff : sms * p->tc_per_sm;
    };
    if (p->logn_a == 8 || p->logn_a == 12) p->tc_grid[0] = grid(kTcRowsPerSm);
    if (p->logn_a == 16) {
        p->tc_grid[0] = grid(kTcColsPerSm);
        p->tc_grid[1] = grid(kTcRowsTPerSm);
    }
    return e;
}

inline unsigned clamp_grid(int64_t units, int slots) {
    return (unsigned)(units < slots ? units : slots);
}

template <int MODE>
cudaError_t launch_mode(const fft_plan_s* p, const float2* in, float2* out, bool inv, cudaStream_t st, int only) {
    const uint4* bm = reinterpret_cast<const uint4*>(p->d_aux) + (inv ? 256 : 0);
    const float2* tabs = p->d_tables;
    auto want = [only](int k) { return only < 0 || only == k; };
    if (p->logn_a == 8 || p->logn_a == 12) {
        if (!want(0) || p->batch <= 0) return cudaSuccess;
        if (p->logn_a == 8) {
            const unsigned g = clamp_grid((p->batch + 15) / 16, p->tc_grid[0]);
            if (inv)
                k_tc_rows<8, 16, MODE, true><<<g, 256, TcRowsCfg<8, 16>::SMEM, st>>>(in, out, p->batch, tabs,
                                                                                     p->d_status, bm);
            else
                k_tc_rows<8, 16, MODE, false><<<g, 256, TcRowsCfg<8, 16>::SMEM, st>>>(in, out, p->batch, tabs,
                                                                                      p->d_status, bm);
        } else {
            const unsigned g = clamp_grid(p->batch, p->tc_grid[0]);
            if (inv)
                k_tc_rows<12, 1, MODE, true><<<g, 256, TcRowsCfg<12, 1>::SMEM, st>>>(in, out, p->batch, tabs,
                                                                                    p->d_status, bm);
            else
                k_tc_rows<12, 1, MODE, false><<<g, 256, TcRowsCfg<12, 1>::SMEM, st>>>(in, out, p->batch, tabs,
                                                                                     p->d_status, bm);
        }
        return cudaGetLastError();
    }
    // 65536 = 256 (columns, stride 256) x 256 (rows, transposed store)
    const int64_t n = 65536, groups = 256 / 16;
    if (p->batch <= 0) return cudaSuccess;
    if (want(0)) {
        const int64_t units = groups * p->batch;
        const unsigned g = clamp_grid(units, p->tc_grid[0]);
        if (inv)
            k_tc_cols256<MODE, true><<<g, 256, tc_cols_smem(), st>>>(in, p->d_work, 256, groups, n, units, tabs,
                                                                     tabs + p->off_lo, tabs + p->off_hi, p->sh,
                                                                     p->d_status, bm);
        else
            k_tc_cols256<MODE, false><<<g, 256, tc_cols_smem(), st>>>(in, p->d_work, 256, groups, n, units, tabs,
                                                                      tabs + p->off_lo, tabs + p->off_hi, p->sh,
                                                                      p->d_status, bm);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (want(1)) {
        const int64_t units = p->batch * 256 / 16;
        const unsigned g = clamp_grid(units, p->tc_grid[1]);
        if (inv)
            k_tc_rowsT256<MODE, true><<<g, 256, tc_rowsT_smem(), st>>>(p->d_work, out, tabs, 256, units,
                                                                      p->d_status, bm);
        else
            k_tc_rowsT256<MODE, false><<<g, 256, tc_rowsT_smem(), st>>>(p->d_work, out, tabs, 256, units,
                                                                       p->d_status, bm);
    }
    return cudaGetLastError();
}

}  // namespace

// Tensor-core plans: 1-D, N in {256, 4096, 65536}.
fft_status build_tc_plan(fft_plan_s* p) {
    if (p->dims != 1) return FFT_ERR_UNSUPPORTED;
    const int64_t n = p->len[0];
    int logn = (n == 256) ? 8 : (n == 4096 ? 12 : (n == 65536 ? 16 : -1));
    if (logn < 0) return FFT_ERR_UNSUPPORTED;
    p->kind = PlanKind::TensorCore;
    p->logn_a = logn;
    // tables: radix-16 Stockham table of 256 (used by both four-step passes)
    // or of 4096; two-level W_65536 table for the four-step twiddle
    const int lt = logn == 12 ? 12 : 8;
    const size_t et = (size_t)pow2_table_entries(lt);
    p->off_a = 0;
    p->sh = 8;
    p->off_lo = et;
    p->off_hi = et + 256;
    if (cudaMalloc(&p->d_tables, sizeof(float2) * (et + 512)) != cudaSuccess) return FFT_ERR_ALLOC;
    if (gen_pow2_table(p->d_tables, lt, 0) != cudaSuccess) return FFT_ERR_CUDA;
    if (logn == 16) {
        if (gen_root_table(p->d_tables + p->off_lo, 256, 1, n, 0) != cudaSuccess) return FFT_ERR_CUDA;
        if (gen_root_table(p->d_tables + p->off_hi, 256, 256, n, 0) != cudaSuccess) return FFT_ERR_CUDA;
        p->work_bytes = (size_t)n * (size_t)p->batch * sizeof(float2);
        if (cudaMalloc(&p->d_work, p->work_bytes) != cudaSuccess) return FFT_ERR_ALLOC;
    }
    // B operands (DFT-16 embedding, hi+lo) for forward and inverse: 8 KB
    if (cudaMalloc(&p->d_aux, 8192) != cudaSuccess) return FFT_ERR_ALLOC;
    const bool bf = p->precision == FFT_TC_BF16 || p->precision == FFT_TC_BF16_PLAIN;
    uint8_t* bm = static_cast<uint8_t*>(p->d_aux);
    for (int d = 0; d < 2; ++d) {
        if (bf) k_tc_bmat<true><<<4, 256>>>(bm + 4096 * d, d);
        else k_tc_bmat<false><<<4, 256>>>(bm + 4096 * d, d);
    }
    if (cudaGetLastError() != cudaSuccess) return FFT_ERR_CUDA;
    cudaError_t e;
    switch (p->precision) {
        case FFT_TC_FP16: e = prep_mode<TC_FP16>(p); break;
        case FFT_TC_BF16: e = prep_mode<TC_BF16>(p); break;
        case FFT_TC_FP16_PLAIN: e = prep_mode<TC_FP16_PLAIN>(p); break;
        default: e = prep_mode<TC_BF16_PLAIN>(p); break;
    }
    if (e != cudaSuccess) return FFT_ERR_CUDA;
    p->kernels = logn == 16 ? 2 : 1;
    static const char* names[] = {"fp32", "fp16 hi+lo", "bf16 hi+lo", "fp16 plain", "bf16 plain"};
    std::snprintf(p->desc, sizeof p->desc, "tensor-core radix-16 (%s) N=2^%d %s, persistent grid=%d (%d per SM)",
                  names[p->precision], logn, logn == 16 ? "four-step 256x256" : "single CTA", p->tc_grid[0],
                  p->tc_per_sm);
    return FFT_OK;
}

fft_status exec_tc(fft_plan_s* p, const float2* in, float2* out, bool inv, cudaStream_t st, int only) {
    cudaError_t e;
    switch (p->precision) {
        case FFT_TC_FP16: e = launch_mode<TC_FP16>(p, in, out, inv, st, only); break;
        case FFT_TC_BF16: e = launch_mode<TC_BF16>(p, in, out, inv, st, only); break;
        case FFT_TC_FP16_PLAIN: e = launch_mode<TC_FP16_PLAIN>(p, in, out, inv, st, only); break;
        default: e = launch_mode<TC_BF16_PLAIN>(p, in, out, inv, st, only); break;
    }
    return e == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
}

}  // namespace b300fft
