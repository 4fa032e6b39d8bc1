// exec.cu -- fft_exec dispatch: enqueue the kernels of a plan on a stream.
#include "launch.h"
#include "plan.h"

namespace b300fft {

fft_status exec_plan(fft_plan_s* p, const float2* in, float2* out, bool inv, cudaStream_t st, int only) {
    cudaError_t e = cudaSuccess;
    auto want = [only](int k) { return only < 0 || only == k; };
    switch (p->kind) {
        case PlanKind::Rows:
            if (want(0)) e = launch_rows(p->logn_a, inv, false, in, out, p->batch, p->d_tables + p->off_a, 1, st);
            break;
        case PlanKind::FourStep: {
            const int64_t n1 = int64_t(1) << p->logn_a, n2 = int64_t(1) << p->logn_b;
            if (want(0))
                e = launch_cols(p->logn_a, p->cols_c, inv, true, in, p->d_work, n2, n2, n1 * n2, p->batch,
                                p->d_tables + p->off_a, p->d_tables + p->off_lo, p->d_tables + p->off_hi, p->sh, st);
            if (e == cudaSuccess && want(1))
                e = launch_rows(p->logn_b, inv, true, p->d_work, out, p->batch * n1, p->d_tables + p->off_b, n1, st);
            break;
        }
        case PlanKind::TwoD: {
            const int64_t h = p->len[0], w = p->len[1];
            if (want(0)) e = launch_rows(p->logn_a, inv, false, in, out, p->batch * h, p->d_tables + p->off_a, 1, st);
            if (e == cudaSuccess && want(1))
                e = launch_cols(p->logn_b, p->cols_c, inv, false, out, out, w, w, h * w, p->batch, p->d_tables + p->off_b,
                                nullptr, nullptr, 0, st);
            break;
        }
        default:
            return FFT_ERR_UNSUPPORTED;
    }
    return e == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
}

fft_status build_generic_1d(fft_plan_s*) { return FFT_ERR_UNSUPPORTED; }
fft_status build_tc_plan(fft_plan_s*) { return FFT_ERR_UNSUPPORTED; }

}  // namespace b300fft
